// Instantiations of the record-layout apply for bf16 storage.
#include "apply_impl.cuh"

namespace hdg {
cudaError_t apply_bf16(const Context* c, int n1, bool diff, const ApplyArgs& a, cudaStream_t s) {
  return diff ? apply_dispatch<__nv_bfloat16, float, float, true>(c, n1, a, s) : apply_dispatch<__nv_bfloat16, float, float, false>(c, n1, a, s);
}
}  // namespace hdg
