// Instantiations of the record-layout apply for bf16 storage.
#include "apply_impl.cuh"

namespace hdg {
cudaError_t apply_bf16(const Context* c, int n1, const ApplyArgs& a, cudaStream_t s) {
  return apply_dispatch<__nv_bfloat16, float, float>(c, n1, a, s);
}
}  // namespace hdg
