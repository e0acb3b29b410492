// Instantiations of the record-layout apply for fp32 storage.
#include "apply_impl.cuh"

namespace hdg {
cudaError_t apply_fp32(const Context* c, int n1, bool diff, const ApplyArgs& a, cudaStream_t s) {
  return diff ? apply_dispatch<float, float, float, true>(c, n1, a, s) : apply_dispatch<float, float, float, false>(c, n1, a, s);
}
}  // namespace hdg
