// Instantiations of the record-layout apply for fp32 storage.
#include "apply_impl.cuh"

namespace hdg {
cudaError_t apply_fp32(const Context* c, int n1, const ApplyArgs& a, cudaStream_t s) {
  return apply_dispatch<float, float, float>(c, n1, a, s);
}
}  // namespace hdg
