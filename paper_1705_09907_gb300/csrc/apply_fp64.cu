// Instantiations of the record-layout apply for fp64 storage.
#include "apply_impl.cuh"

namespace hdg {
cudaError_t apply_fp64(const Context* c, int n1, bool diff, const ApplyArgs& a, cudaStream_t s) {
  return diff ? apply_dispatch<double, double, double, true>(c, n1, a, s) : apply_dispatch<double, double, double, false>(c, n1, a, s);
}
}  // namespace hdg
