// Instantiations of the record-layout apply for double-float (hi, lo) storage
// with FP64 vectors and compensated FP32 arithmetic.
#include "apply_impl.cuh"

namespace hdg {
cudaError_t apply_x2(const Context* c, int n1, bool diff, const ApplyArgs& a, cudaStream_t s) {
  (void)diff;   // ~48-bit arithmetic does not need the mean-subtracted form
  return apply_dispatch<float2, double, dfloat, false>(c, n1, a, s);
}
}  // namespace hdg
