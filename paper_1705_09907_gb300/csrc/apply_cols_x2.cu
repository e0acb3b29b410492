// Instantiations of the column-batched record apply: double-float (hi, lo) storage with FP64 vectors and compensated FP32 arithmetic.
#include "apply_cols.cuh"

namespace hdg {
cudaError_t cols_x2(const Context* c, int n1, bool diff, const ColsArgs& a, cudaStream_t s) {
  (void)diff;   // ~48-bit arithmetic does not need the mean-subtracted form
  return cols_dispatch<float2, double, dfloat, false>(c, n1, a, s);
}
}  // namespace hdg
