// Instantiations of the column-batched record apply: FP64 storage and vectors.
#include "apply_cols.cuh"

namespace hdg {
cudaError_t cols_fp64(const Context* c, int n1, bool diff, const ColsArgs& a, cudaStream_t s) {
  (void)diff;
  return cols_dispatch<double, double, double, false>(c, n1, a, s);
}
}  // namespace hdg
