// Instantiations of the column-batched record apply: FP32 storage and vectors.
#include "apply_cols.cuh"

namespace hdg {
cudaError_t cols_fp32(const Context* c, int n1, bool diff, const ColsArgs& a, cudaStream_t s) {
  return diff ? cols_dispatch<float, float, float, true>(c, n1, a, s)
              : cols_dispatch<float, float, float, false>(c, n1, a, s);
}
}  // namespace hdg
