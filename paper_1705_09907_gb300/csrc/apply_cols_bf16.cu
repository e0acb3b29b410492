// Instantiations of the column-batched record apply: BF16 storage with FP32 vectors and accumulation.
#include "apply_cols.cuh"

namespace hdg {
cudaError_t cols_bf16(const Context* c, int n1, bool diff, const ColsArgs& a, cudaStream_t s) {
  return diff ? cols_dispatch<__nv_bfloat16, float, float, true>(c, n1, a, s)
              : cols_dispatch<__nv_bfloat16, float, float, false>(c, n1, a, s);
}
}  // namespace hdg
