// Dispatch of the record-layout apply and small vector kernels.
#include "apply_impl.cuh"

namespace hdg {

cudaError_t launch_apply(Context* c, int p, int which, int prec, const void* v, const void* cvec, void* y,
                         double alpha, double beta, int nrhs, cudaStream_t s) {
  PLevel& L = c->plev[p];
  const void* rec = nullptr;
  if (prec == HDG_PREC_FP64) rec = which ? (const void*)L.M64 : (const void*)L.S64;
  else if (prec == HDG_PREC_FP32) rec = which ? (const void*)L.M32 : (const void*)L.S32;
  else rec = which ? (const void*)L.M16 : (const void*)L.S16;
  if (!rec) return cudaErrorInvalidValue;
  ApplyArgs a{};
  a.rec = rec; a.v = v; a.cvec = cvec; a.y = y;
  a.alpha = alpha; a.beta = beta;
  a.nx = c->mesh.nx; a.ny = c->mesh.ny;
  a.spr = (c->mesh.nx + kSeg - 1) / kSeg;
  a.nseg = L.nseg; a.nrhs = nrhs; a.err = c->err_flag;
  if (prec == HDG_PREC_FP64) return apply_fp64(c, L.n1, a, s);
  if (prec == HDG_PREC_FP32) return apply_fp32(c, L.n1, a, s);
  return apply_bf16(c, L.n1, a, s);
}

__global__ void fill_kernel_d(double* p, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    p[t] = 0.0;
}
__global__ void fill_kernel_f(float* p, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    p[t] = 0.0f;
}

cudaError_t vec_fill(void* p, int prec, size_t n, cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  if (prec == HDG_PREC_FP64) fill_kernel_d<<<blocks, 256, 0, s>>>((double*)p, n);
  else fill_kernel_f<<<blocks, 256, 0, s>>>((float*)p, n);
  return cudaGetLastError();
}

}  // namespace hdg
