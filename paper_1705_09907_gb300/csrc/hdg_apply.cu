// Dispatch of the record-layout apply and small vector kernels.
#include "apply_cols.cuh"

namespace hdg {

cudaError_t launch_apply(Context* c, int p, int which, int prec, const void* v, const void* cvec, void* y,
                         double alpha, double beta, int nrhs, cudaStream_t s) {
  PLevel& L = c->plev[p];
  if (which == 0 && nrhs == 1 && c->opt.reduced)
    return launch_reduced_apply(c, p, prec, v, cvec, y, alpha, beta, s);
  // float Schwarz applies of one vector: the packed symmetric blocks
  if (which == 1 && nrhs == 1 && prec == HDG_PREC_FP32 && L.Mp32 && c->red_z)
    return launch_sym_schwarz(c, p, v, cvec, y, alpha, beta, s);
  // columns with double vectors: the reduced column kernels (FP64-pipe bound,
  // 2x fewer operations); float columns keep the dense column kernel, which
  // reads the blocks once for all columns and beats the reduced form's scratch
  // round trip when the pass is bandwidth bound (0.27 vs 0.47 ms at 256^2,
  // k = 5, 64 right-hand sides)
  if (which == 0 && nrhs > 1 && c->opt.reduced && c->cur_zb && prec_double(prec)) {
    const size_t need = (size_t)c->nel * L.m * nrhs * sizeof(double);
    if (need <= c->cur_zb_bytes)
      return launch_reduced_cols(c, p, prec, v, cvec, y, alpha, beta, nrhs, c->cur_zb, s);
  }
  const void* rec = nullptr;
  if (prec == HDG_PREC_FP64) rec = which ? (const void*)L.M64 : (const void*)L.S64;
  else if (prec == HDG_PREC_FP32) rec = which ? (const void*)L.M32 : (const void*)L.S32;
  else if (prec == HDG_PREC_F32X2) rec = which ? (const void*)L.M2 : (const void*)L.S2;
  else rec = which ? (const void*)L.M16 : (const void*)L.S16;
  if (!rec) return cudaErrorInvalidValue;
  // the condensed blocks have zero row sums: apply the low-precision copies to
  // x - mean(x) per element; FP64 and the Schwarz blocks use x directly
  const bool diff = (which == 0) && (prec == HDG_PREC_FP32 || prec == HDG_PREC_BF16);
  if (nrhs > 1) {   // right-hand-side-fastest columns: the column-batched kernel
    ColsArgs b{};
    b.rec = rec; b.v = v; b.cvec = cvec; b.y = y;
    b.alpha = alpha; b.beta = beta;
    b.nx = c->mesh.nx; b.ny = c->mesh.ny;
    b.spr = (c->mesh.nx + kSeg - 1) / kSeg;
    b.nseg = L.nseg; b.nb = nrhs;
    if (prec == HDG_PREC_FP64) return cols_fp64(c, L.n1, diff, b, s);
    if (prec == HDG_PREC_F32X2) return cols_x2(c, L.n1, diff, b, s);
    if (prec == HDG_PREC_FP32) return cols_fp32(c, L.n1, diff, b, s);
    return cols_bf16(c, L.n1, diff, b, s);
  }
  ApplyArgs a{};
  a.rec = rec; a.v = v; a.cvec = cvec; a.y = y;
  a.alpha = alpha; a.beta = beta;
  a.nx = c->mesh.nx; a.ny = c->mesh.ny;
  a.spr = (c->mesh.nx + kSeg - 1) / kSeg;
  a.nseg = L.nseg; a.nrhs = nrhs; a.err = c->err_flag;
  a.tune = L.tune[prec][which ? 1 : 0];
  if (prec == HDG_PREC_FP64) return apply_fp64(c, L.n1, diff, a, s);
  if (prec == HDG_PREC_F32X2) return apply_x2(c, L.n1, diff, a, s);
  if (prec == HDG_PREC_FP32) return apply_fp32(c, L.n1, diff, a, s);
  return apply_bf16(c, L.n1, diff, a, s);
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

namespace hdg {

// Set-up autotuner: for every level, precision and block kind, time the
// candidate launch shapes (warps per CTA x ring stages per warp, and the
// segment kernel with 8 / 4 / 2 warps) on a test vector and keep the fastest.
// The shapes differ only in the order in which the products are summed.
// bytes of one ring stage with its x windows and partial sums (matches
// stage_total_bytes in the launcher)
static unsigned stage_bytes_of(int n1, int prec) {
  const unsigned R = 16u * n1 * n1;
  const unsigned w = prec == HDG_PREC_FP64 || prec == HDG_PREC_F32X2 ? 8u : prec == HDG_PREC_FP32 ? 4u : 2u;
  const unsigned wv = prec_double(prec) ? 8u : 4u;
  const unsigned xwb = ((unsigned)kWinRows * kWinSlots * n1 * wv + 15u) / 16u * 16u;
  const unsigned pb = (32u * n1 * wv + 15u) / 16u * 16u;
  return R * kSeg * w + 2 * xwb + pb + 16;
}

__global__ void pattern_kernel(double* d, float* f, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const double v = 0.5 + (double)((t * 7919u) % 1009u) / 1009.0;
    d[t] = v;
    f[t] = (float)v;
  }
}

static size_t seg_bytes_of(int n1, int prec) {
  return (size_t)16 * n1 * n1 * kSeg * (prec == HDG_PREC_FP32 ? 4 : prec == HDG_PREC_BF16 ? 2 : 8) +
         (size_t)8 * n1 * 32 * (prec_double(prec) ? 8 : 4) + 16;
}

cudaError_t autotune_applies(Context* c, cudaStream_t s) {
  if (c->opt.autotune >= 2 && c->opt.autotune <= 4) {   // the segment kernel (8 / 4 / 2 warps) wherever it fits
    const int code = c->opt.autotune == 2 ? kTuneSeg : (c->opt.autotune == 3 ? (kTuneSeg | kTuneSeg4) : (kTuneSeg | kTuneSeg2));
    for (int p = 0; p <= c->k; ++p)
      for (int prec = 0; prec < 4; ++prec)
        for (int which = 0; which < 2; ++which)
          c->plev[p].tune[prec][which] = seg_bytes_of(c->plev[p].n1, prec) <= (size_t)c->smem_optin ? code : 0;
    return cudaSuccess;
  }
  const size_t n = (size_t)c->ndof;
  double *xd, *yd;
  float *xf, *yf;
  HDG_CUDA_TRY(cudaMallocAsync((void**)&xd, n * sizeof(double), s));
  HDG_CUDA_TRY(cudaMallocAsync((void**)&yd, n * sizeof(double), s));
  HDG_CUDA_TRY(cudaMallocAsync((void**)&xf, n * sizeof(float), s));
  HDG_CUDA_TRY(cudaMallocAsync((void**)&yf, n * sizeof(float), s));
  pattern_kernel<<<1024, 256, 0, s>>>(xd, xf, n);
  HDG_CUDA_TRY(cudaGetLastError());
  // Inside a V-cycle every level's blocks arrive cold (gigabytes are read
  // between two uses), so each candidate is timed after writing twice the L2
  // size: a level whose blocks fit in L2 is not tuned on cached data.
  int l2 = 0;
  HDG_CUDA_TRY(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->dev));
  const size_t flush_bytes = 2 * (size_t)(l2 > 0 ? l2 : (128 << 20));
  void* flush = nullptr;
  HDG_CUDA_TRY(cudaMallocAsync(&flush, flush_bytes, s));
  cudaEvent_t e0, e1;
  HDG_CUDA_TRY(cudaEventCreate(&e0));
  HDG_CUDA_TRY(cudaEventCreate(&e1));
  // summed device time of 3 cold launches of the current choice
  auto time_cold = [&](int p, int which, int prec, const void* x, void* y, float* out) -> cudaError_t {
    HDG_CUDA_TRY(launch_apply(c, p, which, prec, x, nullptr, y, 1.0, 0.0, 1, s));
    float sum = 0.f;
    for (int r = 0; r < 3; ++r) {
      HDG_CUDA_TRY(cudaMemsetAsync(flush, r, flush_bytes, s));
      HDG_CUDA_TRY(cudaEventRecord(e0, s));
      HDG_CUDA_TRY(launch_apply(c, p, which, prec, x, nullptr, y, 1.0, 0.0, 1, s));
      HDG_CUDA_TRY(cudaEventRecord(e1, s));
      HDG_CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      HDG_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      sum += ms;
    }
    *out = sum;
    return cudaSuccess;
  };
  const int precs[4] = {HDG_PREC_FP64, HDG_PREC_FP32, HDG_PREC_BF16, HDG_PREC_F32X2};
  for (int p = 0; p <= c->k; ++p) {
    PLevel& L = c->plev[p];
    for (int pi = 0; pi < 4; ++pi) {
      const int prec = precs[pi];
      if (prec != HDG_PREC_FP64 && !c->opt.mixed) continue;
      for (int which = 0; which < 2; ++which) {
        if (which == 1 && p == 0) continue;       // no Schwarz blocks at p = 0
        if (which == 0 && c->opt.reduced) continue;   // condensed blocks: the reduced apply
        const unsigned sb = stage_bytes_of(L.n1, prec);
        const int total = (int)((220u * 1024u) / sb);
        const void* x = prec_double(prec) ? (const void*)xd : (const void*)xf;
        void* y = prec_double(prec) ? (void*)yd : (void*)yf;
        float best = 1e30f;
        int best_tune = 0;
        const int nps[5] = {1, 2, 3, 4, 6};
        for (int wi = 0; wi < 5; ++wi)
          for (int ns = 1; ns <= 3; ++ns) {
            const int nw = nps[wi];                  // warp pairs
            if (nw * ns > total) continue;
            if (prec_double(prec) && nw > 4) continue;   // 8-byte blocks: at most 4 pairs
            L.tune[prec][which] = nw * 16 + ns;
            float ms = 0.f;
            HDG_CUDA_TRY(time_cold(p, which, prec, x, y, &ms));
            if (ms < best) { best = ms; best_tune = nw * 16 + ns; }
          }
        // the one-CTA-per-segment kernel, 8 / 4 / 2 warps (when its stage and
        // partial sums fit)
        if (seg_bytes_of(L.n1, prec) <= (size_t)c->smem_optin) {
          for (const int cand : {kTuneSeg, kTuneSeg | kTuneSeg4, kTuneSeg | kTuneSeg2}) {
            L.tune[prec][which] = cand;
            float ms = 0.f;
            HDG_CUDA_TRY(time_cold(p, which, prec, x, y, &ms));
            if (ms < best) { best = ms; best_tune = cand; }
          }
        }
        L.tune[prec][which] = best_tune;
      }
    }
  }
  HDG_CUDA_TRY(cudaFreeAsync(flush, s));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HDG_CUDA_TRY(cudaFreeAsync(xd, s));
  HDG_CUDA_TRY(cudaFreeAsync(yd, s));
  HDG_CUDA_TRY(cudaFreeAsync(xf, s));
  HDG_CUDA_TRY(cudaFreeAsync(yf, s));
  return cudaSuccess;
}

}  // namespace hdg
