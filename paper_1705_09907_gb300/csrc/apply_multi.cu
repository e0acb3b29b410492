// One persistent launch of the trace apply over several independent meshes of
// uneven size and degree (each with its own context). The segments of all
// instances form one work list (instance-major); every warp pair walks it with
// the same ring / window / partial-sum pipeline as the single-mesh apply and
// dispatches on the instance's degree per segment, so small instances do not
// leave the GPU idle behind large ones and there is one launch for the batch.
#include "apply_impl.cuh"

namespace hdg {

namespace {

constexpr int kMaxInst = 16;
constexpr int kMultiN1Max = 6;             // degrees 0..5

struct MultiArgs {
  ApplyArgs inst[kMaxInst];
  int n1[kMaxInst];
  int seg_off[kMaxInst + 1];               // prefix sums of the instances' segment counts
  int ninst;
  int stages;
  unsigned sbm, xwb, pb;                   // stage, window and partial-sum bytes (largest degree)
  int* err;
};


__host__ __device__ constexpr unsigned rec_bytes(int n1, unsigned w) { return 16u * n1 * n1 * kSeg * w; }

template <int N1, typename TS, typename TV, typename TA, bool DIFF>
__device__ __forceinline__ void multi_compute(const TS* st, const TV* xw, int lseg, int lane, int role,
                                              const ApplyArgs& ia, void* part_raw, int bar_id) {
  using TO = typename OutT<TA>::type;
  TO* part = reinterpret_cast<TO*>(part_raw);
  TA acc[N1];
  partial_segment<N1, TS, TV, TA, DIFF>(st, xw, lseg, lane, role, 0, ia, acc);
  if (role == 1) {
#pragma unroll
    for (int q = 0; q < N1; ++q) part[q * 32 + lane] = finish(acc[q]);
  }
  asm volatile("bar.sync %0, 64;" ::"r"(bar_id) : "memory");
  if (role == 0) {
    TO sum[N1];
#pragma unroll
    for (int q = 0; q < N1; ++q) sum[q] = finish(acc[q]) + part[q * 32 + lane];
    write_face<N1, TV, TO>(sum, lseg, lane, 0, ia);
  }
}

template <typename TV>
__device__ __forceinline__ void multi_window(TV* dst, int n1, int lseg, int lane, const ApplyArgs& ia) {
  const TV* v = (const TV*)ia.v;
  switch (n1) {
    case 1: issue_window<1, TV>(dst, v, lseg, lane, ia); break;
    case 2: issue_window<2, TV>(dst, v, lseg, lane, ia); break;
    case 3: issue_window<3, TV>(dst, v, lseg, lane, ia); break;
    case 4: issue_window<4, TV>(dst, v, lseg, lane, ia); break;
    case 5: issue_window<5, TV>(dst, v, lseg, lane, ia); break;
    default: issue_window<6, TV>(dst, v, lseg, lane, ia); break;
  }
}

__device__ __forceinline__ int find_inst(const MultiArgs& a, int g) {
  int q = 0;
  while (q + 1 < a.ninst && g >= a.seg_off[q + 1]) ++q;
  return q;
}

template <typename TS, typename TV, typename TA, bool DIFF>
__global__ void __launch_bounds__(512) multi_apply_kernel(const __grid_constant__ MultiArgs a) {
  using TO = typename OutT<TA>::type;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int np = blockDim.x >> 6;
  const int pr = w >> 1, role = w & 1;
  const int NS = a.stages;
  const size_t SBM = a.sbm, XWB = a.xwb, PB = a.pb;
  const size_t pair_bytes = (size_t)NS * (SBM + 2 * XWB + PB + 16);
  unsigned char* base = smem_raw + (size_t)pr * pair_bytes;
  unsigned char* ring = base;
  unsigned char* wins = base + (size_t)NS * SBM;
  unsigned char* parts = wins + (size_t)2 * NS * XWB;
  uint64_t* bars = reinterpret_cast<uint64_t*>(parts + (size_t)NS * PB);
  unsigned char* mywin = wins + (size_t)role * NS * XWB;
  const int gp = blockIdx.x * np + pr, tp = gridDim.x * np;
  const int total = a.seg_off[a.ninst];
  const int bar_id = 1 + pr;
  auto load_stage = [&](int s, int g) {
    const int q = find_inst(a, g);
    const int lseg = g - a.seg_off[q];
    const unsigned sb = rec_bytes(a.n1[q], (unsigned)sizeof(TS));
    const unsigned char* src = (const unsigned char*)a.inst[q].rec + (size_t)lseg * sb;
    mbar_expect_tx(&bars[s], sb);
    bulk_load(ring + (size_t)s * SBM, src, sb, &bars[s]);
  };
  if (role == 0 && lane == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int s = 0; s < NS; ++s) {
      const int g = gp + s * tp;
      if (g < total) load_stage(s, g);
    }
  }
  asm volatile("bar.sync %0, 64;" ::"r"(bar_id) : "memory");
  for (int s = 0; s < NS; ++s) {
    const int g = gp + s * tp;
    if (g < total) {
      const int q = find_inst(a, g);
      multi_window<TV>(reinterpret_cast<TV*>(mywin + (size_t)s * XWB), a.n1[q], g - a.seg_off[q], lane, a.inst[q]);
    } else {
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
  }
  for (int it = 0;; ++it) {
    const int g = gp + it * tp;
    if (g >= total) break;
    const int stg = it % NS;
    const unsigned par = (unsigned)((it / NS) & 1);
    window_wait(NS - 1);
    const bool ok = mbar_wait_bounded(&bars[stg], par);
    if (__any_sync(0xffffffffu, !ok)) {
      if (lane == 0) atomicExch(a.err, 2);
      asm volatile("cp.async.wait_all;" ::: "memory");
      for (int s = 1; s < NS; ++s) {
        const int it2 = it + s;
        if (gp + it2 * tp < total) (void)mbar_wait_bounded(&bars[it2 % NS], (unsigned)((it2 / NS) & 1));
      }
      return;
    }
    __syncwarp();
    const int q = find_inst(a, g);
    const int lseg = g - a.seg_off[q];
    const TS* st = reinterpret_cast<const TS*>(ring + (size_t)stg * SBM);
    const TV* xw = reinterpret_cast<const TV*>(mywin + (size_t)stg * XWB);
    void* part = parts + (size_t)stg * PB;
    switch (a.n1[q]) {
      case 1: multi_compute<1, TS, TV, TA, DIFF>(st, xw, lseg, lane, role, a.inst[q], part, bar_id); break;
      case 2: multi_compute<2, TS, TV, TA, DIFF>(st, xw, lseg, lane, role, a.inst[q], part, bar_id); break;
      case 3: multi_compute<3, TS, TV, TA, DIFF>(st, xw, lseg, lane, role, a.inst[q], part, bar_id); break;
      case 4: multi_compute<4, TS, TV, TA, DIFF>(st, xw, lseg, lane, role, a.inst[q], part, bar_id); break;
      case 5: multi_compute<5, TS, TV, TA, DIFF>(st, xw, lseg, lane, role, a.inst[q], part, bar_id); break;
      default: multi_compute<6, TS, TV, TA, DIFF>(st, xw, lseg, lane, role, a.inst[q], part, bar_id); break;
    }
    const int g2 = g + NS * tp;
    if (role == 0) {
      __syncwarp();
      if (lane == 0 && g2 < total) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        load_stage(stg, g2);
      }
    }
    __syncwarp();
    if (g2 < total) {
      const int q2 = find_inst(a, g2);
      multi_window<TV>(reinterpret_cast<TV*>(mywin + (size_t)stg * XWB), a.n1[q2], g2 - a.seg_off[q2], lane,
                       a.inst[q2]);
    } else {
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

template <typename TS, typename TV, typename TA, bool DIFF>
cudaError_t multi_launch(Context* const* ctx, int n, const void* const* x, void* const* y, int prec,
                         cudaStream_t s) {
  using TO = typename OutT<TA>::type;
  MultiArgs a{};
  a.ninst = n;
  a.err = ctx[0]->err_flag;
  a.seg_off[0] = 0;
  for (int q = 0; q < n; ++q) {
    Context* c = ctx[q];
    PLevel& L = c->plev[c->k];
    ApplyArgs& ia = a.inst[q];
    ia.rec = prec == HDG_PREC_FP64 ? (const void*)L.S64 : (const void*)L.S32;
    ia.v = x[q]; ia.cvec = nullptr; ia.y = y[q];
    ia.alpha = 1.0; ia.beta = 0.0;
    ia.nx = c->mesh.nx; ia.ny = c->mesh.ny; ia.spr = (c->mesh.nx + kSeg - 1) / kSeg;
    ia.nseg = L.nseg; ia.nrhs = 1; ia.err = c->err_flag;
    a.n1[q] = L.n1;
    a.seg_off[q + 1] = a.seg_off[q] + L.nseg;
  }
  Context* c0 = ctx[0];
  int n1max = 1;
  for (int q = 0; q < n; ++q) n1max = a.n1[q] > n1max ? a.n1[q] : n1max;
  a.sbm = rec_bytes(n1max, (unsigned)sizeof(TS));
  a.xwb = (unsigned)(((size_t)kWinRows * kWinSlots * n1max * sizeof(TV) + 15) / 16 * 16);
  a.pb = (unsigned)(((size_t)32 * n1max * sizeof(TO) + 15) / 16 * 16);
  const size_t per_stage = (size_t)a.sbm + 2 * a.xwb + a.pb + 16;
  // as in the single-mesh apply: as many warp pairs as fit (up to 4, one per
  // SM sub-partition pair), then a second stage per pair
  const int fit = (int)((220u * 1024u) / per_stage);
  int np = fit < 1 ? 1 : (fit > 4 ? 4 : fit);
  int ns = fit / np;
  if (ns > 2) ns = 2;
  if (ns < 1) ns = 1;
  a.stages = ns;
  const size_t smem = (size_t)np * ns * per_stage;
  if ((size_t)c0->smem_optin < smem) return cudaErrorInvalidValue;
  auto kern = multi_apply_kernel<TS, TV, TA, DIFF>;
  HDG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, c0->smem_optin));
  int blocks = c0->num_sms;
  const int need = (a.seg_off[n] + np - 1) / np;
  if (need < blocks) blocks = need > 0 ? need : 1;
  kern<<<blocks, 64 * np, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

// Validates and launches; all contexts must live on the current device and use
// degrees 0..5 (FP64 or FP32 blocks).
int apply_multi(Context* const* ctx, int n, const void* const* x, void* const* y, int prec, cudaStream_t s) {
  if (n < 1 || n > kMaxInst || !ctx || !x || !y) return HDG_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HDG_ERR_CUDA;
  for (int q = 0; q < n; ++q) {
    if (!ctx[q] || !x[q] || !y[q] || x[q] == y[q]) return HDG_ERR_INVALID_ARG;
    if (ctx[q]->k > kMultiN1Max - 1 || ctx[q]->dev != dev) return HDG_ERR_INVALID_ARG;
    if (prec != HDG_PREC_FP64 && !ctx[q]->opt.mixed) return HDG_ERR_UNSUPPORTED;
  }
  cudaError_t e;
  if (prec == HDG_PREC_FP64) e = multi_launch<double, double, double, false>(ctx, n, x, y, prec, s);
  else if (prec == HDG_PREC_FP32) e = multi_launch<float, float, float, true>(ctx, n, x, y, prec, s);
  else return HDG_ERR_UNSUPPORTED;
  if (e == cudaErrorInvalidValue) return HDG_ERR_INVALID_ARG;
  return e == cudaSuccess ? HDG_OK : HDG_ERR_CUDA;
}

}  // namespace hdg
