// The trace apply over several independent meshes of uneven size and degree
// (each with its own context) in one launch per pass. The work of all instances
// forms one list (instance-major) and each CTA serves one entry of one
// instance, so small instances do not leave SMs idle behind large ones.
//  * reduced blocks (reduced = 1 on every context): the element pass and the
//    face pass of the reduced apply, two launches for the whole batch;
//  * dense owner records: one launch; each CTA bulk-copies one record segment
//    and runs the segment kernel's body for the instance's degree (4 warps, the
//    same arithmetic as the single-mesh segment kernel with 4 warps).
#include "apply_impl.cuh"
#include "reduced_impl.cuh"

namespace hdg {

namespace {

constexpr int kMaxInst = 16;
constexpr int kMultiN1Max = 6;             // degrees 0..5
constexpr int kMultiWarps = 4;

struct MultiArgs {
  ApplyArgs inst[kMaxInst];
  int n1[kMaxInst];
  int seg_off[kMaxInst + 1];               // prefix sums of the instances' segment counts
  int ninst;
  unsigned part_off;                       // byte offset of the partial sums (largest degree's stage)
  unsigned bar_off;                        // byte offset of the mbarrier
};

__host__ __device__ constexpr unsigned rec_bytes(int n1, unsigned w) { return 16u * n1 * n1 * kSeg * w; }

template <typename TS, typename TV, typename TA, bool DIFF>
__global__ void __launch_bounds__(32 * kMultiWarps) multi_apply_kernel(const __grid_constant__ MultiArgs a) {
  using TO = typename OutT<TA>::type;
  extern __shared__ __align__(128) unsigned char multi_smem[];
  TS* st = reinterpret_cast<TS*>(multi_smem);
  TO* part = reinterpret_cast<TO*>(multi_smem + a.part_off);
  uint64_t* bar = reinterpret_cast<uint64_t*>(multi_smem + a.bar_off);
  const int g = blockIdx.x;
  int q = 0;
  while (q + 1 < a.ninst && g >= a.seg_off[q + 1]) ++q;
  const int lseg = g - a.seg_off[q];
  const int n1 = a.n1[q];
  const ApplyArgs& ia = a.inst[q];
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned sb = rec_bytes(n1, (unsigned)sizeof(TS));
    mbar_expect_tx(bar, sb);
    bulk_load(st, (const unsigned char*)ia.rec + (size_t)lseg * sb, sb, bar);
  }
  switch (n1) {
    case 1: seg_body<1, TS, TV, TA, DIFF, kMultiWarps>(ia, lseg, st, part, bar); break;
    case 2: seg_body<2, TS, TV, TA, DIFF, kMultiWarps>(ia, lseg, st, part, bar); break;
    case 3: seg_body<3, TS, TV, TA, DIFF, kMultiWarps>(ia, lseg, st, part, bar); break;
    case 4: seg_body<4, TS, TV, TA, DIFF, kMultiWarps>(ia, lseg, st, part, bar); break;
    case 5: seg_body<5, TS, TV, TA, DIFF, kMultiWarps>(ia, lseg, st, part, bar); break;
    default: seg_body<6, TS, TV, TA, DIFF, kMultiWarps>(ia, lseg, st, part, bar); break;
  }
}

template <typename TS, typename TV, typename TA, bool DIFF>
cudaError_t multi_launch(Context* const* ctx, int n, const void* const* x, void* const* y, int prec,
                         cudaStream_t s) {
  using TO = typename OutT<TA>::type;
  MultiArgs a{};
  a.ninst = n;
  a.seg_off[0] = 0;
  int n1max = 1;
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
    n1max = L.n1 > n1max ? L.n1 : n1max;
  }
  // stage of the largest degree, then the partial sums, then the mbarrier
  a.part_off = rec_bytes(n1max, (unsigned)sizeof(TS));
  a.bar_off = a.part_off + (unsigned)(((size_t)kMultiWarps * n1max * 32 * sizeof(TO) + 15) / 16 * 16);
  const size_t smem = (size_t)a.bar_off + 16;
  Context* c0 = ctx[0];
  if ((size_t)c0->smem_optin < smem) return cudaErrorInvalidValue;
  auto kern = multi_apply_kernel<TS, TV, TA, DIFF>;
  HDG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, c0->smem_optin));
  const int total = a.seg_off[n];
  if (total <= 0) return cudaSuccess;
  kern<<<total, 32 * kMultiWarps, smem, s>>>(a);
  return cudaGetLastError();
}

// Contexts with reduced blocks: the two passes of the reduced apply, each one
// launch over all instances. The blocks of each instance start at a block
// boundary, so a CTA serves one instance and the per-instance arithmetic and
// results equal the instance's own apply.
struct MultiRed {
  red::RedArgs inst[kMaxInst];
  int n1[kMaxInst];
  int eblk[kMaxInst + 1];                  // prefix sums of element-pass CTAs
  int fblk[kMaxInst + 1];                  // prefix sums of face-pass CTAs
  int ninst;
};

__device__ __forceinline__ int find_inst(const int* off, int ninst, int g) {
  int q = 0;
  while (q + 1 < ninst && g >= off[q + 1]) ++q;
  return q;
}

template <typename TS, typename T, bool DIFF>
__global__ void __launch_bounds__(red::kElemThreads) multi_red_elem_kernel(const __grid_constant__ MultiRed m) {
  const int q = find_inst(m.eblk, m.ninst, blockIdx.x);
  const long K = (blockIdx.x - m.eblk[q]) * (long)red::kElemThreads + threadIdx.x;
  const red::RedArgs& a = m.inst[q];
  switch (m.n1[q]) {
    case 1: red::elem_body<1, TS, T, DIFF>(a, K); break;
    case 2: red::elem_body<2, TS, T, DIFF>(a, K); break;
    case 3: red::elem_body<3, TS, T, DIFF>(a, K); break;
    case 4: red::elem_body<4, TS, T, DIFF>(a, K); break;
    case 5: red::elem_body<5, TS, T, DIFF>(a, K); break;
    default: red::elem_body<6, TS, T, DIFF>(a, K); break;
  }
}

template <typename T>
__global__ void __launch_bounds__(red::kFaceThreads) multi_red_face_kernel(const __grid_constant__ MultiRed m) {
  __shared__ T sw[red::kFaceThreads * kMultiN1Max], ss[red::kFaceThreads * kMultiN1Max];
  const int q = find_inst(m.fblk, m.ninst, blockIdx.x);
  const long K0 = (blockIdx.x - m.fblk[q]) * (long)red::kFaceThreads;
  const red::RedArgs& a = m.inst[q];
  switch (m.n1[q]) {
    case 1: red::face_body<1, T>(a, K0, threadIdx.x, sw, ss); break;
    case 2: red::face_body<2, T>(a, K0, threadIdx.x, sw, ss); break;
    case 3: red::face_body<3, T>(a, K0, threadIdx.x, sw, ss); break;
    case 4: red::face_body<4, T>(a, K0, threadIdx.x, sw, ss); break;
    case 5: red::face_body<5, T>(a, K0, threadIdx.x, sw, ss); break;
    default: red::face_body<6, T>(a, K0, threadIdx.x, sw, ss); break;
  }
}

template <typename TS, typename T, bool DIFF>
cudaError_t multi_red_launch(Context* const* ctx, int n, const void* const* x, void* const* y, cudaStream_t s) {
  MultiRed m{};
  m.ninst = n;
  for (int q = 0; q < n; ++q) {
    Context* c = ctx[q];
    PLevel& L = c->plev[c->k];
    red::RedArgs& a = m.inst[q];
    a.R = sizeof(TS) == 8 ? (const void*)L.R64 : (const void*)L.R32;
    if (!a.R) return cudaErrorInvalidValue;
    a.v = x[q]; a.cvec = nullptr; a.y = y[q]; a.z = c->red_z;
    a.alpha = 1.0; a.beta = 0.0;
    a.nx = c->mesh.nx; a.ny = c->mesh.ny;
    m.n1[q] = L.n1;
    m.eblk[q + 1] = m.eblk[q] + (c->nel + red::kElemThreads - 1) / red::kElemThreads;
    m.fblk[q + 1] = m.fblk[q] + (c->nel + red::kFaceThreads - 1) / red::kFaceThreads;
  }
  multi_red_elem_kernel<TS, T, DIFF><<<m.eblk[n], red::kElemThreads, 0, s>>>(m);
  HDG_CUDA_TRY(cudaGetLastError());
  multi_red_face_kernel<T><<<m.fblk[n], red::kFaceThreads, 0, s>>>(m);
  return cudaGetLastError();
}

}  // namespace

// Validates and launches; all contexts must live on the current device and use
// degrees 0..5 (FP64 or FP32 blocks). When every context has the two-launch
// reduced blocks (reduced = 1) the apply is the reduced one, else the dense
// owner-record one.
int apply_multi(Context* const* ctx, int n, const void* const* x, void* const* y, int prec, cudaStream_t s) {
  if (n < 1 || n > kMaxInst || !ctx || !x || !y) return HDG_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HDG_ERR_CUDA;
  for (int q = 0; q < n; ++q) {
    if (!ctx[q] || !x[q] || !y[q] || x[q] == y[q]) return HDG_ERR_INVALID_ARG;
    if (ctx[q]->k > kMultiN1Max - 1 || ctx[q]->dev != dev) return HDG_ERR_INVALID_ARG;
    if (prec != HDG_PREC_FP64 && !ctx[q]->opt.mixed) return HDG_ERR_UNSUPPORTED;
  }
  bool all_reduced = true;
  for (int q = 0; q < n; ++q) all_reduced = all_reduced && ctx[q]->opt.reduced == 1;
  cudaError_t e;
  if (all_reduced) {
    if (prec == HDG_PREC_FP64) e = multi_red_launch<double, double, false>(ctx, n, x, y, s);
    else if (prec == HDG_PREC_FP32) e = multi_red_launch<float, float, true>(ctx, n, x, y, s);
    else return HDG_ERR_UNSUPPORTED;
  } else if (prec == HDG_PREC_FP64) {
    e = multi_launch<double, double, double, false>(ctx, n, x, y, prec, s);
  } else if (prec == HDG_PREC_FP32) {
    e = multi_launch<float, float, float, true>(ctx, n, x, y, prec, s);
  } else {
    return HDG_ERR_UNSUPPORTED;
  }
  if (e == cudaErrorInvalidValue) return HDG_ERR_INVALID_ARG;
  return e == cudaSuccess ? HDG_OK : HDG_ERR_CUDA;
}

}  // namespace hdg
