// Shared-block batched trace apply on the 5th-generation tensor cores.
//
// With a uniform coefficient every element has the same condensed block S, so
// the assembly-free apply of Alg. 3 for nrhs right-hand sides becomes, face by
// face, a dense product with a shared factor:
//   y_e[a, r] = sum_c S[F rows][a, c] x_K[c, r] + sum_c S[F' rows][a, c] x_nb[c, r]
// (F = the face of K on e, F' = the opposite face in the neighbour nb). Written
// as D = A B with
//   A [M = 128 rows x K = 2m cols]: two faces of one type (W or S) times 64
//     right-hand sides, columns = the 2m gathered trace dofs of the element and
//     its neighbour (each column is 64 contiguous values of X, so A is MN-major);
//   B [K x N = 16]: the shared row blocks [S[F rows], S[F' rows]]^T (K-major,
//     zero-padded from k+1 to 16 columns), loaded once per CTA;
//   D [128 x 16] FP32 in tensor memory, read back with tcgen05.ld.
// X is BF16, Y FP32 (kind::f16 with BF16 operands, FP32 accumulation). One
// tcgen05.mma (M = 128, N = 16, K = 16) per 16 columns of K, issued by one
// thread; completion through tcgen05.commit on an mbarrier (bounded wait).
#include <cuda_bf16.h>

#include "hdg_internal.h"

namespace hdg {

namespace {

constexpr int kTilesPerBatch = 4;          // MMA tiles (face pairs) per batch
constexpr int kTileM = 128;
constexpr int kTileN = 16;
constexpr int kThreads = 128;

struct BatchedArgs {
  const __nv_bfloat16* X;     // [ndof][nrhs]
  float* Y;                   // [ndof][nrhs]
  const __nv_bfloat16* B;     // [2][16][Kp] shared blocks, face type W then S (row n, column k)
  int nx, ny, n1, Kp, nrhs, spr, nseg;
  int* err;
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start, leading-byte offset (between
// core matrices along K), stride-byte offset (between 8-row core-matrix groups
// along M/N), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3fff);
  d |= (uint64_t)((lbo >> 4) & 0x3fff) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3fff) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// kind::f16 instruction descriptor: D F32, A and B BF16, A MN-major, B K-major,
// N = 16, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((uint32_t)(kTileN >> 3) << 17) |
                            ((uint32_t)(kTileM >> 4) << 24);

__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_1s(uint64_t* bar, unsigned parity) {
  if (mbar_try(bar, parity)) return true;
  uint64_t t0;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t0));
  for (unsigned it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 63u) == 63u) {
      uint64_t t;
      asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
      if (t - t0 > 1000000000ull) return false;
    }
  }
}

// Offset of element (m, k) of an MN-major tile: core matrices of 8 k-rows x 16
// bytes (8 consecutive m), K-direction core matrices 128 bytes apart, M-direction
// groups of 8 m `sbo` bytes apart.
__device__ __forceinline__ uint32_t a_off(int m8, int k, uint32_t sbo) {
  return (uint32_t)m8 * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(k & 7) * 16u;
}

__global__ void __launch_bounds__(kThreads) batched_apply_kernel(BatchedArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Kp = a.Kp;                                      // padded K (multiple of 16)
  const uint32_t sboA = (uint32_t)(Kp / 8) * 128u;          // bytes between 8-row groups of A
  const uint32_t tileA = (uint32_t)kTileM * Kp * 2;         // bytes of one A tile
  const uint32_t sboB = (uint32_t)(Kp / 8) * 128u;
  const uint32_t tileB = (uint32_t)kTileN * Kp * 2;
  unsigned char* Abuf = sm;                                  // [kTilesPerBatch][tileA]
  unsigned char* Bbuf = sm + kTilesPerBatch * tileA;         // [2][tileB]
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bbuf + 2 * tileB);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);

  // tensor memory: kTilesPerBatch x 16 fp32 columns (64, a power of two >= 32)
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(kTilesPerBatch * kTileN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // shared blocks B (both face types) in the K-major core-matrix layout
  for (int idx = tid; idx < 2 * kTileN * Kp; idx += kThreads) {
    const int t = idx / (kTileN * Kp), rem = idx % (kTileN * Kp);
    const int n = rem / Kp, k = rem % Kp;
    const uint32_t off = (uint32_t)(n >> 3) * sboB + (uint32_t)(k >> 3) * 128u + (uint32_t)(n & 7) * 16u +
                         (uint32_t)(k & 7) * 2u;
    *reinterpret_cast<__nv_bfloat16*>(Bbuf + t * tileB + off) = a.B[idx];
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int n1 = a.n1, m = 4 * n1, twoM = 2 * m;
  const int nx = a.nx, ny = a.ny, nv = (nx + 1) * ny;
  const int chunks = a.nrhs / 64;
  const long items = (long)a.nseg * chunks * (2 * kSeg / 2 / kTilesPerBatch);   // batches of 4 tiles
  const int bps = kSeg / kTilesPerBatch;          // batches per segment (2 W + 2 S)
  unsigned phase = 0;
  bool failed = false;
  for (long item = blockIdx.x; item < items && !failed; item += gridDim.x) {
    const int batch = (int)(item % bps);
    const long rest = item / bps;
    const int chunk = (int)(rest % chunks);
    const int seg = (int)(rest / chunks);
    const int j = seg / a.spr, i0 = (seg % a.spr) * kSeg;
    const int type = batch >= bps / 2 ? 1 : 0;    // 0: W faces, 1: S faces
    const int pair0 = (batch % (bps / 2)) * kTilesPerBatch;   // first face pair of the batch
    // ---- gather A: 4 tiles x 2 faces x Kp columns x 8 groups of 8 rhs ----
    const int per_tile = 2 * Kp * 8;
    for (int idx = tid; idx < kTilesPerBatch * per_tile; idx += kThreads) {
      const int tl = idx / per_tile, rem = idx % per_tile;
      const int s = rem / (Kp * 8), rem2 = rem % (Kp * 8);
      const int k = rem2 >> 3, m8 = rem2 & 7;
      const int L = 2 * (pair0 + tl) + s;          // element lane in the segment
      const int i = i0 + L;
      unsigned char* dst = Abuf + tl * tileA + a_off(s * 8 + m8, k, sboA);
      bool valid = i < nx && k < twoM;
      int ki = i, kj = j;
      int c = k;
      if (k >= m) {                                // neighbour across the face
        c = k - m;
        if (type == 0) ki = i - 1; else kj = j - 1;
        if (ki < 0 || kj < 0) valid = false;
      }
      long row = -1;
      if (valid) {
        const int f = c / n1, nd = c % n1;
        int edge;
        bool bnd;
        if (f == 0) { edge = ki + (nx + 1) * kj; bnd = ki == 0; }
        else if (f == 1) { edge = ki + 1 + (nx + 1) * kj; bnd = ki == nx - 1; }
        else if (f == 2) { edge = nv + ki + nx * kj; bnd = kj == 0; }
        else { edge = nv + ki + nx * (kj + 1); bnd = kj == ny - 1; }
        if (!bnd) row = (long)edge * n1 + nd;
      }
      if (row >= 0) {
        const __nv_bfloat16* src = a.X + (size_t)row * a.nrhs + chunk * 64 + m8 * 8;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(dst)), "l"(src) : "memory");
      } else {
        *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- MMAs: one thread issues Kp/16 steps per tile, then commits ----
    if (tid == 0) {
      for (int tl = 0; tl < kTilesPerBatch; ++tl) {
        const uint32_t abase = su32(Abuf + tl * tileA), bbase = su32(Bbuf + type * tileB);
        const uint32_t dcol = tmem + (uint32_t)(tl * kTileN);
        for (int kk = 0; kk < Kp / 16; ++kk) {
          const uint64_t ad = smem_desc(abase + (uint32_t)kk * 256u, 128u, sboA);
          const uint64_t bd = smem_desc(bbase + (uint32_t)kk * 256u, 128u, sboB);
          const uint32_t acc = kk > 0 ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dcol),
              "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                   : "memory");
    }
    const bool ok = mbar_wait_1s(bar, phase);
    phase ^= 1u;
    // one decision for the whole CTA (each thread timed its own wait)
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(a.err, 2);
        (void)mbar_wait_1s(bar, phase ^ 1u);   // let issued MMAs land before the columns are freed
      }
      failed = true;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!failed) {
      // ---- epilogue: warp w reads lanes 32w..32w+31 (rows = 64 rhs of face s) ----
      const int mrow = warp * 32 + lane;
      const int s = mrow >> 6, r = mrow & 63;
      for (int tl = 0; tl < kTilesPerBatch; ++tl) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(tl * kTileN);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int L = 2 * (pair0 + tl) + s;
        const int i = i0 + L;
        if (i < nx) {
          const bool bndrow = type == 0 ? (i == 0) : (j == 0);
          const int eout = type == 0 ? i + (nx + 1) * j : nv + i + nx * j;
          float* y = a.Y + chunk * 64 + r;
          for (int q = 0; q < n1; ++q)
            y[((size_t)eout * n1 + q) * a.nrhs] = bndrow ? 0.0f : __uint_as_float(v[q]);
          // E / N domain-boundary edges have no owner: zero them
          if (type == 0 && i == nx - 1) {
            const int eb = nx + (nx + 1) * j;
            for (int q = 0; q < n1; ++q) y[((size_t)eb * n1 + q) * a.nrhs] = 0.0f;
          }
          if (type == 1 && j == ny - 1) {
            const int eb = nv + i + nx * ny;
            for (int q = 0; q < n1; ++q) y[((size_t)eb * n1 + q) * a.nrhs] = 0.0f;
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTilesPerBatch * kTileN)
                 : "memory");
}

// B blocks from the shared FP64 block S (element 0 of the finest level):
// type 0 (W faces): row n < k+1: [S[W row n, :], S[E row n, :]]; type 1 (S faces):
// [S[S row n, :], S[N row n, :]]; zero rows n >= k+1 and columns k >= 2m.
__global__ void pack_shared_b_kernel(const double* __restrict__ S, int n1, int Kp, __nv_bfloat16* __restrict__ B) {
  const int m = 4 * n1;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 2 * kTileN * Kp; idx += gridDim.x * blockDim.x) {
    const int t = idx / (kTileN * Kp), rem = idx % (kTileN * Kp);
    const int n = rem / Kp, k = rem % Kp;
    double v = 0.0;
    if (n < n1 && k < 2 * m) {
      const int own_face = t == 0 ? 0 : 2, nb_face = t == 0 ? 1 : 3;
      const int face = k < m ? own_face : nb_face;
      const int c = k < m ? k : k - m;
      v = S[(size_t)(face * n1 + n) * m + c];
    }
    B[idx] = __float2bfloat16_rn((float)v);
  }
}

}  // namespace

int shared_kp(int n1) { return ((8 * n1 + 15) / 16) * 16; }

cudaError_t prepare_shared_blocks(Context* c, cudaStream_t s) {
  const int n1 = c->k + 1, Kp = shared_kp(n1);
  HDG_CUDA_TRY(ctx_alloc(c, (void**)&c->shared_B, (size_t)2 * kTileN * Kp * sizeof(__nv_bfloat16)));
  pack_shared_b_kernel<<<8, 256, 0, s>>>(c->plev[c->k].Sdense, n1, Kp, c->shared_B);
  return cudaGetLastError();
}

size_t batched_smem_bytes(int n1) {
  const int Kp = shared_kp(n1);
  return (size_t)kTilesPerBatch * kTileM * Kp * 2 + (size_t)2 * kTileN * Kp * 2 + 16;
}

cudaError_t launch_batched_apply(Context* c, const void* X, float* Y, int nrhs, cudaStream_t s) {
  BatchedArgs a{};
  a.X = (const __nv_bfloat16*)X; a.Y = Y; a.B = c->shared_B;
  a.nx = c->mesh.nx; a.ny = c->mesh.ny; a.n1 = c->k + 1; a.Kp = shared_kp(a.n1);
  a.nrhs = nrhs; a.spr = (c->mesh.nx + kSeg - 1) / kSeg; a.nseg = a.spr * c->mesh.ny; a.err = c->err_flag;
  const size_t smem = batched_smem_bytes(a.n1);
  if ((size_t)c->smem_optin < smem) return cudaErrorInvalidValue;
  HDG_CUDA_TRY(cudaFuncSetAttribute(batched_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, c->smem_optin));
  const long items = (long)a.nseg * (nrhs / 64) * (kSeg / kTilesPerBatch);
  // up to 4 resident CTAs per SM (64 TMEM columns each, < 60 KB shared memory each)
  long blocks = (long)c->num_sms * 4;
  if (blocks > items) blocks = items;
  batched_apply_kernel<<<(int)blocks, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace hdg
