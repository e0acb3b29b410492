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
// The x window of an item is loaded by five tensor-map (TMA) copies, one per
// edge row, into 128-byte-swizzled shared memory that the MMAs read directly.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "hdg_internal.h"

namespace hdg {

namespace {

constexpr int kTileM = 128;
constexpr int kTileN = 16;

struct BatchedArgs {
  const __nv_bfloat16* X;     // [ndof][nrhs]
  float* Y;                   // [ndof][nrhs]
  const __nv_bfloat16* B;     // [2][16][Kp] shared blocks, face type W then S (row n, column k)
  const double* kappa;        // per-element scale of the two halves of D (tau_K = kappa_K), or null (1)
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

// One bounded probe of an mbarrier phase. The suspend-time hint lets the
// hardware park the polling thread until the phase completes (or ~0.1 ms pass)
// instead of spinning: the three polling threads of a CTA would otherwise take
// most of the SM's issue slots from the drain warps.
__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity), "r"(100000u)
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

// 128-byte-swizzled K/MN-major descriptor (tcgen05 layout type 2): start,
// leading-byte offset = stride between 64-element atoms along M/N, stride-byte
// offset = stride between groups of 8 rows along K, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return smem_desc(addr, lbo, sbo) | ((uint64_t)2 << 61);
}

// x window of one segment and one group of 64 right-hand sides, read by the
// MMAs directly. 5 edge rows (V1: vertical edges of row j-1, V0: row j, Hm:
// horizontal edges of row j-1, H0: row j, H1: row j+1) x 10 slots (slot = i -
// (i0 - 1)); one slot holds one edge as 8 node rows (zero past k+1) x 64
// right-hand sides x 2 bytes = one 1 KB swizzle atom of an MN-major operand
// (a row's 16-byte chunks XOR-permuted by the row index, as the TMA copies
// write them). An MMA's M = 128 rows are two atoms (two neighbouring elements'
// faces, next slot: LBO = 1 KB); its K = 16 columns are two 8-row groups, the
// edges (W, E) of one element (next slot, SBO = 1 KB) or (S, N) (next row).
constexpr int kBS = 8;                      // elements per segment of this kernel
constexpr int kWRows = 5, kWSlots = kBS + 2;
constexpr uint32_t kSlotB = 1024u, kRowB = kWSlots * kSlotB;
constexpr uint32_t kWinTx = kWRows * kRowB; // bytes landed per window
enum { RV1 = 0, RV0 = 1, RHM = 2, RH0 = 3, RH1 = 4 };

// Tensor maps over X restricted to the interior edges, so that every boundary
// or off-mesh edge of a window is outside the map and lands as zeros:
//   tv: vertical edges i = 1..nx-1 of rows j = 0..ny-1, dims (rhs, node, i-1, j)
//   th: horizontal edges j = 1..ny-1, i = 0..nx-1, dims (rhs, node, i, j-1)
// The node box is 8 (past k+1 out of the map: zeros). One copy per edge row.
__device__ __forceinline__ void tma_load_row(unsigned char* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                             int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(su32(dst)), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void load_window(const BatchedArgs& a, const CUtensorMap* tv, const CUtensorMap* th,
                                            unsigned char* W, int seg, int chunk, uint64_t* bar) {
  const int j = seg / a.spr, i0 = (seg % a.spr) * kBS;
  const int x = chunk * 64;            // 128-byte aligned innermost coordinate
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(kWinTx) : "memory");
  // slot 0 is edge i0 - 1: vertical map coordinate i - 1 = i0 - 2
  tma_load_row(W + RV1 * kRowB, tv, x, 0, i0 - 2, j - 1, bar);
  tma_load_row(W + RV0 * kRowB, tv, x, 0, i0 - 2, j, bar);
  tma_load_row(W + RHM * kRowB, th, x, 0, i0 - 1, j - 2, bar);
  tma_load_row(W + RH0 * kRowB, th, x, 0, i0 - 1, j - 1, bar);
  tma_load_row(W + RH1 * kRowB, th, x, 0, i0 - 1, j, bar);
}

// The kBS tiles (kBS/2 W face pairs, kBS/2 S face pairs) x 4 K16 steps of one
// item into the accumulator columns `tm` (one thread), completion on `bar`.
__device__ __forceinline__ void issue_mmas(const unsigned char* W, const unsigned char* Bbuf, uint32_t tm,
                                           uint64_t* bar) {
  constexpr uint32_t tileB = kTileN * 64 * 2;
  constexpr int kTiles = kBS;
  // descriptors = fixed fields + (address >> 4); shared addresses stay below 256 KB,
  // so the 14-bit address field never carries into the next field
  const uint64_t dslot = smem_desc_sw128(0u, kSlotB, kSlotB), drow = smem_desc_sw128(0u, kSlotB, kRowB);
  const uint32_t wb4 = su32(W) >> 4;
  const uint64_t db0 = smem_desc(su32(Bbuf), 128u, 1024u), db1 = smem_desc(su32(Bbuf + tileB), 128u, 1024u);
#pragma unroll
  for (int t = 0; t < kTiles; ++t) {
    const int type = t / (kTiles / 2), L = 2 * (t % (kTiles / 2));
    const int sl = L + 1;                      // slot of the own element's W edge
    const uint64_t bd0 = type ? db1 : db0;
    uint64_t ad[4];
    ad[0] = dslot + wb4 + (uint32_t)(RV0 * kWSlots + sl) * (kSlotB >> 4);   // own W, E
    ad[1] = drow + wb4 + (uint32_t)(RH0 * kWSlots + sl) * (kSlotB >> 4);    // own S, N (N: next row)
    if (type == 0) {                                                         // west neighbour
      ad[2] = dslot + wb4 + (uint32_t)(RV0 * kWSlots + sl - 1) * (kSlotB >> 4);
      ad[3] = drow + wb4 + (uint32_t)(RH0 * kWSlots + sl - 1) * (kSlotB >> 4);
    } else {                                                                 // south neighbour
      ad[2] = dslot + wb4 + (uint32_t)(RV1 * kWSlots + sl) * (kSlotB >> 4);
      ad[3] = drow + wb4 + (uint32_t)(RHM * kWSlots + sl) * (kSlotB >> 4);
    }
    const uint32_t dcol = tm + (uint32_t)(t * kTileN);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const uint64_t bd = bd0 + (uint32_t)p * 16u;            // next 256 bytes of B
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dcol),
          "l"(ad[p]), "l"(bd), "r"(kIdesc), "r"(p > 0 ? 1u : 0u)
          : "memory");
    }
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

// Epilogue of one item: warp w reads lanes 32w..32w+31 of every tile from the
// accumulator columns `tm` and writes the owned faces' outputs (contiguous runs
// of 32 right-hand sides).
__device__ __forceinline__ void drain_item(const BatchedArgs& a, uint32_t tm, int seg, int chunk, int warp,
                                           int lane, int tbeg, int tend) {
  constexpr int kTiles = kBS;
  const int n1 = a.n1;
  const int nx = a.nx, ny = a.ny, nv = (nx + 1) * ny;
  const int j = seg / a.spr, i0 = (seg % a.spr) * kBS;
  const int mrow = (warp & 3) * 32 + lane;                   // TMEM lane quadrant of this warp
  const int s = mrow >> 6, r = mrow & 63;
  float* ybase = a.Y + chunk * 64 + r;
  for (int t0 = tbeg; t0 < tend; t0 += 2) {
    // two tiles per wait: 32 columns of this warp's 32 lanes
    uint32_t v[32];
    const uint32_t taddr = tm + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(t0 * kTileN);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
          "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
          "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int tt = 0; tt < 2; ++tt) {
      const int t = t0 + tt;
      const uint32_t* vt = v + tt * kTileN;
      const int type = t / (kTiles / 2);
      const int i = i0 + 2 * (t % (kTiles / 2)) + s;
      if (i < nx) {
        const bool bndrow = type == 0 ? (i == 0) : (j == 0);
        const int eout = type == 0 ? i + (nx + 1) * j : nv + i + nx * j;
        // columns 0..7 hold the own element's part, 8..15 the neighbour's (west
        // for W faces, south for S faces); each is scaled by its element's kappa
        // when the blocks are kappa_K S_ref
        float so = 1.0f, sn = 1.0f;
        if (a.kappa && !bndrow) {
          so = (float)a.kappa[i + nx * j];
          sn = (float)a.kappa[type == 0 ? (i - 1) + nx * j : i + nx * (j - 1)];
        }
        // fixed-trip loops over the tile's columns keep v in registers; the
        // face's rows are nrhs apart from one base address
        float* yq = ybase + (size_t)eout * n1 * a.nrhs;
        const size_t rs = (size_t)a.nrhs;
#pragma unroll
        for (int q = 0; q < kTileN / 2; ++q)
          if (q < n1)
            yq[q * rs] = bndrow ? 0.0f : so * __uint_as_float(vt[q]) + sn * __uint_as_float(vt[kTileN / 2 + q]);
        if (type == 0 && i == nx - 1) {
          const int eb = nx + (nx + 1) * j;
          for (int q = 0; q < n1; ++q) ybase[((size_t)eb * n1 + q) * a.nrhs] = 0.0f;
        }
        if (type == 1 && j == ny - 1) {
          const int eb = nv + i + nx * ny;
          for (int q = 0; q < n1; ++q) ybase[((size_t)eb * n1 + q) * a.nrhs] = 0.0f;
        }
      }
    }
  }
}

// Persistent CTAs with warp-specialized roles and a two-deep pipeline over items
// (segment x 64 right-hand sides):
//   warp 8 (one thread) loads window n%2 with five TMA copies that complete on
//     full[n%2] (expect-tx of the whole window; off-map parts land as zeros);
//   warp 9 (one thread) waits for full[n%2], issues the item's 32 MMAs into
//     accumulator n%2 and commits them to mma_done[n%2];
//   drain warps 0..7 wait for mma_done[n%2] and write the item's faces (warp w
//     reads TMEM lane quadrant w%4, tiles 4(w/4) .. 4(w/4)+3), then release the
//     accumulator through tmem_free[n%2].
// A window is refilled only after the MMAs that read it completed, an accumulator
// only after it was drained. Every wait is bounded (1 s); a role whose wait runs
// out stops, and the others then run out of their own waits. Before the CTA
// exits after such a stop, the last copy and the last commit issued on each
// buffer get one more bounded wait, so nothing is left in flight.
constexpr int kDrainWarps = 8;
constexpr int kLoadWarp = kDrainWarps, kIssueWarp = kDrainWarps + 1;
constexpr int kSpecThreads = 32 * (kDrainWarps + 2);

__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__global__ void __launch_bounds__(kSpecThreads)
    batched_apply_kernel(BatchedArgs a, const __grid_constant__ CUtensorMap tv, const __grid_constant__ CUtensorMap th) {
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  // the swizzle atoms of the windows must start on 1 KB boundaries of the
  // shared address space: round the dynamic base up (1 KB of slack is requested)
  unsigned char* sm = sm_raw + ((1024u - (su32(sm_raw) & 1023u)) & 1023u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr uint32_t tileB = kTileN * 64 * 2;                // K = 64 (4 steps x 16)
  constexpr uint32_t winB = kWRows * kRowB;
  // windows [2][5][kWSlots][1 KB] at sm and sm + winB (1 KB aligned)
  unsigned char* Bbuf = sm + 2 * winB;                       // [2][tileB]
  uint64_t* full = reinterpret_cast<uint64_t*>(Bbuf + 2 * tileB);       // [2]
  uint64_t* mma_done = full + 2;                                          // [2]
  uint64_t* tmem_free = mma_done + 2;                                     // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tmem_free + 2);
  // [0] drain, [1] load, [2] issuer failed; [3], [4] commits issued per
  // accumulator; [5], [6] windows loaded per buffer
  volatile int* flags = reinterpret_cast<volatile int*>(tmem_slot + 1);
  constexpr int kCols = 2 * kBS * kTileN;                    // two accumulators of 8 tiles x 16 columns

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < 2; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(full + q)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(mma_done + q)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(tmem_free + q)), "r"(kDrainWarps) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int q = 0; q < 7; ++q) flags[q] = 0;
  }
  if (tid == 32 * kLoadWarp) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tv) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&th) : "memory");
  }
  // the shared blocks, K-major without swizzle (core matrices of 8 n x 16 bytes)
  for (int idx = tid; idx < 2 * kTileN * 64; idx += kSpecThreads) {
    const int t = idx / (kTileN * 64), rem = idx % (kTileN * 64);
    const int n = rem / 64, k = rem % 64;
    const uint32_t off = (uint32_t)(n >> 3) * 1024u + (uint32_t)(k >> 3) * 128u + (uint32_t)(n & 7) * 16u +
                         (uint32_t)(k & 7) * 2u;
    *reinterpret_cast<__nv_bfloat16*>(Bbuf + t * tileB + off) = a.B[idx];
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int chunks = a.nrhs / 64;
  const long items = (long)a.nseg * chunks;
  const long first = blockIdx.x, step = gridDim.x;

  if (warp < kDrainWarps) {
    // ---------------- drain ----------------
    unsigned pd0 = 0u, pd1 = 0u;
    const int tbeg = (warp >> 2) * (kBS / 2);
    long n = 0;
    for (long item = first; item < items; item += step, ++n) {
      const int buf = (int)(n & 1);
      if (tid == 0 && !mbar_wait_1s(mma_done + buf, buf ? pd1 : pd0)) flags[0] = 1;
      named_sync(1, 32 * kDrainWarps);
      if (flags[0]) break;
      if (buf) pd1 ^= 1u; else pd0 ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      drain_item(a, tmem + (uint32_t)(buf * kBS * kTileN), (int)(item / chunks), (int)(item % chunks), warp, lane,
                 tbeg, tbeg + kBS / 2);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(tmem_free + buf)) : "memory");
    }
  } else if (warp == kLoadWarp) {
    // ---------------- TMA loads ----------------
    if (lane == 0) {
      unsigned pd0 = 0u, pd1 = 0u;
      long n = 0;
      for (long item = first; item < items; item += step, ++n) {
        const int buf = (int)(n & 1);
        if (n >= 2) {      // window buf was read by item n-2's MMAs
          if (!mbar_wait_1s(mma_done + buf, buf ? pd1 : pd0)) { flags[1] = 1; break; }
          if (buf) pd1 ^= 1u; else pd0 ^= 1u;
        }
        load_window(a, &tv, &th, sm + (buf ? winB : 0u), (int)(item / chunks), (int)(item % chunks), full + buf);
        flags[5 + buf] = flags[5 + buf] + 1;
      }
    }
  } else if (warp == kIssueWarp && lane == 0) {
    // ---------------- MMA issue ----------------
    unsigned pf0 = 0u, pf1 = 0u, pt0 = 0u, pt1 = 0u;
    long n = 0;
    for (long item = first; item < items; item += step, ++n) {
      const int buf = (int)(n & 1);
      if (!mbar_wait_1s(full + buf, buf ? pf1 : pf0)) { flags[2] = 1; break; }
      if (buf) pf1 ^= 1u; else pf0 ^= 1u;
      if (n >= 2) {      // accumulator buf was drained
        if (!mbar_wait_1s(tmem_free + buf, buf ? pt1 : pt0)) { flags[2] = 1; break; }
        if (buf) pt1 ^= 1u; else pt0 ^= 1u;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      issue_mmas(sm + (buf ? winB : 0u), Bbuf, tmem + (uint32_t)(buf * kBS * kTileN), mma_done + buf);
      flags[3 + buf] = flags[3 + buf] + 1;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (flags[0] || flags[1] || flags[2]) {
    // a wait ran out: flag it, and give the last window copy and the last
    // commit issued on each buffer (at most one of each is outstanding) one more
    // bounded wait before the shared and tensor memory are released
    if (tid == 0) {
      atomicExch(a.err, 2);
      for (int q = 0; q < 2; ++q) {
        if (flags[5 + q] > 0) (void)mbar_wait_1s(full + q, (unsigned)((flags[5 + q] - 1) & 1));
        if (flags[3 + q] > 0) (void)mbar_wait_1s(mma_done + q, (unsigned)((flags[3 + q] - 1) & 1));
      }
    }
    __syncthreads();
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

// B blocks from the shared FP64 block S (element 0 of the finest level, times
// `scale`): type 0 (W faces): output row n < k+1 of the own part holds
// [S[W row n, :] on the own element's (W, E), (S, N) edges]; row 8 + n of the
// neighbour part holds [S[E row n, :] on the west neighbour's edges]; type 1 (S
// faces) the same with S / N rows and the south neighbour. All other entries
// are zero (rows past k+1, the own part on the neighbour's K steps and back).
__global__ void pack_shared_b_kernel(const double* __restrict__ S, int n1, double scale,
                                     __nv_bfloat16* __restrict__ B) {
  // B[type][n][k], k = step*16 + h*8 + node: step 0 own (W, E), 1 own (S, N),
  // 2 neighbour (W, E), 3 neighbour (S, N)
  const int m = 4 * n1;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 2 * kTileN * 64; idx += gridDim.x * blockDim.x) {
    const int t = idx / (kTileN * 64), rem = idx % (kTileN * 64);
    const int n = rem / 64, k = rem % 64;
    const int step = k >> 4, h = (k >> 3) & 1, nd = k & 7;
    const bool nb_part = n >= kTileN / 2;
    const int row = n & (kTileN / 2 - 1);
    double v = 0.0;
    if (row < n1 && nd < n1 && nb_part == (step >= 2)) {
      const int own_face = t == 0 ? 0 : 2, nb_face = t == 0 ? 1 : 3;
      const int row_face = step < 2 ? own_face : nb_face;          // rows of S used
      const int col_face = (step & 1) * 2 + h;                      // W, E, S, N
      v = scale * S[(size_t)(row_face * n1 + row) * m + col_face * n1 + nd];
    }
    B[idx] = __float2bfloat16_rn((float)v);
  }
}

}  // namespace

int shared_kp(int n1) { (void)n1; return 64; }

// The shared block of the tensor-core apply: S itself for a uniform kappa, or
// S_ref = S_0 / kappa_0 with tau_K = kappa_K (every S_K = kappa_K S_ref; the
// drain scales each element's part by its kappa). kappa0 is element 0's.
cudaError_t prepare_shared_blocks(Context* c, double kappa0, cudaStream_t s) {
  const int n1 = c->k + 1;
  if (n1 > kTileN / 2) return cudaSuccess;                    // degrees past 7: no shared-block apply
  HDG_CUDA_TRY(ctx_alloc(c, (void**)&c->shared_B, (size_t)2 * kTileN * 64 * sizeof(__nv_bfloat16)));
  c->shared_scaled = c->opt.tau_kappa != 0;
  pack_shared_b_kernel<<<8, 256, 0, s>>>(c->plev[c->k].Sdense, n1, c->shared_scaled ? 1.0 / kappa0 : 1.0,
                                         c->shared_B);
  return cudaGetLastError();
}

size_t batched_smem_bytes(int n1) {
  (void)n1;
  // windows, shared blocks, 6 mbarriers + TMEM slot + 7 flags, alignment slack
  return (size_t)2 * kWRows * kRowB + (size_t)2 * kTileN * 64 * 2 + 80 + 1024;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library), looked up once.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// The two interior-edge maps over X [ndof][nrhs] (BF16): see load_window.
static cudaError_t make_edge_maps(const Context* c, const void* X, int nrhs, CUtensorMap* tv, CUtensorMap* th) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const int nx = c->mesh.nx, ny = c->mesh.ny, n1 = c->k + 1;
  const cuuint64_t rowB = (cuuint64_t)nrhs * 2, edgeB = rowB * n1;
  const size_t nv = (size_t)(nx + 1) * ny;
  const cuuint32_t box[4] = {64, 8, (cuuint32_t)kWSlots, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  {
    char* base = (char*)X + edgeB;                                   // edge i = 1 of row 0
    const cuuint64_t dims[4] = {(cuuint64_t)nrhs, (cuuint64_t)n1, (cuuint64_t)(nx - 1), (cuuint64_t)ny};
    const cuuint64_t str[3] = {rowB, edgeB, edgeB * (cuuint64_t)(nx + 1)};
    if (enc(tv, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, str, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    char* base = (char*)X + edgeB * (cuuint64_t)(nv + (size_t)nx);  // horizontal edge row j = 1
    const cuuint64_t dims[4] = {(cuuint64_t)nrhs, (cuuint64_t)n1, (cuuint64_t)nx, (cuuint64_t)(ny - 1)};
    const cuuint64_t str[3] = {rowB, edgeB, edgeB * (cuuint64_t)nx};
    if (enc(th, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, str, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

cudaError_t launch_batched_apply(Context* c, const void* X, float* Y, int nrhs, cudaStream_t s) {
  BatchedArgs a{};
  a.X = (const __nv_bfloat16*)X; a.Y = Y; a.B = c->shared_B;
  a.kappa = c->shared_scaled ? c->kappa : nullptr;
  a.nx = c->mesh.nx; a.ny = c->mesh.ny; a.n1 = c->k + 1; a.Kp = shared_kp(a.n1);
  a.nrhs = nrhs; a.spr = (c->mesh.nx + kBS - 1) / kBS; a.nseg = a.spr * c->mesh.ny; a.err = c->err_flag;
  if (a.n1 > 8 || c->mesh.nx < 2 || c->mesh.ny < 2) return cudaErrorInvalidValue;
  alignas(64) CUtensorMap tv, th;
  HDG_CUDA_TRY(make_edge_maps(c, X, nrhs, &tv, &th));
  const size_t smem = batched_smem_bytes(a.n1);
  if ((size_t)c->smem_optin < smem) return cudaErrorInvalidValue;
  HDG_CUDA_TRY(cudaFuncSetAttribute(batched_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, c->smem_optin));
  const long items = (long)a.nseg * (nrhs / 64);
  // two resident CTAs per SM (256 TMEM columns and ~107 KB shared memory each)
  long blocks = (long)c->num_sms * 2;
  if (blocks > items) blocks = items;
  batched_apply_kernel<<<(int)blocks, kSpecThreads, smem, s>>>(a, tv, th);
  return cudaGetLastError();
}

}  // namespace hdg
