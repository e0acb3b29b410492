// FP64 shared-block batched apply on the BF16 tensor cores by exact integer
// splitting (the Ozaki scheme), for a uniform coefficient: Y = A X with X, Y in
// FP64 [ndof][nrhs], every S_K equal to one block S.
//
// Splitting. Column c of X is scaled by 2^-e_c (e_c the smallest integer with
// |X[:, c]| < 2^e_c over the interior dofs) and written in fixed point with 56
// fraction bits, F = trunc(|x| 2^(56 - e_c)) (integer operations on the FP64
// bits), then cut into 8 slices of 7 bits, x = sign 2^e_c sum_t d_t 2^-7(t+1),
// d_t in [-127, 127]; S likewise with one exponent e_S for the whole block
// (set-up, host). Every slice is an integer that BF16 holds exactly, and for
// each group g = t + u the sum over the pairs (t, u) of the products of slices
// is an integer below 8 * 64 * 127^2 < 2^23, so the FP32 accumulation of the
// MMAs is exact. The result is
//   y = 2^(e_c + e_S - 63) sum_{g=0..7} D_g 2^7(7-g),   D_g = sum_{t+u=g} S_u X_t,
// the pairs with t + u >= 8 (below 2^-56 of the scale) dropped; the sum is
// formed as a 128-bit integer (two 64-bit words) and rounded once to FP64 with
// integer operations (no FP64 arithmetic on the slow FP64 pipe).
//
// Kernels: ozaki_exp_kernel (column exponents), ozaki_split_kernel (X -> 8 BF16
// slice arrays, [8][ndof][nrhs]), ozaki_apply_kernel (persistent CTAs, one per
// SM: items of 4 elements x 64 right-hand sides; for each slice t one TMA load
// of its x window (the interior-edge tensor maps of the BF16 apply, with the
// slice as a fifth dimension), then the MMAs of the pairs (t, u), u <= 7 - t,
// into the accumulator of group t + u (one MMA per tile and K step covers all
// pairs of a slice: the block slices are stacked along N); two accumulator sets
// of 4 tiles x 8 groups x 8 columns fill the 512 TMEM columns, so 8 drain warps
// combine the groups of one item and store FP64 Y while the next item's MMAs run).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "hdg_internal.h"

namespace hdg {

namespace {

constexpr int kOzSlices = 8, kOzBits = 7;
constexpr int kOzBS = 4;                           // elements per item
constexpr int kOzRows = 5, kOzSlots = kOzBS + 2;   // window: 5 edge rows x 6 slots
constexpr uint32_t kOzSlotB = 1024u, kOzRowB = kOzSlots * kOzSlotB, kOzWinB = kOzRows * kOzRowB;
constexpr int kOzTileN = 16;
enum { OV1 = 0, OV0 = 1, OHM = 2, OH0 = 3, OH1 = 4 };
constexpr int kOzDrainWarps = 8;
constexpr int kOzThreads = 32 * (kOzDrainWarps + 2);
constexpr int kOzGroupN = 8;                         // TMEM columns per group (k + 1 <= 8 outputs)
constexpr int kOzTileCols = kOzSlices * kOzGroupN;   // 64 TMEM columns per tile: 8 groups x 8
constexpr int kOzAccCols = 4 * kOzTileCols;          // one accumulator set: 4 tiles, 256 columns
constexpr int kOzCols = 2 * kOzAccCols;              // two sets (double-buffered): all 512 TMEM columns
constexpr int kOzBRows = 8 + kOzSlices * kOzGroupN;  // per face type: 8 zero rows, then slice u at 8 + 8u
constexpr uint32_t kOzTypeB = (uint32_t)(kOzBRows / 8) * 1024u;   // 9 core-matrix groups of 8 rows

struct OzArgs {
  double* Y;                  // [ndof][nrhs]
  const __nv_bfloat16* B;     // [8 slices][2 types][16][64] shared block slices
  const int* ecol;            // [nrhs] column exponents
  int eS;                     // exponent of the block
  int nx, ny, n1, nrhs, spr, nseg;
  int* err;
};

__device__ __forceinline__ uint32_t oz_su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t oz_desc(uint32_t addr, uint32_t lbo, uint32_t sbo, bool sw128) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3fff);
  d |= (uint64_t)((lbo >> 4) & 0x3fff) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3fff) << 32;
  d |= (uint64_t)1 << 46;
  if (sw128) d |= (uint64_t)2 << 61;
  return d;
}


__device__ __forceinline__ bool oz_try(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(oz_su32(bar)), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0;
}

// bounded wait (~1 s of device time)
__device__ __forceinline__ bool oz_wait(uint64_t* bar, unsigned parity) {
  if (oz_try(bar, parity)) return true;
  uint64_t t0;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t0));
  for (unsigned it = 0;; ++it) {
    if (oz_try(bar, parity)) return true;
    if ((it & 15u) == 15u) {
      uint64_t t;
      asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
      if (t - t0 > 1000000000ull) return false;
    }
  }
}

__device__ __forceinline__ void oz_named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// interior trace dof? (the trace is zero on boundary edges and they are ignored)
__device__ __forceinline__ bool oz_interior_dof(size_t dof, int n1, int nx, int ny) {
  const long e = (long)(dof / (size_t)n1);
  const long nv = (long)(nx + 1) * ny;
  if (e < nv) {
    const int i = (int)(e % (nx + 1));
    return i >= 1 && i <= nx - 1;
  }
  const int j = (int)((e - nv) / nx);
  return j >= 1 && j <= ny - 1;
}

// e_c = 1 + the largest unbiased exponent in column c over the interior dofs,
// so that |X[:, c]| < 2^e_c (entries below 2^-1022 count as zero). A thread
// takes 8 consecutive columns of a row (one 64-byte read); a block covers 256 / g
// rows at a time (g = nrhs / 8 threads per row), reduces in shared memory, and
// then issues one atomicMax per column.
__global__ void ozaki_exp_kernel(const double* __restrict__ X, size_t ndof, int nrhs, int n1, int nx, int ny,
                                 int* __restrict__ ecol) {
  __shared__ int red[256 * 8];
  const int g = nrhs / 8, tid = threadIdx.x;
  const int cg = tid % g, rl = tid / g, rows = 256 / g;
  int emax[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) emax[q] = -4000;
  if (rl < rows) {
    for (size_t r = (size_t)blockIdx.x * rows + rl; r < ndof; r += (size_t)gridDim.x * rows) {
      if (!oz_interior_dof(r, n1, nx, ny)) continue;
      // four 16-byte loads (X is 16-byte aligned)
      const longlong2* src = reinterpret_cast<const longlong2*>(X + r * nrhs + cg * 8);
      const longlong2 v0 = src[0], v1 = src[1], v2 = src[2], v3 = src[3];
      const long long b[8] = {v0.x, v0.y, v1.x, v1.y, v2.x, v2.y, v3.x, v3.y};
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int E = (int)((b[q] >> 52) & 0x7ff);
        if (E != 0) emax[q] = max(emax[q], E - 1022);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) red[tid * 8 + q] = emax[q];
  __syncthreads();
  // thread c < nrhs reduces column c over the block's row lanes
  for (int c = tid; c < nrhs; c += blockDim.x) {
    const int cgc = c / 8, q = c % 8;
    int e = -4000;
    for (int r = 0; r < rows; ++r) e = max(e, red[(r * g + cgc) * 8 + q]);
    atomicMax(&ecol[c], e);
  }
}

// X -> 8 BF16 slices S_t[dof][col] (integers in [-127, 127]) of the 56-bit
// fixed point F = trunc(|x| 2^(56 - e_c)), x ~ sign 2^e_c sum_t d_t 2^-7(t+1).
// A thread takes 8 consecutive columns of a row: one 64-byte read, then one
// 16-byte store per slice. Boundary dofs are not written (the tensor maps never
// read them).
__global__ void ozaki_split_kernel(const double* __restrict__ X, size_t ndof, int nrhs, int n1, int nx, int ny,
                                   const int* __restrict__ ecol, __nv_bfloat16* __restrict__ XS) {
  const int g = nrhs / 8;
  const size_t plane = ndof * (size_t)nrhs, groups = ndof * (size_t)g;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < groups;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t r = idx / (size_t)g;
    if (!oz_interior_dof(r, n1, nx, ny)) continue;
    const int c0 = (int)(idx - r * g) * 8;
    const size_t off = r * nrhs + c0;
    const longlong2* src = reinterpret_cast<const longlong2*>(X + off);   // X is 16-byte aligned
    const longlong2 v0 = src[0], v1 = src[1], v2 = src[2], v3 = src[3];
    const long long b[8] = {v0.x, v0.y, v1.x, v1.y, v2.x, v2.y, v3.x, v3.y};
    unsigned long long F[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int E = (int)((b[q] >> 52) & 0x7ff);
      F[q] = 0ull;
      if (E != 0) {
        const unsigned long long m = ((unsigned long long)b[q] & 0xfffffffffffffull) | (1ull << 52);
        const int s = E - 1019 - ecol[c0 + q];         // F = m 2^s, s <= 3
        if (s >= 0) F[q] = m << s;
        else if (s > -64) F[q] = m >> (-s);
      }
    }
#pragma unroll
    for (int t = 0; t < kOzSlices; ++t) {
      uint32_t w[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        uint32_t pair = 0u;
#pragma unroll
        for (int e2 = 0; e2 < 2; ++e2) {
          const int q = 2 * h + e2;
          const int d = (int)((F[q] >> (kOzBits * (kOzSlices - 1 - t))) & 127ull);
          const __nv_bfloat16 bv = __float2bfloat16_rn((float)(b[q] < 0 ? -d : d));
          pair |= (uint32_t)__bfloat16_as_ushort(bv) << (16 * e2);
        }
        w[h] = pair;
      }
      *reinterpret_cast<uint4*>(XS + (size_t)t * plane + off) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// value (hi 2^28 + lo) 2^e rounded to the nearest FP64 (ties to even), |hi|,
// |lo| < 2^46, by integer operations only: the 128-bit sum is normalised into a
// 64-bit window (top bit at 63) plus a sticky bit for what falls off, then
// rounded to 53 bits.
__device__ __forceinline__ double oz_to_double(long long hi, long long lo, int e) {
  // two's complement 128-bit T = hi 2^28 + lo as (w1, w0)
  unsigned long long w0 = ((unsigned long long)hi << 28) + (unsigned long long)lo;
  const unsigned long long carry = w0 < ((unsigned long long)hi << 28) ? 1ull : 0ull;
  unsigned long long w1 = (unsigned long long)(hi >> 36) + (unsigned long long)(lo >> 63) + carry;
  const bool neg = (long long)w1 < 0;
  if (neg) {                                        // magnitude
    w0 = ~w0 + 1ull;
    w1 = ~w1 + (w0 == 0ull ? 1ull : 0ull);
  }
  if (w1 == 0ull && w0 == 0ull) return 0.0;
  const int msb = w1 ? 127 - __clzll((long long)w1) : 63 - __clzll((long long)w0);
  const int sh = msb - 63;                          // right shift bringing the top bit to 63
  unsigned long long M;
  bool sticky = false;
  if (sh > 0) {
    M = (w1 << (64 - sh)) | (w0 >> sh);
    sticky = (w0 << (64 - sh)) != 0ull;
  } else {
    M = w0 << (-sh);
  }
  unsigned long long mant = M >> 11;                // 53 bits
  const unsigned long long rem = M & 0x7ffull;
  if (rem > 0x400ull || (rem == 0x400ull && (sticky || (mant & 1ull)))) ++mant;
  int ex = msb + e;                                 // unbiased exponent of the leading bit
  if (mant >> 53) { mant >>= 1; ++ex; }
  const int biased = ex + 1023;
  if (biased >= 2047)                               // overflow: infinity
    return __longlong_as_double((long long)(((unsigned long long)neg << 63) | 0x7ff0000000000000ull));
  if (biased <= 0) return neg ? -0.0 : 0.0;        // below the normal range: flushed
  return __longlong_as_double(
      (long long)(((unsigned long long)neg << 63) | ((unsigned long long)biased << 52) | (mant & 0xfffffffffffffull)));
}

// One slice window (segment seg, right-hand sides chunk*64.., slice t) by five
// TMA copies of the slice tensor maps (interior edges only; the rest reads as 0).
__device__ __forceinline__ void oz_load_window(const OzArgs& a, const CUtensorMap* tv, const CUtensorMap* th,
                                               unsigned char* W, int seg, int chunk, int t, uint64_t* bar) {
  const int j = seg / a.spr, i0 = (seg % a.spr) * kOzBS;
  const int x = chunk * 64;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(oz_su32(bar)), "r"(kOzWinB) : "memory");
  const int rows[5] = {OV1, OV0, OHM, OH0, OH1};
  const CUtensorMap* maps[5] = {tv, tv, th, th, th};
  const int c2[5] = {i0 - 2, i0 - 2, i0 - 1, i0 - 1, i0 - 1};
  const int c3[5] = {j - 1, j, j - 2, j - 1, j};
#pragma unroll
  for (int r = 0; r < 5; ++r)
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
        ::"r"(oz_su32(W + rows[r] * kOzRowB)), "l"((uint64_t)maps[r]), "r"(x), "r"(0), "r"(c2[r]), "r"(c3[r]), "r"(t),
        "r"(oz_su32(bar))
        : "memory");
}

// The MMAs of the pairs (t, u), u = 0 .. 7 - t, for one loaded slice window.
// The block slices are stacked along N behind 8 zero rows (slice u at rows
// 8 + 8u .. 8 + 8u + 7, the own element's and the neighbour's rows summed into
// the same 8 outputs), so one MMA writes pair (t, u) to TMEM columns 8 (t + u) of
// the tile's 64 (group g = t + u in the same place for every t): N = 8 (8 - t)
// from B row 8 at column 8t, or, when 8 - t is odd (N must be a multiple of 16),
// N = 8 (9 - t) from the zero rows at column 8 (t - 1), which adds 0 to the
// finished group t - 1. Per tile (2 W face pairs, 2 S face pairs) 4 K16 steps.
// Slice 0 (N = 64) writes every group first and overwrites.
__device__ __forceinline__ void oz_issue(const unsigned char* W, const unsigned char* Bbuf, uint32_t tmem, int t) {
  const uint64_t dslot = oz_desc(0u, kOzSlotB, kOzSlotB, true), drow = oz_desc(0u, kOzSlotB, kOzRowB, true);
  const uint32_t wb4 = oz_su32(W) >> 4;
  const bool odd = ((kOzSlices - t) & 1) != 0;
  const uint32_t ncols = (uint32_t)(kOzGroupN * (kOzSlices - t + (odd ? 1 : 0)));
  const uint32_t col0 = (uint32_t)(kOzGroupN * (t - (odd ? 1 : 0)));
  const uint32_t brow0 = odd ? 0u : 1024u;          // zero rows first, or slice 0 first
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((ncols >> 3) << 17) |
                         ((uint32_t)(128 >> 4) << 24);
#pragma unroll
  for (int tile = 0; tile < 4; ++tile) {
    const int type = tile >> 1, L = 2 * (tile & 1);
    const int sl = L + 1;                                     // slot of the own element's W edge
    const uint64_t bd0 = oz_desc(oz_su32(Bbuf + (uint32_t)type * kOzTypeB + brow0), 128u, 1024u, false);
    uint64_t ad[4];
    ad[0] = dslot + wb4 + (uint32_t)(OV0 * kOzSlots + sl) * (kOzSlotB >> 4);
    ad[1] = drow + wb4 + (uint32_t)(OH0 * kOzSlots + sl) * (kOzSlotB >> 4);
    if (type == 0) {
      ad[2] = dslot + wb4 + (uint32_t)(OV0 * kOzSlots + sl - 1) * (kOzSlotB >> 4);
      ad[3] = drow + wb4 + (uint32_t)(OH0 * kOzSlots + sl - 1) * (kOzSlotB >> 4);
    } else {
      ad[2] = dslot + wb4 + (uint32_t)(OV1 * kOzSlots + sl) * (kOzSlotB >> 4);
      ad[3] = drow + wb4 + (uint32_t)(OHM * kOzSlots + sl) * (kOzSlotB >> 4);
    }
    const uint32_t dcol = tmem + (uint32_t)(tile * kOzTileCols) + col0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const uint64_t bd = bd0 + (uint32_t)p * 16u;
      const uint32_t acc = (t > 0 || p > 0) ? 1u : 0u;
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dcol),
          "l"(ad[p]), "l"(bd), "r"(idesc), "r"(acc)
          : "memory");
    }
  }
}

// Drain of one item from the accumulator set at `tmem`: warp w reads TMEM lane
// quadrant w % 4 (M rows 32(w%4)..: face half s = row / 64, right-hand side
// row % 64) of tiles 2(w/4), 2(w/4)+1; per output it sums the groups as exact
// integers into T = sum_g D_g 2^7(7-g) (two 64-bit halves) and rounds
// T 2^(e_c + e_S - 63) to FP64.
__device__ __forceinline__ void oz_drain(const OzArgs& a, uint32_t tmem, int seg, int chunk, int warp, int lane) {
  const int n1 = a.n1;
  const int nx = a.nx, ny = a.ny, nv = (nx + 1) * ny;
  const int j = seg / a.spr, i0 = (seg % a.spr) * kOzBS;
  const int quad = warp & 3;
  const int mrow = quad * 32 + lane;
  const int s = mrow >> 6, r = mrow & 63;
  const int col = chunk * 64 + r;
  const int escale = a.ecol[col] + a.eS - 63;
  double* ybase = a.Y + col;
  for (int tt = 0; tt < 2; ++tt) {
    const int tile = 2 * (warp >> 2) + tt;
    // per output node: P[m] = D_2m 2^7 + D_2m+1 (exact in 32 bits: |D| < 2^23)
    int P[4][8];
#pragma unroll
    for (int half = 0; half < 2; ++half) {  // groups 4 half .. 4 half + 3: 32 columns
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(tile * kOzTileCols + 32 * half);
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
      for (int pp = 0; pp < 2; ++pp) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (q >= n1) break;
          // exact integers below 2^23 (own and neighbour parts summed by the MMA)
          const int d0 = __float2int_rn(__uint_as_float(v[kOzGroupN * (2 * pp) + q]));
          const int d1 = __float2int_rn(__uint_as_float(v[kOzGroupN * (2 * pp + 1) + q]));
          P[2 * half + pp][q] = d0 * (1 << kOzBits) + d1;
        }
      }
    }
    const int type = tile >> 1;
    const int i = i0 + 2 * (tile & 1) + s;
    if (i >= nx) continue;
    const bool bndrow = type == 0 ? (i == 0) : (j == 0);
    const int eout = type == 0 ? i + (nx + 1) * j : nv + i + nx * j;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (q >= n1) break;
      // T = sum_g D_g 2^7(7-g) = hi 2^28 + lo, hi = P0 2^14 + P1, lo = P2 2^14 + P3
      const long long hi = (long long)P[0][q] * (1ll << 14) + P[1][q];
      const long long lo = (long long)P[2][q] * (1ll << 14) + P[3][q];
      ybase[((size_t)eout * n1 + q) * a.nrhs] = bndrow ? 0.0 : oz_to_double(hi, lo, escale);
    }
    if (type == 0 && i == nx - 1) {
      const int eb = nx + (nx + 1) * j;
      for (int q = 0; q < n1; ++q) ybase[((size_t)eb * n1 + q) * a.nrhs] = 0.0;
    }
    if (type == 1 && j == ny - 1) {
      const int eb = nv + i + nx * ny;
      for (int q = 0; q < n1; ++q) ybase[((size_t)eb * n1 + q) * a.nrhs] = 0.0;
    }
  }
}

// Persistent CTAs (one per SM: all 512 TMEM columns, two accumulator sets of
// 4 tiles x 8 groups x 8 columns). Roles:
//   warp 8 (one thread): the slice windows, in order (item, t), into buffer
//     seq % 2 after the MMAs that read seq - 2 completed (window_free);
//   warp 9 (one thread): item n into accumulator set n % 2 once the drain of
//     item n - 2 released it; per slice waits for its window, issues its MMAs
//     and commits them to window_free[buf]; after slice 7 commits to
//     acc_full[n % 2];
//   drain warps 0..7: wait for acc_full[n % 2], combine and store, release
//     acc_free[n % 2] -- while the MMAs of item n + 1 run on the other set.
// Every wait is bounded (1 s); before exit after a give-up the last copy and
// commit on each barrier get one more bounded wait.
__global__ void __launch_bounds__(kOzThreads)
    ozaki_apply_kernel(OzArgs a, const __grid_constant__ CUtensorMap tv, const __grid_constant__ CUtensorMap th) {
  extern __shared__ __align__(1024) unsigned char oz_raw[];
  unsigned char* sm = oz_raw + ((1024u - (oz_su32(oz_raw) & 1023u)) & 1023u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* Bbuf = sm + 2 * kOzWinB;                                   // [2 types][kOzTypeB]
  uint64_t* full = reinterpret_cast<uint64_t*>(Bbuf + 2 * kOzTypeB);        // [2]
  uint64_t* wfree = full + 2;                                                // [2]
  uint64_t* acc_full = wfree + 2;                                            // [2]
  uint64_t* acc_free = acc_full + 2;                                         // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_free + 2);
  // [0] drain, [1] load, [2] issue gave up; [3] [4] loads per buffer; [5] [6]
  // window commits per buffer; [7] [8] accumulator commits per set
  volatile int* flags = reinterpret_cast<volatile int*>(tmem_slot + 1);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(oz_su32(tmem_slot)),
                 "r"(kOzCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < 2; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz_su32(full + q)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz_su32(wfree + q)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz_su32(acc_full + q)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(oz_su32(acc_free + q)), "r"(kOzDrainWarps)
                   : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int q = 0; q < 9; ++q) flags[q] = 0;
  }
  if (tid == 32 * kOzDrainWarps) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tv) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&th) : "memory");
  }
  // the block slices, K-major without swizzle (core matrices of 8 n x 16 bytes):
  // per face type 8 zero rows, then slice u at rows 8 + 8u .. 8 + 8u + 7
  for (uint32_t o = (uint32_t)tid * 16u; o < 2u * kOzTypeB; o += kOzThreads * 16u)
    *reinterpret_cast<uint4*>(Bbuf + o) = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  for (int idx = tid; idx < kOzSlices * 2 * kOzTileN * 64; idx += kOzThreads) {
    const int tb = idx / (kOzTileN * 64), rem = idx % (kOzTileN * 64);
    const int u = tb >> 1, type = tb & 1;
    const int nl = rem / 64, k = rem % 64;
    if (nl >= kOzGroupN) continue;                           // rows 8..15 of a slice are zero
    const int n = 8 + kOzGroupN * u + nl;
    const uint32_t off = (uint32_t)(n >> 3) * 1024u + (uint32_t)(k >> 3) * 128u + (uint32_t)(n & 7) * 16u +
                         (uint32_t)(k & 7) * 2u;
    *reinterpret_cast<__nv_bfloat16*>(Bbuf + (uint32_t)type * kOzTypeB + off) = a.B[idx];
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int chunks = a.nrhs / 64;
  const long items = (long)a.nseg * chunks;
  const long first = blockIdx.x, step = gridDim.x;

  if (warp < kOzDrainWarps) {
    unsigned pa[2] = {0u, 0u};
    long n = 0;
    for (long item = first; item < items; item += step, ++n) {
      const int set = (int)(n & 1);
      if (tid == 0 && !oz_wait(acc_full + set, pa[set])) flags[0] = 1;
      oz_named_sync(1, 32 * kOzDrainWarps);
      if (flags[0]) break;
      pa[set] ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      oz_drain(a, tmem + (uint32_t)(set * kOzAccCols), (int)(item / chunks), (int)(item % chunks), warp, lane);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(oz_su32(acc_free + set)) : "memory");
    }
  } else if (warp == kOzDrainWarps) {
    if (lane == 0) {
      unsigned pf[2] = {0u, 0u};
      long seq = 0;
      bool stop = false;
      for (long item = first; item < items && !stop; item += step) {
        for (int t = 0; t < kOzSlices; ++t, ++seq) {
          const int buf = (int)(seq & 1);
          if (seq >= 2) {     // the window was read by the MMAs of seq - 2
            if (!oz_wait(wfree + buf, pf[buf])) { flags[1] = 1; stop = true; break; }
            pf[buf] ^= 1u;
          }
          oz_load_window(a, &tv, &th, sm + (buf ? kOzWinB : 0u), (int)(item / chunks), (int)(item % chunks), t,
                         full + buf);
          flags[3 + buf] = flags[3 + buf] + 1;
        }
      }
    }
  } else if (lane == 0) {
    unsigned pw[2] = {0u, 0u}, pfree[2] = {0u, 0u};
    long seq = 0, n = 0;
    bool stop = false;
    for (long item = first; item < items && !stop; item += step, ++n) {
      const int set = (int)(n & 1);
      if (n >= 2) {           // the accumulators of item n - 2 were drained
        if (!oz_wait(acc_free + set, pfree[set])) { flags[2] = 1; break; }
        pfree[set] ^= 1u;
      }
      const uint32_t acc = tmem + (uint32_t)(set * kOzAccCols);
      for (int t = 0; t < kOzSlices; ++t, ++seq) {
        const int buf = (int)(seq & 1);
        if (!oz_wait(full + buf, pw[buf])) { flags[2] = 1; stop = true; break; }
        pw[buf] ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        oz_issue(sm + (buf ? kOzWinB : 0u), Bbuf, acc, t);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         oz_su32(wfree + buf))
                     : "memory");
        flags[5 + buf] = flags[5 + buf] + 1;
      }
      if (stop) break;
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       oz_su32(acc_full + set))
                   : "memory");
      flags[7 + set] = flags[7 + set] + 1;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (flags[0] || flags[1] || flags[2]) {
    if (tid == 0) {
      atomicExch(a.err, 2);
      for (int q = 0; q < 2; ++q) {
        if (flags[3 + q] > 0) (void)oz_wait(full + q, (unsigned)((flags[3 + q] - 1) & 1));
        if (flags[5 + q] > 0) (void)oz_wait(wfree + q, (unsigned)((flags[5 + q] - 1) & 1));
        if (flags[7 + q] > 0) (void)oz_wait(acc_full + q, (unsigned)((flags[7 + q] - 1) & 1));
      }
    }
    __syncthreads();
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kOzCols) : "memory");
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side

static PFN_cuTensorMapEncodeTiled_v12000 oz_encoder() {
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

// The BF16 block slices [8][2][16][64] of the shared block S (m x m, row-major,
// host) and its exponent: S / 2^e_S in 56-bit fixed point, 7 bits per slice.
// Row n < k+1 of face type 0 (W faces) holds, along K = own (W, E), own (S, N),
// neighbour (W, E), neighbour (S, N), the W row n of S on the own element's
// edges and the E row n on the west neighbour's (type 1: S / N rows, south
// neighbour), so one output column sums both elements' parts; rows 8..15 are 0.
static void oz_block_slices(const std::vector<double>& S, int n1, std::vector<uint16_t>& B, int& eS) {
  const int m = 4 * n1;
  double mx = 0.0;
  for (double v : S) mx = std::max(mx, std::fabs(v));
  int e = 0;
  if (mx > 0.0) std::frexp(mx, &e);                 // mx < 2^e
  eS = e;
  B.assign((size_t)kOzSlices * 2 * kOzTileN * 64, 0);
  for (int u = 0; u < kOzSlices; ++u)
    for (int ty = 0; ty < 2; ++ty)
      for (int n = 0; n < n1; ++n)
        for (int k = 0; k < 64; ++k) {
          const int step = k >> 4, h = (k >> 3) & 1, nd = k & 7;
          if (nd >= n1) continue;
          const int own_face = ty == 0 ? 0 : 2, nb_face = ty == 0 ? 1 : 3;
          const int row_face = step < 2 ? own_face : nb_face;
          const int col_face = (step & 1) * 2 + h;
          const double v = S[(size_t)(row_face * n1 + n) * m + col_face * n1 + nd];
          const unsigned long long F = (unsigned long long)std::ldexp(std::fabs(v), 56 - eS);   // truncates
          const int d = (int)((F >> (kOzBits * (kOzSlices - 1 - u))) & 127ull);
          const float f = (float)(v < 0 ? -d : d);      // an integer of at most 7 bits: exact in BF16
          uint32_t fb;
          std::memcpy(&fb, &f, sizeof(fb));
          B[(((size_t)u * 2 + ty) * kOzTileN + n) * 64 + k] = (uint16_t)(fb >> 16);
        }
}

cudaError_t prepare_ozaki_blocks(Context* c, cudaStream_t s) {
  const int n1 = c->k + 1, m = 4 * n1;
  if (n1 > kOzTileN / 2) return cudaSuccess;
  std::vector<double> S((size_t)m * m);
  HDG_CUDA_TRY(cudaMemcpyAsync(S.data(), c->plev[c->k].Sdense, S.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  HDG_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<uint16_t> B;
  oz_block_slices(S, n1, B, c->oz_eS);
  HDG_CUDA_TRY(ctx_alloc(c, (void**)&c->oz_B, B.size() * sizeof(uint16_t)));
  HDG_CUDA_TRY(cudaMemcpyAsync(c->oz_B, B.data(), B.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, s));
  return cudaStreamSynchronize(s);
}

static cudaError_t oz_maps(const Context* c, const void* XS, int nrhs, CUtensorMap* tv, CUtensorMap* th) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = oz_encoder();
  if (!enc) return cudaErrorNotSupported;
  const int nx = c->mesh.nx, ny = c->mesh.ny, n1 = c->k + 1;
  const cuuint64_t rowB = (cuuint64_t)nrhs * 2, edgeB = rowB * n1;
  const cuuint64_t plane = (cuuint64_t)c->ndof * nrhs * 2;
  const size_t nv = (size_t)(nx + 1) * ny;
  const cuuint32_t box[5] = {64, 8, (cuuint32_t)kOzSlots, 1, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  {
    char* base = (char*)XS + edgeB;
    const cuuint64_t dims[5] = {(cuuint64_t)nrhs, (cuuint64_t)n1, (cuuint64_t)(nx - 1), (cuuint64_t)ny,
                                (cuuint64_t)kOzSlices};
    const cuuint64_t str[4] = {rowB, edgeB, edgeB * (cuuint64_t)(nx + 1), plane};
    if (enc(tv, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims, str, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    char* base = (char*)XS + edgeB * (cuuint64_t)(nv + (size_t)nx);
    const cuuint64_t dims[5] = {(cuuint64_t)nrhs, (cuuint64_t)n1, (cuuint64_t)nx, (cuuint64_t)(ny - 1),
                                (cuuint64_t)kOzSlices};
    const cuuint64_t str[4] = {rowB, edgeB, edgeB * (cuuint64_t)nx, plane};
    if (enc(th, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims, str, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

size_t ozaki_smem_bytes() {
  // two slice windows, the block slices, barriers + TMEM slot + flags, alignment
  // slack; at least 120 KB so that one CTA holds an SM (and all 512 TMEM columns)
  const size_t need = (size_t)2 * kOzWinB + (size_t)2 * kOzTypeB + 128 + 1024;
  return need > 120 * 1024 ? need : 120 * 1024;
}

cudaError_t launch_ozaki_apply(Context* c, const double* X, double* Y, int nrhs, cudaStream_t s) {
  if (!c->oz_B || c->k + 1 > 8 || c->mesh.nx < 2 || c->mesh.ny < 2) return cudaErrorInvalidValue;
  const size_t ndof = (size_t)c->ndof;
  // scratch: the slices [8][ndof][nrhs] BF16 and the column exponents
  const size_t xs_bytes = (size_t)kOzSlices * ndof * nrhs * 2;
  if (c->opt.max_device_bytes && c->oz_xs_bytes < xs_bytes &&
      c->bytes + xs_bytes + (size_t)nrhs * sizeof(int) > c->opt.max_device_bytes)
    return cudaErrorMemoryAllocation;                 // the context's memory cap
  if (c->oz_xs_bytes < xs_bytes) {
    if (c->oz_XS) { cudaFree(c->oz_XS); c->oz_XS = nullptr; c->oz_xs_bytes = 0; }
    HDG_CUDA_TRY(cudaMalloc(&c->oz_XS, xs_bytes));
    c->oz_xs_bytes = xs_bytes;
  }
  if (c->oz_ecol_n < nrhs) {
    if (c->oz_ecol) { cudaFree(c->oz_ecol); c->oz_ecol = nullptr; c->oz_ecol_n = 0; }
    HDG_CUDA_TRY(cudaMalloc((void**)&c->oz_ecol, (size_t)nrhs * sizeof(int)));
    c->oz_ecol_n = nrhs;
  }
  HDG_CUDA_TRY(cudaMemsetAsync(c->oz_ecol, 0x80, (size_t)nrhs * sizeof(int), s));   // very negative
  if (nrhs > 2048) return cudaErrorInvalidValue;     // 8 columns per thread, <= 256 threads per row
  {
    const long rows = 256 / (nrhs / 8);
    long bx = (long)((ndof + rows - 1) / rows);
    if (bx > (long)c->num_sms * 4) bx = (long)c->num_sms * 4;
    ozaki_exp_kernel<<<(unsigned)bx, 256, 0, s>>>(X, ndof, nrhs, c->k + 1, c->mesh.nx, c->mesh.ny, c->oz_ecol);
    HDG_CUDA_TRY(cudaGetLastError());
  }
  {
    size_t b = (ndof * (nrhs / 8) + 255) / 256;
    const size_t cap = (size_t)c->num_sms * 16;
    if (b > cap) b = cap;
    ozaki_split_kernel<<<(unsigned)b, 256, 0, s>>>(X, ndof, nrhs, c->k + 1, c->mesh.nx, c->mesh.ny, c->oz_ecol,
                                                   (__nv_bfloat16*)c->oz_XS);
    HDG_CUDA_TRY(cudaGetLastError());
  }
  alignas(64) CUtensorMap tv, th;
  HDG_CUDA_TRY(oz_maps(c, c->oz_XS, nrhs, &tv, &th));
  OzArgs a{};
  a.Y = Y; a.B = (const __nv_bfloat16*)c->oz_B; a.ecol = c->oz_ecol; a.eS = c->oz_eS;
  a.nx = c->mesh.nx; a.ny = c->mesh.ny; a.n1 = c->k + 1; a.nrhs = nrhs;
  a.spr = (c->mesh.nx + kOzBS - 1) / kOzBS; a.nseg = a.spr * c->mesh.ny; a.err = c->err_flag;
  const size_t smem = ozaki_smem_bytes();
  if ((size_t)c->smem_optin < smem) return cudaErrorInvalidValue;
  HDG_CUDA_TRY(cudaFuncSetAttribute(ozaki_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const long items = (long)a.nseg * (nrhs / 64);
  long blocks = c->num_sms;
  if (blocks > items) blocks = items;
  ozaki_apply_kernel<<<(int)blocks, kOzThreads, smem, s>>>(a, tv, th);
  return cudaGetLastError();
}

}  // namespace hdg
