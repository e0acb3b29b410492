// Assembly-free apply of an element-block operator on the owner-record layout
// (Alg. 3 of the paper, re-organised for sm_103a):
//
//   y[e] = beta * c[e] + alpha * sum_{K in {K1, K2}} B_K[e rows, :] v_K
//
// for every interior edge e, where v_K gathers the element's 4 faces and B_K is
// the condensed block S_K (trace apply) or a weighted Schwarz block (smoother).
// Boundary edges get y = 0 and boundary entries of v are read as 0.
//
// Work split: the mesh row j is cut into segments of 16 elements; one warp owns
// one segment at a time. Lanes 0-15 compute the W faces of the 16 elements and
// lanes 16-31 their S faces, so every face is written by exactly one thread and
// no atomics or grid barriers are needed. The row blocks a segment needs are
// contiguous in memory (the record layout), so each warp streams them into its
// own shared-memory ring with one 1-D bulk copy (cp.async.bulk, completion on an
// mbarrier) per segment, NS stages deep, while it computes on the previous one.
// Within a stage the blocks are element-fastest, so the 16 lanes of a face read
// 16 consecutive words: no bank conflicts.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

#include "hdg_internal.h"

namespace hdg {

// Launch shape of the apply: warp pairs per CTA (one CTA per SM, at most 8
// pairs) and ring stages per pair. `tune` packs a choice made by the set-up
// autotuner (pairs * 16 + stages); 0 = the default: as many pairs as fit up to
// 4 (two warps per SM sub-partition), then more stages.
// stage_bytes: one stage of blocks plus its x windows and partial sums.
inline void apply_shape(unsigned stage_bytes, int tune, int* np, int* ns) {
  const int total = (int)((220u * 1024u) / stage_bytes);   // stages that fit
  if (tune > 0) {
    *np = tune >> 4; *ns = tune & 15;
    if (*np >= 1 && *np <= 8 && *ns >= 1 && *np * *ns <= total) return;
  }
  if (total <= 0) { *np = 1; *ns = 1; return; }
  int p = total < 4 ? total : 4;
  int st = total / p;
  if (st > 3) st = 3;
  *np = p; *ns = st < 1 ? 1 : st;
}

struct ApplyArgs {
  const void* rec;     // record array of the level (type TS)
  const void* v;       // gathered vector (type TV)
  const void* cvec;    // addend (type TV) or nullptr
  void* y;             // output (type TV)
  double alpha, beta;
  int nx, ny, spr, nseg, nrhs;
  int stages;          // NS
  unsigned stage_bytes;
  int* err;            // device error flag (2 = bounded wait gave up)
  int tune;            // launch shape from the autotuner (0 = default)
};

// Double-float value hi + lo (|lo| <= ulp(hi)/2 after renormalisation).
struct dfloat {
  float hi, lo;
};

__device__ __forceinline__ float to_acc(__nv_bfloat16 v, float) { return __bfloat162float(v); }
__device__ __forceinline__ dfloat to_acc(float2 v, dfloat) { return dfloat{v.x, v.y}; }
// double -> (hi, lo) with integer operations and one FP32 subtraction (the FP64
// pipe, which also runs int <-> float and float <-> double conversions, is slow on
// this GPU): hi keeps the leading 24 significant bits (truncated); lo is the
// remaining 29 bits rounded to 24: the rounded bits are placed under the exponent
// 2^E of lo's scale, and subtracting 2^E (exact, both operands in [2^E, 2^(E+1)])
// leaves them as a float. hi + lo = v to about 2^-47 relative for 2^-103 <= |v| <
// 2^128. Outside that range, still with integer operations only: below 2^-103 hi
// keeps 24 bits and lo is 0, below 2^-126 the value becomes +-0, beyond 2^128 +-inf,
// and inf / nan keep their class.
__device__ __forceinline__ dfloat split_double(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long mant = b & 0xfffffffffffffull;
  if (e >= 920 && e <= 1150) {
    const unsigned int hib = sign | ((unsigned int)(e - 1023 + 127) << 23) | (unsigned int)(mant >> 29);
    const unsigned int rem = (unsigned int)(mant & 0x1fffffffull);        // 29 bits below hi
    // lo = rem * 2^(e - 1075) = (2^E + rounded rem) - 2^E with E = e - 1046
    const unsigned int eb = (unsigned int)(e - 919) << 23;                // float bits of 2^E
    const float top = __uint_as_float(eb + ((rem + 32u) >> 6));           // mantissa carry rounds up to 2^(E+1)
    float lo = top - __uint_as_float(eb);
    lo = __uint_as_float(__float_as_uint(lo) | sign);
    return dfloat{__uint_as_float(hib), lo};
  }
  unsigned int hib = sign;                                                // |v| < 2^-126 and zero
  if (e >= 897 && e < 920) hib = sign | ((unsigned int)(e - 896) << 23) | (unsigned int)(mant >> 29);
  else if (e > 1150) hib = sign | 0x7f800000u | ((e == 2047 && mant) ? 0x400000u : 0u);
  return dfloat{__uint_as_float(hib), 0.0f};
}
__device__ __forceinline__ dfloat to_acc(double v, dfloat) { return split_double(v); }
// acc + s*x with an error-free product (FMA residual) and an error-free sum
// (Knuth's two-sum) of the leading parts; the trailing parts are summed in
// plain FP32, which keeps ~48 significant bits for these short dot products.
__device__ __forceinline__ float mac(float s, float x, float acc) { return fmaf(s, x, acc); }
__device__ __forceinline__ double mac(double s, double x, double acc) { return ::fma(s, x, acc); }
__device__ __forceinline__ dfloat mac(dfloat s, dfloat x, dfloat acc) {
  const float p = s.hi * x.hi;
  float e = fmaf(s.hi, x.hi, -p);
  e = fmaf(s.hi, x.lo, e);
  e = fmaf(s.lo, x.hi, e);
  const float sum = acc.hi + p;
  const float bb = sum - acc.hi;
  const float err = (acc.hi - (sum - bb)) + (p - bb);
  return dfloat{sum, acc.lo + (err + e)};
}
// float -> double from the bits, exactly, with integer operations only (the
// conversion instruction runs on the FP64 pipe, which is slow on this GPU):
// normal floats re-biased, subnormals normalised by a leading-zero count, zero,
// inf and nan keeping their class
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned int ex = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned long long b;
  if (ex != 0u && ex != 255u) {
    b = sign | ((unsigned long long)(ex + 896u) << 52) | ((unsigned long long)m << 29);
  } else if (ex == 255u) {
    b = sign | (0x7ffull << 52) | ((unsigned long long)m << 29);
  } else if (m == 0u) {
    b = sign;
  } else {
    const int p = 31 - __clz((int)m);                       // leading one of the subnormal mantissa
    b = sign | ((unsigned long long)(p - 149 + 1023) << 52) |
        (((unsigned long long)m << (52 - p)) & 0xfffffffffffffull);
  }
  return __longlong_as_double((long long)b);
}
// value of an accumulator in the output arithmetic (one FP64 add for hi + lo)
__device__ __forceinline__ double finish(dfloat a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }
__device__ __forceinline__ double finish(double a) { return a; }
__device__ __forceinline__ float finish(float a) { return a; }
template <typename TA> struct OutT { using type = TA; };
template <> struct OutT<dfloat> { using type = double; };
__device__ __forceinline__ float to_acc(float v, float) { return v; }
__device__ __forceinline__ double to_acc(double v, double) { return v; }
__device__ __forceinline__ double to_acc(float v, double) { return (double)v; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// One probe of an mbarrier phase; the suspend-time hint (~0.1 ms) lets the
// hardware park the polling thread until the phase completes, so that it does
// not take issue slots from the other CTAs' arithmetic on the SM.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0;
}

// x window of a segment (row j, elements i0..i0+15): 5 edge rows x 18 slots,
// slot = i - (i0 - 1); each row is one contiguous range of the trace vector:
//   row 0: vertical edges of row j      row 1: vertical edges of row j-1
//   row 2: horizontal edges of row j    row 3: horizontal edges of row j+1
//   row 4: horizontal edges of row j-1
constexpr int kWinRows = 5, kWinSlots = kSeg + 2;

template <int N1, typename TV>
__device__ __forceinline__ void issue_window(TV* __restrict__ dst, const TV* __restrict__ v, int seg, int lane,
                                             const ApplyArgs& a) {
  const int j = seg / a.spr, i0 = (seg % a.spr) * kSeg;
  const int nx = a.nx, nv = (nx + 1) * a.ny;
  const int s0 = i0 == 0 ? 1 : 0;                                   // slot 0 is i = -1
  const int sv1 = min(kWinSlots, nx - i0 + 2), sh1 = min(kWinSlots, nx - i0 + 1);
#pragma unroll
  for (int r = 0; r < kWinRows; ++r) {
    if ((r == 1 || r == 4) && j == 0) continue;
    const bool vert = r < 2;
    const int jr = (r == 0 || r == 2) ? j : (r == 3 ? j + 1 : j - 1);
    const long e0 = vert ? (long)(i0 - 1) + (long)(nx + 1) * jr : (long)nv + (i0 - 1) + (long)nx * jr;
    const int hi = (vert ? sv1 : sh1) * N1;
    TV* d = dst + r * kWinSlots * N1;
    for (int idx = s0 * N1 + lane; idx < hi; idx += 32) {
      const TV* src = v + e0 * N1 + idx;
      if (sizeof(TV) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(d + idx)), "l"(src) : "memory");
      else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(d + idx)), "l"(src) : "memory");
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void window_wait(int pending) {
  // groups complete in order; `pending` = groups allowed to stay in flight
  if (pending <= 0) asm volatile("cp.async.wait_group 0;" ::: "memory");
  else if (pending == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
  else asm volatile("cp.async.wait_group 2;" ::: "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait: gives up after ~1 s of device time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (unsigned it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 63u && global_ns() - t0 > 1000000000ull) return false;
  }
}

// The segment kernels' wait for their block copy (thread 0; `bar` is followed
// by 8 spare bytes of shared memory). While the context's probe count
// (err[1], hdg_options.wait_probe) is positive, block 0 of a launch first waits
// on a second barrier that nothing ever completes: the bounded wait gives up
// and the caller takes the timeout path (flag, drain its own copy, exit).
__device__ __forceinline__ bool seg_first_wait(const ApplyArgs& a, uint64_t* bar) {
  if (blockIdx.x == 0) {
    volatile int* probe = a.err + 1;
    const int left = *probe;
    if (left > 0) {
      *probe = left - 1;
      uint64_t* never = bar + 1;
      mbar_init(never, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      if (!mbar_wait_bounded(never, 0)) return false;
    }
  }
  return mbar_wait_bounded(bar, 0);
}

__device__ __forceinline__ void pair_barrier(int id) {
  asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory");
}

// One thread: lane -> (face, element) of the segment, `slot` = 0 for the
// element's own row block, 1 for the neighbour across that face. Returns the
// partial sums of the N1 outputs of the face. x values come from the window
// (nrhs = 1) or straight from global memory (nrhs > 1).
template <int N1, typename TS, typename TV, typename TA, bool DIFF>
__device__ __forceinline__ void partial_segment(const TS* __restrict__ st, const TV* __restrict__ xw, int seg, int lane,
                                                int slot, int r, const ApplyArgs& a, TA (&acc)[N1]) {
  constexpr int M = 4 * N1;
  const int face = lane >> 4, t = lane & 15;
  const int j = seg / a.spr, i = (seg % a.spr) * kSeg + t;
  const int nx = a.nx, ny = a.ny, nv = (nx + 1) * ny;
#pragma unroll
  for (int q = 0; q < N1; ++q) acc[q] = TA{};
  const bool bndrow = face == 0 ? (i == 0) : (j == 0);
  if (i >= nx || bndrow) return;
  const int ki = (slot == 1 && face == 0) ? i - 1 : i;
  const int kj = (slot == 1 && face == 1) ? j - 1 : j;
  int edge[4], wpos[4];
  bool bnd[4];
  edge[0] = ki + (nx + 1) * kj;       bnd[0] = ki <= 0;
  edge[1] = ki + 1 + (nx + 1) * kj;   bnd[1] = ki >= nx - 1;
  edge[2] = nv + ki + nx * kj;        bnd[2] = kj <= 0;
  edge[3] = nv + ki + nx * (kj + 1);  bnd[3] = kj >= ny - 1;
  {
    const int sl = ki - (i - t) + 1;
    const int vrow = (kj == j) ? 0 : 1;
    const int hlo = (kj == j) ? 2 : 4, hhi = (kj == j) ? 3 : 2;
    wpos[0] = (vrow * kWinSlots + sl) * N1;
    wpos[1] = (vrow * kWinSlots + sl + 1) * N1;
    wpos[2] = (hlo * kWinSlots + sl) * N1;
    wpos[3] = (hhi * kWinSlots + sl) * N1;
  }
  const TV* __restrict__ v = (const TV*)a.v;
  const int nrhs = a.nrhs;
  TA xv[M];
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int b = 0; b < N1; ++b)
      xv[f * N1 + b] = bnd[f] ? TA{}
                              : to_acc(xw ? xw[wpos[f] + b] : __ldg(&v[((size_t)edge[f] * N1 + b) * nrhs + r]), TA{});
  if constexpr (DIFF) {
    TA mean = TA(0);
#pragma unroll
    for (int c = 0; c < M; ++c) mean += xv[c];
    mean *= TA(1.0 / M);
#pragma unroll
    for (int c = 0; c < M; ++c) xv[c] -= mean;
  }
  const TS* __restrict__ rows = st + (size_t)((face * 2 + slot) * N1 * M) * kSeg + t;
#pragma unroll
  for (int c = 0; c < M; ++c)
#pragma unroll
    for (int q = 0; q < N1; ++q) acc[q] = mac(to_acc(rows[(q * M + c) * kSeg], TA{}), xv[c], acc[q]);
}

// Epilogue of one face (slot-0 warp): y = beta c + alpha (own + neighbour).
template <int N1, typename TV, typename TO>
__device__ __forceinline__ void write_face(const TO (&sum)[N1], int seg, int lane, int r, const ApplyArgs& a) {
  const int face = lane >> 4, t = lane & 15;
  const int j = seg / a.spr, i = (seg % a.spr) * kSeg + t;
  const int nx = a.nx, ny = a.ny, nv = (nx + 1) * ny;
  if (i >= nx) return;
  const TV* __restrict__ cv = (const TV*)a.cvec;
  TV* __restrict__ y = (TV*)a.y;
  const int nrhs = a.nrhs;
  const bool bndrow = face == 0 ? (i == 0) : (j == 0);
  const int eout = face == 0 ? i + (nx + 1) * j : nv + i + nx * j;
  const TO al = (TO)a.alpha, be = (TO)a.beta;
  // y = A v, y = c - A v and y = c + A v take no multiply (FP64 ops are slow here)
  const int form = (al == TO(1) && (!cv || be == TO(0))) ? 0
                   : (cv && be == TO(1) && al == TO(-1)) ? 1 : (cv && be == TO(1) && al == TO(1)) ? 2 : 3;
#pragma unroll
  for (int q = 0; q < N1; ++q) {
    const size_t o = ((size_t)eout * N1 + q) * nrhs + r;
    TO val = TO(0);
    if (!bndrow) {
      if (form == 0) val = sum[q];
      else if (form == 1) val = (TO)cv[o] - sum[q];
      else if (form == 2) val = (TO)cv[o] + sum[q];
      else {
        val = al * sum[q];
        if (cv) val = mac(be, (TO)cv[o], val);
      }
    }
    y[o] = (TV)val;
  }
  // the E / N domain-boundary edges have no owner element: zero them here
  if (face == 0 && i == nx - 1) {
    const int eb = nx + (nx + 1) * j;
#pragma unroll
    for (int q = 0; q < N1; ++q) y[((size_t)eb * N1 + q) * nrhs + r] = TV(0);
  }
  if (face == 1 && j == ny - 1) {
    const int eb = nv + i + nx * ny;
#pragma unroll
    for (int q = 0; q < N1; ++q) y[((size_t)eb * N1 + q) * nrhs + r] = TV(0);
  }
}

// Shared-memory bytes of one ring stage: blocks + two x windows + partials.
template <int N1, typename TS, typename TV, typename TO>
constexpr size_t stage_total_bytes() {
  return (size_t)16 * N1 * N1 * kSeg * sizeof(TS) +
         2 * (((size_t)kWinRows * kWinSlots * N1 * sizeof(TV) + 15) / 16 * 16) +
         (((size_t)32 * N1 * sizeof(TO) + 15) / 16 * 16) + 16;
}

// Work split: warp pairs. Both warps of a pair stream the same segments through
// the pair's ring; warp 0 of the pair applies each element's own row blocks,
// warp 1 the neighbours' row blocks and hands its partial sums to warp 0
// through shared memory (named barrier per pair), which writes the faces.
// 8-byte blocks (FP64, F32X2) never fit more than 4 warp pairs per CTA, so they
// get up to 255 registers; 2- and 4-byte blocks may use 8 pairs.
template <typename TS>
struct ApplyMaxThreads { static constexpr int value = sizeof(TS) >= 8 ? 256 : 512; };

template <int N1, typename TS, typename TV, typename TA, bool DIFF>
__global__ void __launch_bounds__(ApplyMaxThreads<TS>::value) apply_kernel(ApplyArgs a) {
  using TO = typename OutT<TA>::type;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int np = blockDim.x >> 6;                 // pairs per CTA
  const int pr = w >> 1, role = w & 1;            // role 0: own blocks, 1: neighbour blocks
  const int NS = a.stages;
  const unsigned SB = a.stage_bytes;
  constexpr size_t XWB = ((size_t)kWinRows * kWinSlots * N1 * sizeof(TV) + 15) / 16 * 16;
  constexpr size_t PB = ((size_t)32 * N1 * sizeof(TO) + 15) / 16 * 16;
  const size_t pair_bytes = (size_t)NS * (SB + 2 * XWB + PB + 16);
  unsigned char* base = smem_raw + (size_t)pr * pair_bytes;
  unsigned char* ring = base;                                    // [NS][SB]
  unsigned char* wins = base + (size_t)NS * SB;                  // [2][NS][XWB]
  unsigned char* parts = wins + (size_t)2 * NS * XWB;            // [NS][PB]
  uint64_t* bars = reinterpret_cast<uint64_t*>(parts + (size_t)NS * PB);   // [NS]
  TV* mywin = reinterpret_cast<TV*>(wins + (size_t)role * NS * XWB);
  const int gp = blockIdx.x * np + pr, tp = gridDim.x * np;
  const TS* rec = (const TS*)a.rec;
  const TV* vin = (const TV*)a.v;
  const size_t seg_elems = (size_t)SB / sizeof(TS);
  const bool use_win = (a.nrhs == 1);
  const int bar_id = 1 + pr;
  if (role == 0 && lane == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int s = 0; s < NS; ++s) {
      const int seg = gp + s * tp;
      if (seg < a.nseg) {
        mbar_expect_tx(&bars[s], SB);
        bulk_load(ring + (size_t)s * SB, rec + (size_t)seg * seg_elems, SB, &bars[s]);
      }
    }
  }
  pair_barrier(bar_id);            // barriers initialised before the partner waits
  if (use_win) {
    for (int s = 0; s < NS; ++s) {
      const int seg = gp + s * tp;
      if (seg < a.nseg) issue_window<N1, TV>(mywin + (size_t)s * (XWB / sizeof(TV)), vin, seg, lane, a);
      else asm volatile("cp.async.commit_group;" ::: "memory");
    }
  }
  for (int it = 0;; ++it) {
    const int seg = gp + it * tp;
    if (seg >= a.nseg) break;
    const int stg = it % NS;
    const unsigned par = (unsigned)((it / NS) & 1);
    if (use_win) window_wait(NS - 1);
    const bool ok = mbar_wait_bounded(&bars[stg], par);
    if (__any_sync(0xffffffffu, !ok)) {
      if (lane == 0) atomicExch(a.err, 2);
      asm volatile("cp.async.wait_all;" ::: "memory");
      for (int s = 1; s < NS; ++s) {
        const int it2 = it + s;
        if (gp + it2 * tp < a.nseg) (void)mbar_wait_bounded(&bars[it2 % NS], (unsigned)((it2 / NS) & 1));
      }
      return;      // the partner warp times out on the same barrier and returns too
    }
    __syncwarp();
    const TS* st = reinterpret_cast<const TS*>(ring + (size_t)stg * SB);
    const TV* xw = use_win ? mywin + (size_t)stg * (XWB / sizeof(TV)) : nullptr;
    TO* part = reinterpret_cast<TO*>(parts + (size_t)stg * PB);
    for (int r = 0; r < a.nrhs; ++r) {
      TA acc[N1];
      partial_segment<N1, TS, TV, TA, DIFF>(st, xw, seg, lane, role, r, a, acc);
      if (role == 1) {
#pragma unroll
        for (int q = 0; q < N1; ++q) part[q * 32 + lane] = finish(acc[q]);
      }
      pair_barrier(bar_id);
      if (role == 0) {
        TO sum[N1];
#pragma unroll
        for (int q = 0; q < N1; ++q) sum[q] = finish(acc[q]) + part[q * 32 + lane];
        write_face<N1, TV, TO>(sum, seg, lane, r, a);
      }
      if (a.nrhs > 1) pair_barrier(bar_id);   // partials consumed before the next right-hand side
    }
    const int nseg2 = seg + NS * tp;
    if (role == 0) {
      __syncwarp();
      if (lane == 0 && nseg2 < a.nseg) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bars[stg], SB);
        bulk_load(ring + (size_t)stg * SB, rec + (size_t)nseg2 * seg_elems, SB, &bars[stg]);
      }
    }
    if (use_win) {
      __syncwarp();
      if (nseg2 < a.nseg) issue_window<N1, TV>(mywin + (size_t)stg * (XWB / sizeof(TV)), vin, nseg2, lane, a);
      else asm volatile("cp.async.commit_group;" ::: "memory");
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// ---------------------------------------------------------------------------
// One CTA per record segment (nrhs = 1). One bulk copy stages the segment's
// row blocks; the NW warps split the products by (side, group of input faces):
// warp (side, g) gives every lane (element t, owned face W or S) the products of
// its block rows with faces g*8/NW .. of the element on that side (own or
// neighbour). The NW partial sums of each output are added in a fixed order
// through shared memory. Several CTAs share an SM, so one CTA's copy overlaps
// the others' arithmetic: the FP64 pipe stays fed without a deep ring. NW = 8
// spreads the products widest; NW = 4 halves the partial sums (which also run
// on the FP64 pipe in FP64); NW = 2 (one warp per side) leaves one add per output.
constexpr int kTuneSeg = 0x400;      // tune flag: this kernel, 8 warps
constexpr int kTuneSeg4 = 0x800;     // with kTuneSeg: 4 warps
constexpr int kTuneSeg2 = 0x1000;    // with kTuneSeg: 2 warps (one per side, all four faces)

template <int N1, typename TS, typename TO, int NW>
constexpr size_t seg_smem_bytes() {
  return (size_t)16 * N1 * N1 * kSeg * sizeof(TS) + (size_t)NW * N1 * 32 * sizeof(TO) + 16;
}

// The segment's products, partial sums and outputs once its blocks are being
// copied into `st` (completion on `bar`); `part` holds NW x N1 x 32 outputs.
// Shared by the single-mesh kernel and the multi-mesh launch.
template <int N1, typename TS, typename TV, typename TA, bool DIFF, int NW>
__device__ __forceinline__ void seg_body(const ApplyArgs& a, int seg, const TS* st,
                                         typename OutT<TA>::type* part, uint64_t* bar) {
  using TO = typename OutT<TA>::type;
  constexpr int M = 4 * N1;
  constexpr int GPS = NW / 2;                  // face groups per side
  constexpr int FPW = 4 / GPS;                 // faces per warp
  constexpr int NC = FPW * N1;                 // block columns per warp
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nx = a.nx, ny = a.ny, nv = (nx + 1) * ny;
  const int j = seg / a.spr, i0 = (seg % a.spr) * kSeg;
  const int oface = lane >> 4, t = lane & 15, i = i0 + t;
  const int side = warp / GPS, g0 = (warp % GPS) * FPW;
  const bool active = i < nx && !(oface == 0 ? (i == 0) : (j == 0));
  // x of faces g0 .. g0+FPW-1 of the element on this side (loaded while the
  // blocks arrive)
  TA xf[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) xf[c] = TA{};
  if (active) {
    const TV* __restrict__ v = (const TV*)a.v;
    const int ki = (side == 1 && oface == 0) ? i - 1 : i;
    const int kj = (side == 1 && oface == 1) ? j - 1 : j;
    int edge[4];
    bool bnd[4];
    edge[0] = ki + (nx + 1) * kj;       bnd[0] = ki <= 0;
    edge[1] = ki + 1 + (nx + 1) * kj;   bnd[1] = ki >= nx - 1;
    edge[2] = nv + ki + nx * kj;        bnd[2] = kj <= 0;
    edge[3] = nv + ki + nx * (kj + 1);  bnd[3] = kj >= ny - 1;
    if constexpr (DIFF) {
      // blocks with zero row sums act on x - mean(x) (boundary entries count as 0)
      TA xa[M];
#pragma unroll
      for (int g = 0; g < 4; ++g)
#pragma unroll
        for (int b = 0; b < N1; ++b) xa[g * N1 + b] = bnd[g] ? TA{} : to_acc(__ldg(&v[(size_t)edge[g] * N1 + b]), TA{});
      TA mean = TA(0);
#pragma unroll
      for (int c = 0; c < M; ++c) mean += xa[c];
      mean *= TA(1.0 / M);
#pragma unroll
      for (int lf = 0; lf < FPW; ++lf)
#pragma unroll
        for (int b = 0; b < N1; ++b) {
          TA xv = xa[b];
#pragma unroll
          for (int g = 1; g < 4; ++g) xv = (g0 + lf == g) ? xa[g * N1 + b] : xv;
          xf[lf * N1 + b] = xv - mean;
        }
    } else {
#pragma unroll
      for (int lf = 0; lf < FPW; ++lf) {
        const int gg = g0 + lf;
        const int ef = gg == 0 ? edge[0] : (gg == 1 ? edge[1] : (gg == 2 ? edge[2] : edge[3]));
        const bool bf = gg == 0 ? bnd[0] : (gg == 1 ? bnd[1] : (gg == 2 ? bnd[2] : bnd[3]));
        if (!bf) {
#pragma unroll
          for (int b = 0; b < N1; ++b) xf[lf * N1 + b] = to_acc(__ldg(&v[(size_t)ef * N1 + b]), TA{});
        }
      }
    }
  }
  // one thread polls the copy's mbarrier (bounded) while the others sleep in the
  // block barrier, leaving the issue slots to the SM's other CTAs
  if (__syncthreads_or(threadIdx.x == 0 ? !seg_first_wait(a, bar) : 0)) {
    // the copy did not land within the bound: flag it, give it one more bounded
    // wait (it writes this CTA's shared memory), and leave together
    if (threadIdx.x == 0) {
      atomicExch(a.err, 2);
      (void)mbar_wait_bounded(bar, 0);
    }
    __syncthreads();
    return;
  }
  TA acc[N1];
#pragma unroll
  for (int q = 0; q < N1; ++q) acc[q] = TA{};
  if (active) {
    const TS* rows = st + (size_t)((oface * 2 + side) * N1 * M + g0 * N1) * kSeg + t;
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int q = 0; q < N1; ++q) acc[q] = mac(to_acc(rows[(q * M + c) * kSeg], TA{}), xf[c], acc[q]);
  }
#pragma unroll
  for (int q = 0; q < N1; ++q) part[(warp * N1 + q) * 32 + lane] = finish(acc[q]);
  __syncthreads();
  // epilogue: output o = (owned face, element, row), row fastest (contiguous y)
  const TV* __restrict__ cv = (const TV*)a.cvec;
  TV* __restrict__ y = (TV*)a.y;
  const TO al = (TO)a.alpha, be = (TO)a.beta;
  // y = A v, y = c - A v (the V-cycle's residuals) and y = c + A v take no multiply
  const int form = (al == TO(1) && (!cv || be == TO(0))) ? 0
                   : (cv && be == TO(1) && al == TO(-1)) ? 1 : (cv && be == TO(1) && al == TO(1)) ? 2 : 3;
  for (int o = threadIdx.x; o < 32 * N1; o += 32 * NW) {
    const int q = o % N1, ln = o / N1;
    const int of = ln >> 4, ii = i0 + (ln & 15);
    if (ii >= nx) continue;
    const bool br = of == 0 ? (ii == 0) : (j == 0);
    const size_t eout = of == 0 ? (size_t)ii + (size_t)(nx + 1) * j : (size_t)nv + ii + (size_t)nx * j;
    TO sum = part[q * 32 + ln];
#pragma unroll
    for (int w = 1; w < NW; ++w) sum += part[(w * N1 + q) * 32 + ln];
    TO val = TO(0);
    if (!br) {
      if (form == 0) val = sum;
      else if (form == 1) val = (TO)cv[eout * N1 + q] - sum;
      else if (form == 2) val = (TO)cv[eout * N1 + q] + sum;
      else {
        val = al * sum;
        if (cv) val = mac(be, (TO)cv[eout * N1 + q], val);
      }
    }
    y[eout * N1 + q] = (TV)val;
    // the E / N domain-boundary edges have no owner element: zero them here
    if (of == 0 && ii == nx - 1) y[((size_t)nx + (size_t)(nx + 1) * j) * N1 + q] = TV(0);
    if (of == 1 && j == ny - 1) y[((size_t)nv + ii + (size_t)nx * ny) * N1 + q] = TV(0);
  }
}

template <int N1, typename TS, typename TV, typename TA, bool DIFF, int NW>
__global__ void __launch_bounds__(32 * NW) apply_seg_kernel(ApplyArgs a) {
  using TO = typename OutT<TA>::type;
  constexpr int R = 16 * N1 * N1;
  constexpr unsigned SB = (unsigned)(R * kSeg * sizeof(TS));
  extern __shared__ __align__(128) unsigned char seg_smem[];
  TS* st = reinterpret_cast<TS*>(seg_smem);
  TO* part = reinterpret_cast<TO*>(seg_smem + SB);                          // [NW][N1][32]
  uint64_t* bar = reinterpret_cast<uint64_t*>(seg_smem + SB + (size_t)NW * N1 * 32 * sizeof(TO));
  const int seg = blockIdx.x;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, SB);
    bulk_load(st, (const TS*)a.rec + (size_t)seg * (SB / sizeof(TS)), SB, bar);
  }
  seg_body<N1, TS, TV, TA, DIFF, NW>(a, seg, st, part, bar);
}

template <int N1, typename TS, typename TV, typename TA, bool DIFF, int NW>
cudaError_t seg_launch(const Context* c, const ApplyArgs& a, cudaStream_t s) {
  using TO = typename OutT<TA>::type;
  const size_t smem = seg_smem_bytes<N1, TS, TO, NW>();
  if ((size_t)c->smem_optin < smem) return cudaErrorInvalidValue;
  auto kern = apply_seg_kernel<N1, TS, TV, TA, DIFF, NW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, c->smem_optin);
  if (e != cudaSuccess) return e;
  if (a.nseg <= 0) return cudaSuccess;
  kern<<<a.nseg, 32 * NW, smem, s>>>(a);
  return cudaGetLastError();
}

// Host-side launcher for one (degree, storage, vector) combination.
template <int N1, typename TS, typename TV, typename TA, bool DIFF>
cudaError_t apply_launch(const Context* c, const ApplyArgs& args0, cudaStream_t s) {
  using TO = typename OutT<TA>::type;
  ApplyArgs a = args0;
  if (a.tune & kTuneSeg) {
    if (a.tune & kTuneSeg4) return seg_launch<N1, TS, TV, TA, DIFF, 4>(c, a, s);
    if (a.tune & kTuneSeg2) return seg_launch<N1, TS, TV, TA, DIFF, 2>(c, a, s);
    return seg_launch<N1, TS, TV, TA, DIFF, 8>(c, a, s);
  }
  a.stage_bytes = (unsigned)(16 * N1 * N1 * kSeg * sizeof(TS));
  int np = 0, NS = 0;
  apply_shape((unsigned)stage_total_bytes<N1, TS, TV, TO>(), a.tune, &np, &NS);
  if (64 * np > ApplyMaxThreads<TS>::value) np = ApplyMaxThreads<TS>::value / 64;
  a.stages = NS;
  const size_t smem = (size_t)np * NS * stage_total_bytes<N1, TS, TV, TO>();
  auto kern = apply_kernel<N1, TS, TV, TA, DIFF>;
  // one kernel serves launches with different ring sizes (S and Schwarz blocks,
  // tuned shapes), some of them replayed later from a captured graph: allow the
  // device's whole opt-in shared memory once instead of the size of this launch
  if ((size_t)c->smem_optin < smem) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, c->smem_optin);
  if (e != cudaSuccess) return e;
  int blocks = c->num_sms;
  const int need = (a.nseg + np - 1) / np;
  if (need < blocks) blocks = need > 0 ? need : 1;
  kern<<<blocks, 64 * np, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename TS, typename TV, typename TA, bool DIFF>
cudaError_t apply_dispatch(const Context* c, int n1, const ApplyArgs& a, cudaStream_t s) {
  switch (n1) {
    case 1: return apply_launch<1, TS, TV, TA, DIFF>(c, a, s);
    case 2: return apply_launch<2, TS, TV, TA, DIFF>(c, a, s);
    case 3: return apply_launch<3, TS, TV, TA, DIFF>(c, a, s);
    case 4: return apply_launch<4, TS, TV, TA, DIFF>(c, a, s);
    case 5: return apply_launch<5, TS, TV, TA, DIFF>(c, a, s);
    case 6: return apply_launch<6, TS, TV, TA, DIFF>(c, a, s);
    case 7: return apply_launch<7, TS, TV, TA, DIFF>(c, a, s);
    case 8: return apply_launch<8, TS, TV, TA, DIFF>(c, a, s);
    default: return cudaErrorInvalidValue;
  }
}

// diff = true applies the blocks to x - mean(x) per element (for blocks with
// zero row sums, i.e. the condensed operator S); false for the Schwarz blocks
cudaError_t apply_fp64(const Context* c, int n1, bool diff, const ApplyArgs& a, cudaStream_t s);
cudaError_t apply_fp32(const Context* c, int n1, bool diff, const ApplyArgs& a, cudaStream_t s);
cudaError_t apply_bf16(const Context* c, int n1, bool diff, const ApplyArgs& a, cudaStream_t s);
cudaError_t apply_x2(const Context* c, int n1, bool diff, const ApplyArgs& a, cudaStream_t s);

}  // namespace hdg
