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
};

__device__ __forceinline__ float to_acc(__nv_bfloat16 v, float) { return __bfloat162float(v); }
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

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
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

template <int N1, typename TS, typename TV, typename TA>
__device__ __forceinline__ void apply_segment(const TS* __restrict__ st, int seg, int lane, const ApplyArgs& a) {
  constexpr int M = 4 * N1;
  const int face = lane >> 4;           // 0: W faces, 1: S faces
  const int t = lane & 15;
  const int j = seg / a.spr;
  const int i = (seg % a.spr) * kSeg + t;
  if (i >= a.nx) return;
  const int nx = a.nx, ny = a.ny;
  const int nv = (nx + 1) * ny;
  const TV* __restrict__ v = (const TV*)a.v;
  const TV* __restrict__ cv = (const TV*)a.cvec;
  TV* __restrict__ y = (TV*)a.y;
  const bool bndrow = face == 0 ? (i == 0) : (j == 0);
  const int eout = face == 0 ? i + (nx + 1) * j : nv + i + nx * j;
  const int nrhs = a.nrhs;
  for (int r = 0; r < nrhs; ++r) {
    TA acc[N1];
#pragma unroll
    for (int q = 0; q < N1; ++q) acc[q] = TA(0);
    if (!bndrow) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int ki = (s == 1 && face == 0) ? i - 1 : i;
        const int kj = (s == 1 && face == 1) ? j - 1 : j;
        const TS* __restrict__ rows = st + (size_t)((face * 2 + s) * N1 * M) * kSeg + t;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          int edge;
          bool bnd;
          if (f == 0) { edge = ki + (nx + 1) * kj; bnd = ki == 0; }
          else if (f == 1) { edge = ki + 1 + (nx + 1) * kj; bnd = ki == nx - 1; }
          else if (f == 2) { edge = nv + ki + nx * kj; bnd = kj == 0; }
          else { edge = nv + ki + nx * (kj + 1); bnd = kj == ny - 1; }
          TA xv[N1];
#pragma unroll
          for (int b = 0; b < N1; ++b)
            xv[b] = bnd ? TA(0) : to_acc(__ldg(&v[((size_t)edge * N1 + b) * nrhs + r]), TA(0));
#pragma unroll
          for (int q = 0; q < N1; ++q) {
#pragma unroll
            for (int b = 0; b < N1; ++b) acc[q] = fma(to_acc(rows[(q * M + f * N1 + b) * kSeg], TA(0)), xv[b], acc[q]);
          }
        }
      }
    }
    const TA al = (TA)a.alpha, be = (TA)a.beta;
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      const size_t o = ((size_t)eout * N1 + q) * nrhs + r;
      TA val = TA(0);
      if (!bndrow) {
        val = al * acc[q];
        if (cv) val = fma(be, to_acc(cv[o], TA(0)), val);
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
}

template <int N1, typename TS, typename TV, typename TA>
__global__ void __launch_bounds__(256) apply_kernel(ApplyArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int NS = a.stages;
  const unsigned SB = a.stage_bytes;
  unsigned char* ring = smem_raw + (size_t)w * NS * SB;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)nw * NS * SB) + w * NS;
  const int gw = blockIdx.x * nw + w, tw = gridDim.x * nw;
  const TS* rec = (const TS*)a.rec;
  const size_t seg_elems = (size_t)SB / sizeof(TS);
  if (lane == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int s = 0; s < NS; ++s) {
      const int seg = gw + s * tw;
      if (seg < a.nseg) {
        mbar_expect_tx(&bars[s], SB);
        bulk_load(ring + (size_t)s * SB, rec + (size_t)seg * seg_elems, SB, &bars[s]);
      }
    }
  }
  __syncwarp();
  int it = 0;
  for (;; ++it) {
    const int seg = gw + it * tw;
    if (seg >= a.nseg) break;
    const int stg = it % NS;
    const unsigned par = (unsigned)((it / NS) & 1);
    const bool ok = mbar_wait_bounded(&bars[stg], par);
    if (__any_sync(0xffffffffu, !ok)) {
      if (lane == 0) atomicExch(a.err, 2);
      // let any other copy this warp issued land before the warp exits
      for (int s = 1; s < NS; ++s) {
        const int it2 = it + s;
        if (gw + it2 * tw < a.nseg) (void)mbar_wait_bounded(&bars[it2 % NS], (unsigned)((it2 / NS) & 1));
      }
      return;
    }
    apply_segment<N1, TS, TV, TA>(reinterpret_cast<const TS*>(ring + (size_t)stg * SB), seg, lane, a);
    __syncwarp();
    if (lane == 0) {
      const int nseg2 = seg + NS * tw;
      if (nseg2 < a.nseg) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bars[stg], SB);
        bulk_load(ring + (size_t)stg * SB, rec + (size_t)nseg2 * seg_elems, SB, &bars[stg]);
      }
    }
    __syncwarp();
  }
}

// Host-side launcher for one (degree, storage, vector) combination.
template <int N1, typename TS, typename TV, typename TA>
cudaError_t apply_launch(const Context* c, const ApplyArgs& args0, cudaStream_t s) {
  ApplyArgs a = args0;
  constexpr int R = 4 * N1 * 4 * N1;
  a.stage_bytes = (unsigned)(R * kSeg * sizeof(TS));
  // ring budget ~220 KB per CTA: 3 stages per warp when that still leaves two
  // or more warps, else 2, else 1; at most 8 warps
  const size_t budget = 220 * 1024;
  int NS = 3;
  int nw = (int)(budget / ((size_t)NS * a.stage_bytes));
  if (nw < 2) { NS = 2; nw = (int)(budget / ((size_t)NS * a.stage_bytes)); }
  if (nw < 1) { NS = 1; nw = 1; }
  if (nw > 8) nw = 8;
  a.stages = NS;
  const size_t smem = (size_t)nw * NS * a.stage_bytes + (size_t)nw * NS * sizeof(uint64_t);
  auto kern = apply_kernel<N1, TS, TV, TA>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int blocks = c->num_sms;
  const int need = (a.nseg + nw - 1) / nw;
  if (need < blocks) blocks = need > 0 ? need : 1;
  kern<<<blocks, 32 * nw, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename TS, typename TV, typename TA>
cudaError_t apply_dispatch(const Context* c, int n1, const ApplyArgs& a, cudaStream_t s) {
  switch (n1) {
    case 1: return apply_launch<1, TS, TV, TA>(c, a, s);
    case 2: return apply_launch<2, TS, TV, TA>(c, a, s);
    case 3: return apply_launch<3, TS, TV, TA>(c, a, s);
    case 4: return apply_launch<4, TS, TV, TA>(c, a, s);
    case 5: return apply_launch<5, TS, TV, TA>(c, a, s);
    case 6: return apply_launch<6, TS, TV, TA>(c, a, s);
    case 7: return apply_launch<7, TS, TV, TA>(c, a, s);
    case 8: return apply_launch<8, TS, TV, TA>(c, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t apply_fp64(const Context* c, int n1, const ApplyArgs& a, cudaStream_t s);
cudaError_t apply_fp32(const Context* c, int n1, const ApplyArgs& a, cudaStream_t s);
cudaError_t apply_bf16(const Context* c, int n1, const ApplyArgs& a, cudaStream_t s);

}  // namespace hdg
