// Column-batched apply of an element-block operator on the owner-record layout
// (Alg. 3 of the paper with many right-hand sides): the same operation as the
// single-vector apply,
//
//   Y[e][:] = beta * C[e][:] + alpha * sum_{K in {K1, K2}} B_K[e rows, :] X_K[:, :]
//
// for vectors stored right-hand-side fastest, X[dof][nb]. One CTA takes one
// record segment (16 elements of a mesh row). It stages the segment's row blocks
// once in shared memory, element-major so that a thread reads four consecutive
// columns of a block row with one vector load, and then reuses them for every
// right-hand side: the lanes of a warp run over 32 consecutive right-hand sides,
// so every load of X and store of Y is one contiguous 32-column row. A warp
// item is (element, owned face W or S, chunk of 32 columns); each face is
// written by exactly one lane per column, no atomics.
#pragma once
#include "apply_impl.cuh"

namespace hdg {

struct ColsArgs {
  const void* rec;     // record array of the level (type TS)
  const void* v;       // X [ndof][nb] (type TV)
  const void* cvec;    // C [ndof][nb] (type TV) or nullptr
  void* y;             // Y [ndof][nb] (type TV)
  double alpha, beta;
  int nx, ny, spr, nseg, nb;
};

constexpr int kColsThreads = 256;

// rows of the staged blocks of one element: R = 16 (p+1)^2 entries
template <int N1>
struct ColsShape {
  static constexpr int M = 4 * N1, R = 16 * N1 * N1;
};

template <typename TS>
struct alignas(4 * sizeof(TS)) Quad {
  TS v[4];
};

// type of the staged blocks: BF16 records are widened to float as they are
// staged (once per CTA) instead of in the product loop, where every lane of a
// warp would convert the same broadcast entries again
template <typename TS> struct StagedT { using type = TS; };
template <> struct StagedT<__nv_bfloat16> { using type = float; };
__device__ __forceinline__ float stage_conv(__nv_bfloat16 v, float) { return __bfloat162float(v); }
template <typename TS>
__device__ __forceinline__ TS stage_conv(TS v, TS) { return v; }

// columns per lane: float accumulators take two (one block load feeds two
// FMAs), the wider double / double-float accumulators one
template <typename TA>
struct ColsPerLane { static constexpr int value = sizeof(TA) == 4 ? 2 : 1; };

// registers sized for three CTAs per SM (85 per thread): at k >= 5 this spills a
// few hundred bytes, and is still faster than two CTAs without spills (measured
// at 256 x 256, k = 5, 64 right-hand sides, all precisions)
template <int N1, typename TS, typename TV, typename TA, bool DIFF>
__global__ void __launch_bounds__(kColsThreads, 3) apply_cols_kernel(ColsArgs a) {
  using TO = typename OutT<TA>::type;
  constexpr int M = ColsShape<N1>::M, R = ColsShape<N1>::R;
  constexpr int CPL = ColsPerLane<TA>::value;
  constexpr int VEC = 16 / sizeof(TS);             // entries per 16-byte global load
  using TSS = typename StagedT<TS>::type;
  extern __shared__ __align__(128) unsigned char cols_smem[];
  TSS* sS = reinterpret_cast<TSS*>(cols_smem);     // [16][R], element-major
  const int seg = blockIdx.x;
  // stage: global [(seg*R + r)*16 + t] -> sS[t*R + r], up to 8 16-byte loads
  // in flight per thread before their stores
  {
    const uint4* g = reinterpret_cast<const uint4*>((const TS*)a.rec + (size_t)seg * R * kSeg);
    constexpr int NV = R * kSeg / VEC;
    constexpr int PER = (NV + kColsThreads - 1) / kColsThreads;
    constexpr int BATCH = PER < 8 ? PER : 8;
#pragma unroll 1
    for (int b0 = 0; b0 < PER; b0 += BATCH) {
      union Pk { uint4 u; TS s[VEC]; };
      Pk buf[BATCH];
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        const int idx = (b0 + u) * kColsThreads + (int)threadIdx.x;
        if (b0 + u < PER && idx < NV) buf[u].u = __ldg(g + idx);
      }
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        const int idx = (b0 + u) * kColsThreads + (int)threadIdx.x;
        if (b0 + u < PER && idx < NV) {
          const int r = (idx * VEC) / kSeg, t0 = (idx * VEC) % kSeg;
#pragma unroll
          for (int q = 0; q < VEC; ++q) sS[(t0 + q) * R + r] = stage_conv(buf[u].s[q], TSS{});
        }
      }
    }
  }
  __syncthreads();
  const int nx = a.nx, ny = a.ny, nv = (nx + 1) * ny, nb = a.nb;
  const int j = seg / a.spr, i0 = (seg % a.spr) * kSeg;
  constexpr int CPW = 32 * CPL;                    // columns per warp item
  const int nchunk = (nb + CPW - 1) / CPW;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TV* __restrict__ v = (const TV*)a.v;
  const TV* __restrict__ cv = (const TV*)a.cvec;
  TV* __restrict__ y = (TV*)a.y;
  const TO al = (TO)a.alpha, be = (TO)a.beta;
  // y = A v, y = c - A v and y = c + A v take no multiply (FP64 ops are slow here)
  const int form = (al == TO(1) && (!cv || be == TO(0))) ? 0
                   : (cv && be == TO(1) && al == TO(-1)) ? 1 : (cv && be == TO(1) && al == TO(1)) ? 2 : 3;
  // two float columns per lane with nb a multiple of 64: the lane's columns are
  // adjacent, every row of x, y and c one float2 access per lane
  const bool pair = CPL == 2 && sizeof(TV) == 4 && (nb % CPW) == 0 &&
                    (((uintptr_t)a.v | (uintptr_t)a.cvec | (uintptr_t)a.y) & 7) == 0;
  for (int item = warp; item < 32 * nchunk; item += (kColsThreads >> 5)) {
    // warp-uniform: element t of the segment, owned face (W or S), column chunk
    const int chunk = item >> 5, face = (item >> 4) & 1, t = item & 15;
    const int i = i0 + t;
    if (i >= nx) continue;
    int colc[CPL];
    bool live[CPL];
#pragma unroll
    for (int u = 0; u < CPL; ++u) {
      // paired columns (2 lane, 2 lane + 1) move as one 8-byte access
      const int col = pair ? chunk * CPW + 2 * lane + u : chunk * CPW + u * 32 + lane;
      live[u] = col < nb;
      colc[u] = live[u] ? col : nb - 1;            // dead lanes load a valid column
    }
    const bool bndrow = face == 0 ? (i == 0) : (j == 0);
    const int eout = face == 0 ? i + (nx + 1) * j : nv + i + nx * j;
    TO cpre[CPL][N1];
#pragma unroll
    for (int u = 0; u < CPL; ++u)
#pragma unroll
      for (int q = 0; q < N1; ++q) cpre[u][q] = TO(0);
    TA acc[CPL][N1];
#pragma unroll
    for (int u = 0; u < CPL; ++u)
#pragma unroll
      for (int q = 0; q < N1; ++q) acc[u][q] = TA{};
    if (!bndrow) {
#pragma unroll(CPL == 2 ? 2 : 1)
      for (int side = 0; side < 2; ++side) {
        const int ki = (side == 1 && face == 0) ? i - 1 : i;
        const int kj = (side == 1 && face == 1) ? j - 1 : j;
        int edge[4];
        bool bnd[4];
        edge[0] = ki + (nx + 1) * kj;       bnd[0] = ki <= 0;
        edge[1] = ki + 1 + (nx + 1) * kj;   bnd[1] = ki >= nx - 1;
        edge[2] = nv + ki + nx * kj;        bnd[2] = kj <= 0;
        edge[3] = nv + ki + nx * (kj + 1);  bnd[3] = kj >= ny - 1;
        TA xv[CPL][M];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          if (!bnd[f]) {                           // warp-uniform branch
            const TV* bp = v + (size_t)edge[f] * N1 * nb;
            if constexpr (CPL == 2 && sizeof(TV) == 4) {
              if (pair) {
                const float2* bp2 = reinterpret_cast<const float2*>(bp + colc[0]);
#pragma unroll
                for (int b = 0; b < N1; ++b) {
                  const float2 w2 = bp2[(size_t)b * (nb >> 1)];
                  xv[0][f * N1 + b] = to_acc(w2.x, TA{});
                  xv[1][f * N1 + b] = to_acc(w2.y, TA{});
                }
                continue;
              }
            }
#pragma unroll
            for (int b = 0; b < N1; ++b)
#pragma unroll
              for (int u = 0; u < CPL; ++u) xv[u][f * N1 + b] = to_acc(bp[(size_t)b * nb + colc[u]], TA{});
          } else {
#pragma unroll
            for (int b = 0; b < N1; ++b)
#pragma unroll
              for (int u = 0; u < CPL; ++u) xv[u][f * N1 + b] = TA{};
          }
        }
        if constexpr (DIFF) {
          // S_K 1 = 0: apply the block to x - mean(x) 1 (boundary entries count as
          // 0), so the rounded FP32 / BF16 entries see the variation of x over the
          // element rather than its (smooth, large) value
#pragma unroll
          for (int u = 0; u < CPL; ++u) {
            TA mean = TA(0);
#pragma unroll
            for (int c = 0; c < M; ++c) mean += xv[u][c];
            mean *= TA(1.0 / M);
#pragma unroll
            for (int c = 0; c < M; ++c) xv[u][c] -= mean;
          }
        }
        if (side == 1 && cv) {
          // the addend's loads are issued before the last products so their
          // latency overlaps them
          bool done = false;
          if constexpr (CPL == 2 && sizeof(TV) == 4) {
            if (pair) {
              const float2* cp2 = reinterpret_cast<const float2*>(cv + (size_t)eout * N1 * nb + colc[0]);
#pragma unroll
              for (int q = 0; q < N1; ++q) {
                const float2 w2 = cp2[(size_t)q * (nb >> 1)];
                cpre[0][q] = (TO)w2.x;
                cpre[1][q] = (TO)w2.y;
              }
              done = true;
            }
          }
          if (!done) {
#pragma unroll
            for (int u = 0; u < CPL; ++u)
#pragma unroll
              for (int q = 0; q < N1; ++q) cpre[u][q] = (TO)cv[((size_t)eout * N1 + q) * nb + colc[u]];
          }
        }
        const TSS* rows = sS + t * R + (face * 2 + side) * N1 * M;
#pragma unroll
        for (int q = 0; q < N1; ++q)
#pragma unroll
          for (int c = 0; c < M; c += 4) {
            const Quad<TSS> s4 = *reinterpret_cast<const Quad<TSS>*>(rows + q * M + c);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              const TA sv = to_acc(s4.v[w], TA{});
#pragma unroll
              for (int u = 0; u < CPL; ++u) acc[u][q] = mac(sv, xv[u][c + w], acc[u][q]);
            }
          }
      }
    }
    TO outv[CPL][N1];
#pragma unroll
    for (int u = 0; u < CPL; ++u)
#pragma unroll
      for (int q = 0; q < N1; ++q) {
        TO val = TO(0);
        if (!bndrow) {
          const TO sum = finish(acc[u][q]);
          if (form == 0) val = sum;
          else if (form == 1) val = cpre[u][q] - sum;
          else if (form == 2) val = cpre[u][q] + sum;
          else {
            val = al * sum;
            if (cv) val = mac(be, cpre[u][q], val);
          }
        }
        outv[u][q] = val;
      }
    if constexpr (CPL == 2 && sizeof(TV) == 4) {
      if (pair) {
        float2* yp2 = reinterpret_cast<float2*>(y + (size_t)eout * N1 * nb + colc[0]);
#pragma unroll
        for (int q = 0; q < N1; ++q) yp2[(size_t)q * (nb >> 1)] = make_float2((float)outv[0][q], (float)outv[1][q]);
      }
    }
#pragma unroll
    for (int u = 0; u < CPL; ++u) {
      if (!live[u]) continue;
      const int col = colc[u];
      if (!pair) {
#pragma unroll
        for (int q = 0; q < N1; ++q) y[((size_t)eout * N1 + q) * nb + col] = (TV)outv[u][q];
      }
      // the E / N domain-boundary edges have no owner element: zero them here
      if (face == 0 && i == nx - 1) {
        const size_t eb = (size_t)nx + (size_t)(nx + 1) * j;
#pragma unroll
        for (int q = 0; q < N1; ++q) y[(eb * N1 + q) * nb + col] = TV(0);
      }
      if (face == 1 && j == ny - 1) {
        const size_t eb = (size_t)nv + i + (size_t)nx * ny;
#pragma unroll
        for (int q = 0; q < N1; ++q) y[(eb * N1 + q) * nb + col] = TV(0);
      }
    }
  }
}

template <int N1, typename TS, typename TV, typename TA, bool DIFF>
cudaError_t cols_launch(const Context* c, const ColsArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)ColsShape<N1>::R * kSeg * sizeof(typename StagedT<TS>::type);
  if ((size_t)c->smem_optin < smem) return cudaErrorInvalidValue;
  auto kern = apply_cols_kernel<N1, TS, TV, TA, DIFF>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, c->smem_optin);
  if (e != cudaSuccess) return e;
  if (a.nseg <= 0) return cudaSuccess;
  kern<<<a.nseg, kColsThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename TS, typename TV, typename TA, bool DIFF>
cudaError_t cols_dispatch(const Context* c, int n1, const ColsArgs& a, cudaStream_t s) {
  switch (n1) {
    case 1: return cols_launch<1, TS, TV, TA, DIFF>(c, a, s);
    case 2: return cols_launch<2, TS, TV, TA, DIFF>(c, a, s);
    case 3: return cols_launch<3, TS, TV, TA, DIFF>(c, a, s);
    case 4: return cols_launch<4, TS, TV, TA, DIFF>(c, a, s);
    case 5: return cols_launch<5, TS, TV, TA, DIFF>(c, a, s);
    case 6: return cols_launch<6, TS, TV, TA, DIFF>(c, a, s);
    case 7: return cols_launch<7, TS, TV, TA, DIFF>(c, a, s);
    case 8: return cols_launch<8, TS, TV, TA, DIFF>(c, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t cols_fp64(const Context* c, int n1, bool diff, const ColsArgs& a, cudaStream_t s);
cudaError_t cols_fp32(const Context* c, int n1, bool diff, const ColsArgs& a, cudaStream_t s);
cudaError_t cols_bf16(const Context* c, int n1, bool diff, const ColsArgs& a, cudaStream_t s);
cudaError_t cols_x2(const Context* c, int n1, bool diff, const ColsArgs& a, cudaStream_t s);

}  // namespace hdg
