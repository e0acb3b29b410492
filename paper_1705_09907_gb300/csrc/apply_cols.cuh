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

template <int N1, typename TS, typename TV, typename TA, bool DIFF>
__device__ __forceinline__ void cols_gather(const TV* __restrict__ v, int ki, int kj, int col, bool live,
                                            const ColsArgs& a, TA (&xv)[4 * N1]) {
  const int nx = a.nx, ny = a.ny, nv = (nx + 1) * ny, nb = a.nb;
  int edge[4];
  bool bnd[4];
  edge[0] = ki + (nx + 1) * kj;       bnd[0] = ki <= 0;
  edge[1] = ki + 1 + (nx + 1) * kj;   bnd[1] = ki >= nx - 1;
  edge[2] = nv + ki + nx * kj;        bnd[2] = kj <= 0;
  edge[3] = nv + ki + nx * (kj + 1);  bnd[3] = kj >= ny - 1;
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int b = 0; b < N1; ++b)
      xv[f * N1 + b] = (bnd[f] || !live) ? TA{} : to_acc(v[((size_t)edge[f] * N1 + b) * nb + col], TA{});
  if constexpr (DIFF) {
    TA mean = TA(0);
#pragma unroll
    for (int c = 0; c < 4 * N1; ++c) mean += xv[c];
    mean *= TA(1.0 / (4 * N1));
#pragma unroll
    for (int c = 0; c < 4 * N1; ++c) xv[c] -= mean;
  }
}

template <int N1, typename TS, typename TV, typename TA, bool DIFF>
__global__ void __launch_bounds__(kColsThreads) apply_cols_kernel(ColsArgs a) {
  using TO = typename OutT<TA>::type;
  constexpr int M = ColsShape<N1>::M, R = ColsShape<N1>::R;
  constexpr int VEC = 16 / sizeof(TS);             // entries per 16-byte global load
  extern __shared__ __align__(128) unsigned char cols_smem[];
  TS* sS = reinterpret_cast<TS*>(cols_smem);       // [16][R], element-major
  const int seg = blockIdx.x;
  // stage: global [(seg*R + r)*16 + t] -> sS[t*R + r]
  {
    const uint4* g = reinterpret_cast<const uint4*>((const TS*)a.rec + (size_t)seg * R * kSeg);
    constexpr int NV = R * kSeg / VEC;
    for (int idx = threadIdx.x; idx < NV; idx += blockDim.x) {
      union { uint4 u; TS s[VEC]; } pk;
      pk.u = __ldg(g + idx);
      const int r = (idx * VEC) / kSeg, t0 = (idx * VEC) % kSeg;
#pragma unroll
      for (int q = 0; q < VEC; ++q) sS[(t0 + q) * R + r] = pk.s[q];
    }
  }
  __syncthreads();
  const int nx = a.nx, ny = a.ny, nv = (nx + 1) * ny, nb = a.nb;
  const int j = seg / a.spr, i0 = (seg % a.spr) * kSeg;
  const int nchunk = (nb + 31) >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TV* __restrict__ v = (const TV*)a.v;
  const TV* __restrict__ cv = (const TV*)a.cvec;
  TV* __restrict__ y = (TV*)a.y;
  const TO al = (TO)a.alpha, be = (TO)a.beta;
  for (int item = warp; item < 32 * nchunk; item += (kColsThreads >> 5)) {
    const int chunk = item >> 5, face = (item >> 4) & 1, t = item & 15;
    const int i = i0 + t;
    if (i >= nx) continue;
    const int col = chunk * 32 + lane;
    const bool live = col < nb;
    const bool bndrow = face == 0 ? (i == 0) : (j == 0);
    TA acc[N1];
#pragma unroll
    for (int q = 0; q < N1; ++q) acc[q] = TA{};
    if (!bndrow) {
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int ki = (side == 1 && face == 0) ? i - 1 : i;
        const int kj = (side == 1 && face == 1) ? j - 1 : j;
        TA xv[M];
        cols_gather<N1, TS, TV, TA, DIFF>(v, ki, kj, col, live, a, xv);
        const TS* rows = sS + t * R + (face * 2 + side) * N1 * M;
#pragma unroll
        for (int q = 0; q < N1; ++q)
#pragma unroll
          for (int c = 0; c < M; c += 4) {
            const Quad<TS> s4 = *reinterpret_cast<const Quad<TS>*>(rows + q * M + c);
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[q] = mac(to_acc(s4.v[u], TA{}), xv[c + u], acc[q]);
          }
      }
    }
    if (!live) continue;
    const int eout = face == 0 ? i + (nx + 1) * j : nv + i + nx * j;
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      const size_t o = ((size_t)eout * N1 + q) * nb + col;
      TO val = TO(0);
      if (!bndrow) {
        val = al * finish(acc[q]);
        if (cv) val = mac(be, (TO)cv[o], val);
      }
      y[o] = (TV)val;
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

template <int N1, typename TS, typename TV, typename TA, bool DIFF>
cudaError_t cols_launch(const Context* c, const ColsArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)ColsShape<N1>::R * kSeg * sizeof(TS);
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
