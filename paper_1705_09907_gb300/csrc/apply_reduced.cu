// Condensed-block apply on symmetry-reduced element blocks.
//
// On a rectangle with a constant coefficient and a constant tau, the local
// problem of Eqs. shur0/shur1 is invariant under the reflections x -> -x and
// y -> -y about the element centre, and the Gauss-Legendre trace nodes of each
// face are symmetric. So every S_K commutes with both reflections acting on the
// face dofs [W | E | S | N] (nodes in increasing coordinate):
//   sigma_x: W <-> E (node order kept), S and N reversed,
//   sigma_y: S <-> N (node order kept), W and E reversed.
// In the coordinates t = F x built from face sums/differences (P = W + E,
// M = W - E, P' = S + N, M' = S - N) and then node-pair sums/differences on
// each of them (even part: v_i + v_{n-1-i} and the middle node, odd part:
// v_i - v_{n-1-i}), S_K is block diagonal with one block per character of the
// group (sigma_x, sigma_y) = (+,+), (+,-), (-,+), (-,-):
//   B0 on [even P, even P'],  B1 on [odd P, even M'],
//   B2 on [even M, odd P'],   B3 on [odd M, odd M'].
// F has orthogonal rows of +-1 entries, F F^T = D (the number of dofs each
// coordinate combines), so with B = D^-1 F S_K F^T D^-1:
//   S_K x = F^T B (F x).
// The blocks are symmetric and stored as packed upper triangles: at k = 4
// 61 numbers per element instead of the 400 of S_K (5 / 12 / 25 / 40 / 61 /
// 84 / 113 / 144 for k = 0..7), and a product costs sum d_b^2 multiply-adds
// plus 16(k+1) additions for F and F^T instead of 16(k+1)^2 multiply-adds.
//
// The apply y = beta c + alpha sum_{K} A_K^T S_K A_K v (boundary dofs of v
// ignored, boundary rows of y zero) writes every face once, as its own
// element's output plus its neighbour's (W face: own + west neighbour's E; S
// face: own + south neighbour's N), with no atomics. One thread computes one
// element product at a time. Two forms with identical results:
//   reduced = 1: every element product to a scratch [4n][nel], then every face
//      (the faster form on GB300: many small independent CTAs keep more loads
//      in flight; the scratch round trip mostly stays in L2).
//   reduced = 2: one CTA per 32 x kTileRows tile finishes every face inside the
//      tile (shuffles across the row, registers and shared memory up the
//      column); the faces on tile edges go through a small second launch.
// The blocks are read once, directly from HBM with coalesced streaming loads
// (warp chunks [nel/32][Q][32]: the 32 lanes of a warp read 32 consecutive
// elements' entry q, and a warp's Q entries are one contiguous chunk; the FP32
// copy keeps four entries of an element together, [nel/32][Q/4][32][4], and is
// read as float4 before any arithmetic).
#include "reduced_impl.cuh"

namespace hdg {

namespace {

using namespace red;

template <int N1, typename TS, typename T, bool DIFF>
__global__ void __launch_bounds__(kElemThreads) reduced_elem_kernel(const RedArgs a) {
  elem_body<N1, TS, T, DIFF>(a, blockIdx.x * (long)kElemThreads + threadIdx.x);
}

template <int N1, typename T>
__global__ void __launch_bounds__(kFaceThreads) reduced_face_kernel(const RedArgs a) {
  __shared__ T sw[kFaceThreads * N1], ss[kFaceThreads * N1];
  face_body<N1, T>(a, blockIdx.x * (long)kFaceThreads, threadIdx.x, sw, ss);
}

// One tile per CTA (reduced = 2): 32 columns (the lanes) x kTileRows rows;
// warp w walks rows w*kRowsPerWarp.. upwards. Each face that has both of its
// elements in the tile is finished here: the W face takes the E output of the
// lane to its left (shuffle), the S face the N output of the row below (the
// same thread's previous row, or the warp below through shared memory). The
// faces on the tile's left column and bottom row park their own contribution
// in the scratch, as do the tile's right column (E) and top row (N) for the
// neighbouring tiles; reduced_fix_kernel finishes those faces. The sums are
// taken in the same order as in the two-launch form (own element first), so
// both forms give identical results.
constexpr int kTileWarps = 2, kRowsPerWarp = 4, kTileRows = kTileWarps * kRowsPerWarp;

// the value of the lane to the left (lane 0 keeps its own)
template <typename T>
__device__ __forceinline__ T shfl_up1(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ dd shfl_up1(dd v) {
  return dd(__shfl_up_sync(0xffffffffu, v.hi, 1), __shfl_up_sync(0xffffffffu, v.lo, 1));
}

template <int N1, typename TS, typename T, bool DIFF>
__global__ void __launch_bounds__(32 * kTileWarps) reduced_tile_kernel(const RedArgs a) {
  __shared__ T north[kTileWarps][N1][32];
  const int nx = a.nx, ny = a.ny;
  const long nel = (long)nx * ny;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int tiles_x = (nx + 31) >> 5;
  const int bx = blockIdx.x % tiles_x, by = blockIdx.x / tiles_x;
  const int i = bx * 32 + lane;
  const int j0 = by * kTileRows + w * kRowsPerWarp;
  const bool col = i < nx;
  using VT = typename VecT<T>::type;
  T* __restrict__ z = (T*)a.z;
  VT* __restrict__ y = (VT*)a.y;
  const Form<VT> form(a);
  const long nv = (long)(nx + 1) * ny;
  T zn_prev[N1], zs_first[N1];
#pragma unroll
  for (int q = 0; q < N1; ++q) { zn_prev[q] = T(0); zs_first[q] = T(0); }
  int rows = 0;
#pragma unroll 1
  for (int r = 0; r < kRowsPerWarp; ++r) {
    const int j = j0 + r;
    if (j >= ny) break;                                   // warp-uniform
    ++rows;
    const long K = i + (long)nx * j;
    T zw[N1], ze[N1], zs[N1], zn[N1];
    if (col) {
      elem_product<N1, TS, T, DIFF>(a, nel, K, i, j, zw, ze, zs, zn);
    } else {
#pragma unroll
      for (int q = 0; q < N1; ++q) { zw[q] = T(0); ze[q] = T(0); zs[q] = T(0); zn[q] = T(0); }
    }
    T ew[N1];                                             // E output of the element to the left
#pragma unroll
    for (int q = 0; q < N1; ++q) ew[q] = shfl_up1(ze[q]);
    if (col) {
      const long eW = i + (long)(nx + 1) * j, eS = nv + i + (long)nx * j;
      // W face
      if (i == 0) {
#pragma unroll
        for (int q = 0; q < N1; ++q) y[eW * N1 + q] = VT(0);
      } else if (lane == 0) {
#pragma unroll
        for (int q = 0; q < N1; ++q) z[(size_t)(0 * N1 + q) * nel + K] = zw[q];
      } else {
#pragma unroll
        for (int q = 0; q < N1; ++q) y[eW * N1 + q] = form(to_vec(zw[q] + ew[q]), (size_t)eW * N1 + q);
      }
      if (lane == 31 && i < nx - 1) {
#pragma unroll
        for (int q = 0; q < N1; ++q) z[(size_t)(1 * N1 + q) * nel + K] = ze[q];
      }
      if (i == nx - 1) {
#pragma unroll
        for (int q = 0; q < N1; ++q) y[(eW + 1) * N1 + q] = VT(0);
      }
      // S face
      if (j == 0) {
#pragma unroll
        for (int q = 0; q < N1; ++q) y[eS * N1 + q] = VT(0);
      } else if (r > 0) {
#pragma unroll
        for (int q = 0; q < N1; ++q) y[eS * N1 + q] = form(to_vec(zs[q] + zn_prev[q]), (size_t)eS * N1 + q);
      } else if (w > 0) {
#pragma unroll
        for (int q = 0; q < N1; ++q) zs_first[q] = zs[q];
      } else {
#pragma unroll
        for (int q = 0; q < N1; ++q) z[(size_t)(2 * N1 + q) * nel + K] = zs[q];
      }
      if (j == ny - 1) {
#pragma unroll
        for (int q = 0; q < N1; ++q) y[(eS + nx) * N1 + q] = VT(0);
      } else if (w == kTileWarps - 1 && r == kRowsPerWarp - 1) {
#pragma unroll
        for (int q = 0; q < N1; ++q) z[(size_t)(3 * N1 + q) * nel + K] = zn[q];
      }
    }
#pragma unroll
    for (int q = 0; q < N1; ++q) zn_prev[q] = zn[q];
  }
  // the N outputs of each warp's last row, for the first row of the warp above
  if (rows == kRowsPerWarp) {
#pragma unroll
    for (int q = 0; q < N1; ++q) north[w][q][lane] = zn_prev[q];
  }
  __syncthreads();
  if (w > 0 && rows > 0 && col && j0 > 0) {
    const long eS = nv + i + (long)nx * j0;
#pragma unroll
    for (int q = 0; q < N1; ++q) y[eS * N1 + q] = form(to_vec(zs_first[q] + north[w - 1][q][lane]), (size_t)eS * N1 + q);
  }
}

// The faces on tile edges: W faces of columns 32, 64, .. and S faces of rows
// kTileRows, 2 kTileRows, .. (own contribution + the neighbour's, as above).
template <int N1, typename T>
__global__ void __launch_bounds__(256) reduced_fix_kernel(const RedArgs a) {
  const int nx = a.nx, ny = a.ny;
  const long nel = (long)nx * ny;
  const int tiles_x = (nx + 31) >> 5, tiles_y = (ny + kTileRows - 1) / kTileRows;
  const long nvert = (long)(tiles_x - 1) * ny, total = nvert + (long)(tiles_y - 1) * nx;
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= total) return;
  using VT = typename VecT<T>::type;
  const T* __restrict__ z = (const T*)a.z;
  VT* __restrict__ y = (VT*)a.y;
  const Form<VT> form(a);
  long e, K, Kn;
  int fo;
  if (t < nvert) {
    const int j = (int)(t / (tiles_x - 1)), i = 32 * (int)(t % (tiles_x - 1) + 1);
    K = i + (long)nx * j; Kn = K - 1; fo = 0;
    e = i + (long)(nx + 1) * j;
  } else {
    const long u = t - nvert;
    const int i = (int)(u % nx), j = kTileRows * (int)(u / nx + 1);
    K = i + (long)nx * j; Kn = K - nx; fo = 2;
    e = (long)(nx + 1) * ny + i + (long)nx * j;
  }
#pragma unroll
  for (int q = 0; q < N1; ++q)
    y[e * N1 + q] = form(to_vec(z[(size_t)(fo * N1 + q) * nel + K] + z[(size_t)((fo + 1) * N1 + q) * nel + Kn]),
                         (size_t)e * N1 + q);
}

template <int N1, typename TS, typename T, bool DIFF>
cudaError_t red_launch(const RedArgs& a, long nel, int mode, cudaStream_t s) {
  if (mode == 1) {
    const unsigned g1 = (unsigned)((nel + kElemThreads - 1) / kElemThreads),
                   g2 = (unsigned)((nel + kFaceThreads - 1) / kFaceThreads);
    reduced_elem_kernel<N1, TS, T, DIFF><<<g1, kElemThreads, 0, s>>>(a);
    HDG_CUDA_TRY(cudaGetLastError());
    reduced_face_kernel<N1, T><<<g2, kFaceThreads, 0, s>>>(a);
    return cudaGetLastError();
  }
  const int tiles_x = (a.nx + 31) / 32, tiles_y = (a.ny + kTileRows - 1) / kTileRows;
  reduced_tile_kernel<N1, TS, T, DIFF><<<(unsigned)(tiles_x * tiles_y), 32 * kTileWarps, 0, s>>>(a);
  HDG_CUDA_TRY(cudaGetLastError());
  const long fix = (long)(tiles_x - 1) * a.ny + (long)(tiles_y - 1) * a.nx;
  if (fix > 0) {
    reduced_fix_kernel<N1, T><<<(unsigned)((fix + 255) / 256), 256, 0, s>>>(a);
    HDG_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

template <typename TS, typename T, bool DIFF>
cudaError_t red_dispatch(int n1, const RedArgs& a, long nel, int mode, cudaStream_t s) {
  switch (n1) {
    case 1: return red_launch<1, TS, T, DIFF>(a, nel, mode, s);
    case 2: return red_launch<2, TS, T, DIFF>(a, nel, mode, s);
    case 3: return red_launch<3, TS, T, DIFF>(a, nel, mode, s);
    case 4: return red_launch<4, TS, T, DIFF>(a, nel, mode, s);
    case 5: return red_launch<5, TS, T, DIFF>(a, nel, mode, s);
    case 6: return red_launch<6, TS, T, DIFF>(a, nel, mode, s);
    case 7: return red_launch<7, TS, T, DIFF>(a, nel, mode, s);
    case 8: return red_launch<8, TS, T, DIFF>(a, nel, mode, s);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// Set-up: reduced blocks from the dense element blocks.
struct Coord {
  int dof[4];
  double sg[4];
  int cnt;
};

// coordinate `idx` of block b (see the file comment): the face dofs it
// combines and their signs
__device__ Coord coord_of(int n1, int b, int idx) {
  const int h = n1 / 2, se = h + (n1 & 1), so = h;
  // (face pair: 0 = W/E, 1 = S/N; face sign; node parity 0 = even, 1 = odd; node index)
  int pair, fsg, par, nd;
  const int first = (b == 0) ? se : (b == 1) ? so : (b == 2) ? se : so;
  const bool lo = idx < first;
  const int ii = lo ? idx : idx - first;
  switch (b) {
    case 0: pair = lo ? 0 : 1; fsg = 1; par = 0; break;
    case 1: pair = lo ? 0 : 1; fsg = lo ? 1 : -1; par = lo ? 1 : 0; break;
    case 2: pair = lo ? 0 : 1; fsg = lo ? -1 : 1; par = lo ? 0 : 1; break;
    default: pair = lo ? 0 : 1; fsg = -1; par = 1; break;
  }
  nd = ii;
  const int f1 = pair == 0 ? 0 : 2, f2 = f1 + 1;
  Coord c{};
  if (par == 0 && (n1 & 1) && nd == h) {        // middle node
    c.dof[0] = f1 * n1 + h; c.sg[0] = 1.0;
    c.dof[1] = f2 * n1 + h; c.sg[1] = (double)fsg;
    c.cnt = 2;
  } else {
    const double ns = par == 0 ? 1.0 : -1.0;
    c.dof[0] = f1 * n1 + nd;          c.sg[0] = 1.0;
    c.dof[1] = f1 * n1 + n1 - 1 - nd; c.sg[1] = ns;
    c.dof[2] = f2 * n1 + nd;          c.sg[2] = (double)fsg;
    c.dof[3] = f2 * n1 + n1 - 1 - nd; c.sg[3] = (double)fsg * ns;
    c.cnt = 4;
  }
  return c;
}

__global__ void reduced_blocks_kernel(long nel, int n1, const double* __restrict__ Sd, double* __restrict__ R64,
                                      float* __restrict__ R32, float2* __restrict__ R2) {
  const int h = n1 / 2, se = h + (n1 & 1), so = h;
  const int d[4] = {2 * se, so + se, se + so, 2 * so};
  int Q = 0;
  for (int b = 0; b < 4; ++b) Q += d[b] * (d[b] + 1) / 2;
  const int m = 4 * n1;
  const long total = nel * Q;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int q = (int)(t / nel);
    const long K = t % nel;
    // q -> (block, row, column) of the packed upper triangles
    int b = 0, r = q;
    while (r >= d[b] * (d[b] + 1) / 2) { r -= d[b] * (d[b] + 1) / 2; ++b; }
    int ii = 0;
    while (r >= d[b] - ii) { r -= d[b] - ii; ++ii; }
    const int jj = ii + r;
    const Coord ci = coord_of(n1, b, ii), cj = coord_of(n1, b, jj);
    const double* S = Sd + (size_t)K * m * m;
    double acc = 0.0;
    for (int x = 0; x < ci.cnt; ++x)
      for (int y = 0; y < cj.cnt; ++y) acc += ci.sg[x] * cj.sg[y] * S[ci.dof[x] * m + cj.dof[y]];
    const double val = acc / (double)(ci.cnt * cj.cnt);
    R64[red_base(K, Q) + (size_t)q * 32] = val;
    if (R32) R32[red_index32(K, Q, q)] = (float)val;
    if (R2) {
      const float hi = (float)val;
      R2[red_base(K, Q) + (size_t)q * 32] = make_float2(hi, (float)(val - (double)hi));
    }
  }
}

constexpr int kColsWarps = 4;             // elements per CTA of the column kernels

template <int N1, typename TS, typename T, bool DIFF>
__global__ void __launch_bounds__(32 * kColsWarps) reduced_cols_elem_kernel(const RedArgs a, int nb) {
  cols_elem_body<N1, TS, T, DIFF>(a, blockIdx.x * (long)kColsWarps + (threadIdx.x >> 5), nb,
                                  blockIdx.y * 32 + (threadIdx.x & 31));
}

template <int N1, typename T>
__global__ void __launch_bounds__(32 * kColsWarps) reduced_cols_face_kernel(const RedArgs a, int nb) {
  cols_face_body<N1, T>(a, blockIdx.x * (long)kColsWarps + (threadIdx.x >> 5), nb,
                        blockIdx.y * 32 + (threadIdx.x & 31));
}

template <int N1, typename TS, typename T, bool DIFF>
cudaError_t red_cols_launch(const RedArgs& a, long nel, int nb, cudaStream_t s) {
  const dim3 g((unsigned)((nel + kColsWarps - 1) / kColsWarps), (unsigned)((nb + 31) / 32));
  reduced_cols_elem_kernel<N1, TS, T, DIFF><<<g, 32 * kColsWarps, 0, s>>>(a, nb);
  HDG_CUDA_TRY(cudaGetLastError());
  reduced_cols_face_kernel<N1, T><<<g, 32 * kColsWarps, 0, s>>>(a, nb);
  return cudaGetLastError();
}

template <typename TS, typename T, bool DIFF>
cudaError_t red_cols_dispatch(int n1, const RedArgs& a, long nel, int nb, cudaStream_t s) {
  switch (n1) {
    case 1: return red_cols_launch<1, TS, T, DIFF>(a, nel, nb, s);
    case 2: return red_cols_launch<2, TS, T, DIFF>(a, nel, nb, s);
    case 3: return red_cols_launch<3, TS, T, DIFF>(a, nel, nb, s);
    case 4: return red_cols_launch<4, TS, T, DIFF>(a, nel, nb, s);
    case 5: return red_cols_launch<5, TS, T, DIFF>(a, nel, nb, s);
    case 6: return red_cols_launch<6, TS, T, DIFF>(a, nel, nb, s);
    case 7: return red_cols_launch<7, TS, T, DIFF>(a, nel, nb, s);
    case 8: return red_cols_launch<8, TS, T, DIFF>(a, nel, nb, s);
    default: return cudaErrorInvalidValue;
  }
}

// dth_K = -psi_K^T (S_K lambda_K): the reduced product of lambda, dotted with
// the element's four faces of psi (boundary faces read as zero)
template <int N1>
__global__ void __launch_bounds__(kElemThreads) reduced_theta_kernel(const RedArgs a, const double* __restrict__ psi,
                                                                     double* __restrict__ dth) {
  const int nx = a.nx, ny = a.ny;
  const long nel = (long)nx * ny;
  const long K = blockIdx.x * (long)kElemThreads + threadIdx.x;
  if (K >= nel) return;
  const int i = (int)(K % nx), j = (int)(K / nx);
  double zw[N1], ze[N1], zs[N1], zn[N1];
  elem_product<N1, double, double, false>(a, nel, K, i, j, zw, ze, zs, zn);
  const long eW = i + (long)(nx + 1) * j, eS = (long)(nx + 1) * ny + i + (long)nx * j;
  double d = 0.0;
#pragma unroll
  for (int q = 0; q < N1; ++q) {
    if (i > 0) d = fma(psi[eW * N1 + q], zw[q], d);
    if (i < nx - 1) d = fma(psi[(eW + 1) * N1 + q], ze[q], d);
    if (j > 0) d = fma(psi[eS * N1 + q], zs[q], d);
    if (j < ny - 1) d = fma(psi[(eS + nx) * N1 + q], zn[q], d);
  }
  dth[K] = -d;
}

// ---------------------------------------------------------------------------
// Schwarz blocks of the float cycles, packed. A weighted patch inverse
// M_K = W A_patch^-1 W is symmetric but has none of the reflection symmetry of
// S_K (the patch takes the neighbours' face blocks, whose coefficients differ),
// so it is stored as one packed upper triangle per element (m(m+1)/2 of its m^2
// entries, m = 4(k+1): 210 of 400 at k = 4) in the warp chunks of the reduced
// blocks, and applied like them: an element pass u_K = M_K x_K (each stored
// entry used for both of its positions) into the scratch, then the face pass of
// the reduced apply. The owner-record apply streams all m^2 entries; the float
// Schwarz applies are bandwidth bound, so this halves their block bytes.
__global__ void sym_pack_kernel(long nel, int m, const double* __restrict__ Md, float* __restrict__ Mp) {
  const int Q = m * (m + 1) / 2;
  const long total = nel * Q;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int q = (int)(t / nel);
    const long K = t % nel;
    int i = 0, r = q;
    while (r >= m - i) { r -= m - i; ++i; }
    const int j = i + r;
    const double* M = Md + (size_t)K * m * m;
    Mp[red_base(K, Q) + (size_t)q * 32] = (float)(0.5 * (M[i * m + j] + M[j * m + i]));
  }
}

template <int N1>
__global__ void __launch_bounds__(kElemThreads) sym_elem_kernel(const RedArgs a) {
  constexpr int D = 4 * N1, Q = D * (D + 1) / 2;
  const int nx = a.nx, ny = a.ny;
  const long nel = (long)nx * ny;
  const long K = blockIdx.x * (long)kElemThreads + threadIdx.x;
  if (K >= nel) return;
  const int i = (int)(K % nx), j = (int)(K / nx);
  const float* __restrict__ v = (const float*)a.v;
  const long eW = i + (long)(nx + 1) * j, eS = (long)(nx + 1) * ny + i + (long)nx * j;
  const bool has[4] = {i > 0, i < nx - 1, j > 0, j < ny - 1};
  const long ed[4] = {eW, eW + 1, eS, eS + nx};
  float x[D], u[D];
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int q = 0; q < N1; ++q) x[f * N1 + q] = has[f] ? __ldg(v + ed[f] * N1 + q) : 0.0f;
  // u = M x row by row of the packed triangle: a row's entries are loaded
  // together before its multiply-adds, so they are in flight at once (the
  // products and their order are those of sym_block)
  {
    const float* __restrict__ R = (const float*)a.R + red_base(K, Q);
#pragma unroll
    for (int r = 0; r < D; ++r) u[r] = 0.0f;
    int q = 0;
#pragma unroll
    for (int r = 0; r < D; ++r) {
      float e[D];
#pragma unroll
      for (int c = r; c < D; ++c) e[c] = __ldcs(R + (size_t)(q + c - r) * 32);
#pragma unroll
      for (int c = r; c < D; ++c) {
        u[r] = fmaf(e[c], x[c], u[r]);
        if (c != r) u[c] = fmaf(e[c], x[r], u[c]);
      }
      q += D - r;
    }
  }
  float* __restrict__ z = (float*)a.z;
#pragma unroll
  for (int r = 0; r < D; ++r) z[(size_t)r * nel + K] = u[r];
}

template <int N1>
cudaError_t sym_launch(const RedArgs& a, long nel, cudaStream_t s) {
  const unsigned g1 = (unsigned)((nel + kElemThreads - 1) / kElemThreads),
                 g2 = (unsigned)((nel + kFaceThreads - 1) / kFaceThreads);
  sym_elem_kernel<N1><<<g1, kElemThreads, 0, s>>>(a);
  HDG_CUDA_TRY(cudaGetLastError());
  reduced_face_kernel<N1, float><<<g2, kFaceThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_reduced_cols(Context* c, int p, int prec, const void* v, const void* cvec, void* y, double alpha,
                                double beta, int nb, void* z, cudaStream_t s) {
  PLevel& L = c->plev[p];
  RedArgs a{};
  a.v = v; a.cvec = cvec; a.y = y; a.z = z;
  a.alpha = alpha; a.beta = beta;
  a.nx = c->mesh.nx; a.ny = c->mesh.ny;
  if (prec == HDG_PREC_F32X2 && L.R2) {   // double-float product on the FP32 pipe
    a.R = L.R2;
    return red_cols_dispatch<float2, dd, false>(L.n1, a, c->nel, nb, s);
  }
  if (prec_double(prec)) {
    if (!L.R64) return cudaErrorInvalidValue;
    a.R = L.R64;
    return red_cols_dispatch<double, double, false>(L.n1, a, c->nel, nb, s);
  }
  if (!L.R32) return cudaErrorInvalidValue;
  a.R = L.R32;
  return red_cols_dispatch<float, float, true>(L.n1, a, c->nel, nb, s);
}

cudaError_t launch_reduced_theta(Context* c, const double* lam, const double* psi, double* dth, cudaStream_t s) {
  PLevel& L = c->plev[c->k];
  if (!L.R64) return cudaErrorInvalidValue;
  RedArgs a{};
  a.R = L.R64; a.v = lam;
  a.nx = c->mesh.nx; a.ny = c->mesh.ny;
  const unsigned g = (unsigned)((c->nel + kElemThreads - 1) / kElemThreads);
  switch (L.n1) {
    case 1: reduced_theta_kernel<1><<<g, kElemThreads, 0, s>>>(a, psi, dth); break;
    case 2: reduced_theta_kernel<2><<<g, kElemThreads, 0, s>>>(a, psi, dth); break;
    case 3: reduced_theta_kernel<3><<<g, kElemThreads, 0, s>>>(a, psi, dth); break;
    case 4: reduced_theta_kernel<4><<<g, kElemThreads, 0, s>>>(a, psi, dth); break;
    case 5: reduced_theta_kernel<5><<<g, kElemThreads, 0, s>>>(a, psi, dth); break;
    case 6: reduced_theta_kernel<6><<<g, kElemThreads, 0, s>>>(a, psi, dth); break;
    case 7: reduced_theta_kernel<7><<<g, kElemThreads, 0, s>>>(a, psi, dth); break;
    case 8: reduced_theta_kernel<8><<<g, kElemThreads, 0, s>>>(a, psi, dth); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int reduced_tile_rows() { return kTileRows; }

int reduced_entries(int n1) {
  const int h = n1 / 2, se = h + (n1 & 1), so = h;
  const int d[4] = {2 * se, so + se, se + so, 2 * so};
  int Q = 0;
  for (int b = 0; b < 4; ++b) Q += d[b] * (d[b] + 1) / 2;
  return Q;
}

cudaError_t launch_reduced_blocks(Context* c, int p, cudaStream_t s) {
  PLevel& L = c->plev[p];
  const long total = (long)c->nel * reduced_entries(L.n1);
  int blocks = (int)((total + 255) / 256);
  if (blocks > c->num_sms * 32) blocks = c->num_sms * 32;
  reduced_blocks_kernel<<<blocks, 256, 0, s>>>(c->nel, L.n1, L.Sdense, L.R64, L.R32, L.R2);
  return cudaGetLastError();
}

cudaError_t launch_sym_pack(Context* c, int p, const double* Md, cudaStream_t s) {
  PLevel& L = c->plev[p];
  if (!L.Mp32) return cudaErrorInvalidValue;
  const long total = (long)c->nel * L.m * (L.m + 1) / 2;
  int blocks = (int)((total + 255) / 256);
  if (blocks > c->num_sms * 32) blocks = c->num_sms * 32;
  sym_pack_kernel<<<blocks, 256, 0, s>>>(c->nel, L.m, Md, L.Mp32);
  return cudaGetLastError();
}
cudaError_t launch_sym_schwarz(Context* c, int p, const void* v, const void* cvec, void* y, double alpha,
                               double beta, cudaStream_t s) {
  PLevel& L = c->plev[p];
  if (!L.Mp32 || !c->red_z) return cudaErrorInvalidValue;
  RedArgs a{};
  a.R = L.Mp32; a.v = v; a.cvec = cvec; a.y = y; a.z = c->red_z;
  a.alpha = alpha; a.beta = beta;
  a.nx = c->mesh.nx; a.ny = c->mesh.ny;
  switch (L.n1) {
    case 1: return sym_launch<1>(a, c->nel, s);
    case 2: return sym_launch<2>(a, c->nel, s);
    case 3: return sym_launch<3>(a, c->nel, s);
    case 4: return sym_launch<4>(a, c->nel, s);
    case 5: return sym_launch<5>(a, c->nel, s);
    case 6: return sym_launch<6>(a, c->nel, s);
    case 7: return sym_launch<7>(a, c->nel, s);
    case 8: return sym_launch<8>(a, c->nel, s);
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t launch_reduced_apply(Context* c, int p, int prec, const void* v, const void* cvec, void* y,
                                 double alpha, double beta, cudaStream_t s) {
  PLevel& L = c->plev[p];
  RedArgs a{};
  a.v = v; a.cvec = cvec; a.y = y; a.z = c->red_z;
  a.alpha = alpha; a.beta = beta;
  a.nx = c->mesh.nx; a.ny = c->mesh.ny;
  const long nel = c->nel;
  if (prec == HDG_PREC_F32X2 && L.R2) {   // double-float product on the FP32 pipe
    a.R = L.R2;
    return red_dispatch<float2, dd, false>(L.n1, a, nel, c->opt.reduced, s);
  }
  if (prec_double(prec)) {   // FP64 (and F32X2 without the float2 blocks): FP64 blocks
    if (!L.R64) return cudaErrorInvalidValue;
    a.R = L.R64;
    return red_dispatch<double, double, false>(L.n1, a, nel, c->opt.reduced, s);
  }
  // FP32 / BF16 cycles (float vectors): FP32 blocks applied to v - mean
  if (!L.R32) return cudaErrorInvalidValue;
  a.R = L.R32;
  return red_dispatch<float, float, true>(L.n1, a, nel, c->opt.reduced, s);
}

}  // namespace hdg
