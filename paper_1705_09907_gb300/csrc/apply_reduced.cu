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
// ignored, boundary rows of y zero) runs in two launches:
//   1. one thread per element: gather the element's four faces of v, form
//      z_K = S_K v_K by the reduced product and store z (face-major [4n][nel]);
//   2. one thread per element: each owned face (W and S) adds its two element
//      contributions, own first, and writes y once (E / N domain-boundary
//      edges are zeroed by their only element).
// Both orders of summation are fixed, so results are deterministic.
#include "hdg_internal.h"

namespace hdg {

namespace {

template <int N1>
struct Red {
  static constexpr int n = N1, h = N1 / 2, se = N1 / 2 + (N1 & 1), so = N1 / 2;
  static constexpr int d0 = 2 * se, d1 = so + se, d2 = se + so, d3 = 2 * so;
  static constexpr int q0 = 0, q1 = d0 * (d0 + 1) / 2, q2 = q1 + d1 * (d1 + 1) / 2, q3 = q2 + d2 * (d2 + 1) / 2;
  static constexpr int Q = q3 + d3 * (d3 + 1) / 2;
};

// u = B t for one symmetric block of dimension D stored as a packed upper
// triangle (row-major) at R[(qoff + idx) * nel + K]
template <int D, typename T, typename TS>
__device__ __forceinline__ void sym_block(const TS* __restrict__ R, int qoff, long nel, long K, const T (&t)[D > 0 ? D : 1],
                                          T (&u)[D > 0 ? D : 1]) {
#pragma unroll
  for (int i = 0; i < D; ++i) u[i] = T(0);
  int q = qoff;
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int j = i; j < D; ++j, ++q) {
      const T b = (T)__ldcs(R + (size_t)q * nel + K);
      if (j == i) {
        u[i] = fma(b, t[i], u[i]);
      } else {
        u[i] = fma(b, t[j], u[i]);
        u[j] = fma(b, t[i], u[j]);
      }
    }
  }
}

// even / odd node parts of a face vector (see the file comment)
template <int N1, typename T>
__device__ __forceinline__ void split_nodes(const T (&v)[N1], T* ev, T* od) {
  constexpr int h = N1 / 2;
#pragma unroll
  for (int i = 0; i < h; ++i) {
    ev[i] = v[i] + v[N1 - 1 - i];
    od[i] = v[i] - v[N1 - 1 - i];
  }
  if (N1 & 1) ev[h] = v[h];
}

// transpose of split_nodes
template <int N1, typename T>
__device__ __forceinline__ void join_nodes(const T* ev, const T* od, T (&v)[N1]) {
  constexpr int h = N1 / 2;
#pragma unroll
  for (int i = 0; i < h; ++i) {
    v[i] = ev[i] + od[i];
    v[N1 - 1 - i] = ev[i] - od[i];
  }
  if (N1 & 1) v[h] = ev[h];
}

struct RedArgs {
  const void* R;       // reduced blocks [Q][nel] (type TS)
  const void* v;       // input vector (type T)
  const void* cvec;    // addend or nullptr
  void* y;             // output
  void* z;             // element products [4 n1][nel] (type T)
  double alpha, beta;
  int nx, ny;
};

template <int N1, typename TS, typename T, bool DIFF>
__global__ void __launch_bounds__(128) reduced_elem_kernel(const RedArgs a) {
  using RD = Red<N1>;
  constexpr int se = RD::se, so = RD::so;
  const int nx = a.nx, ny = a.ny;
  const long nel = (long)nx * ny;
  const long K = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (K >= nel) return;
  const int i = (int)(K % nx), j = (int)(K / nx);
  const T* __restrict__ v = (const T*)a.v;
  const long eW = i + (long)(nx + 1) * j, eS = (long)(nx + 1) * ny + i + (long)nx * j;
  const bool hW = i > 0, hE = i < nx - 1, hS = j > 0, hN = j < ny - 1;
  T xw[N1], xe[N1], xs[N1], xn[N1];
#pragma unroll
  for (int q = 0; q < N1; ++q) {
    xw[q] = hW ? v[eW * N1 + q] : T(0);
    xe[q] = hE ? v[(eW + 1) * N1 + q] : T(0);
    xs[q] = hS ? v[eS * N1 + q] : T(0);
    xn[q] = hN ? v[(eS + nx) * N1 + q] : T(0);
  }
  if (DIFF) {   // S_K has zero row sums: apply it to v_K - mean(v_K)
    T sum = T(0);
#pragma unroll
    for (int q = 0; q < N1; ++q) sum += (xw[q] + xe[q]) + (xs[q] + xn[q]);
    const T mu = sum * (T(1) / T(4 * N1));
#pragma unroll
    for (int q = 0; q < N1; ++q) { xw[q] -= mu; xe[q] -= mu; xs[q] -= mu; xn[q] -= mu; }
  }
  T P[N1], M[N1], Pp[N1], Mp[N1];
#pragma unroll
  for (int q = 0; q < N1; ++q) {
    P[q] = xw[q] + xe[q]; M[q] = xw[q] - xe[q];
    Pp[q] = xs[q] + xn[q]; Mp[q] = xs[q] - xn[q];
  }
  // t-coordinates of the four blocks
  T t0[RD::d0 > 0 ? RD::d0 : 1], t1[RD::d1 > 0 ? RD::d1 : 1], t2[RD::d2 > 0 ? RD::d2 : 1],
      t3[RD::d3 > 0 ? RD::d3 : 1];
  {
    T ev[se > 0 ? se : 1], od[so > 0 ? so : 1];
    split_nodes<N1>(P, ev, od);
#pragma unroll
    for (int q = 0; q < se; ++q) t0[q] = ev[q];
#pragma unroll
    for (int q = 0; q < so; ++q) t1[q] = od[q];
    split_nodes<N1>(Pp, ev, od);
#pragma unroll
    for (int q = 0; q < se; ++q) t0[se + q] = ev[q];
#pragma unroll
    for (int q = 0; q < so; ++q) t2[se + q] = od[q];
    split_nodes<N1>(M, ev, od);
#pragma unroll
    for (int q = 0; q < se; ++q) t2[q] = ev[q];
#pragma unroll
    for (int q = 0; q < so; ++q) t3[q] = od[q];
    split_nodes<N1>(Mp, ev, od);
#pragma unroll
    for (int q = 0; q < se; ++q) t1[so + q] = ev[q];
#pragma unroll
    for (int q = 0; q < so; ++q) t3[so + q] = od[q];
  }
  const TS* __restrict__ R = (const TS*)a.R;
  T u0[RD::d0 > 0 ? RD::d0 : 1], u1[RD::d1 > 0 ? RD::d1 : 1], u2[RD::d2 > 0 ? RD::d2 : 1],
      u3[RD::d3 > 0 ? RD::d3 : 1];
  sym_block<RD::d0, T>(R, RD::q0, nel, K, t0, u0);
  sym_block<RD::d1, T>(R, RD::q1, nel, K, t1, u1);
  sym_block<RD::d2, T>(R, RD::q2, nel, K, t2, u2);
  sym_block<RD::d3, T>(R, RD::q3, nel, K, t3, u3);
  // back to face dofs: z = F^T u
  T Po[N1], Mo[N1], Ppo[N1], Mpo[N1];
  {
    T ev[se > 0 ? se : 1], od[so > 0 ? so : 1];
#pragma unroll
    for (int q = 0; q < se; ++q) ev[q] = u0[q];
#pragma unroll
    for (int q = 0; q < so; ++q) od[q] = u1[q];
    join_nodes<N1>(ev, od, Po);
#pragma unroll
    for (int q = 0; q < se; ++q) ev[q] = u2[q];
#pragma unroll
    for (int q = 0; q < so; ++q) od[q] = u3[q];
    join_nodes<N1>(ev, od, Mo);
#pragma unroll
    for (int q = 0; q < se; ++q) ev[q] = u0[se + q];
#pragma unroll
    for (int q = 0; q < so; ++q) od[q] = u2[se + q];
    join_nodes<N1>(ev, od, Ppo);
#pragma unroll
    for (int q = 0; q < se; ++q) ev[q] = u1[so + q];
#pragma unroll
    for (int q = 0; q < so; ++q) od[q] = u3[so + q];
    join_nodes<N1>(ev, od, Mpo);
  }
  T* __restrict__ z = (T*)a.z;
#pragma unroll
  for (int q = 0; q < N1; ++q) {
    z[(size_t)(0 * N1 + q) * nel + K] = Po[q] + Mo[q];     // W
    z[(size_t)(1 * N1 + q) * nel + K] = Po[q] - Mo[q];     // E
    z[(size_t)(2 * N1 + q) * nel + K] = Ppo[q] + Mpo[q];   // S
    z[(size_t)(3 * N1 + q) * nel + K] = Ppo[q] - Mpo[q];   // N
  }
}

template <int N1, typename T>
__global__ void __launch_bounds__(256) reduced_face_kernel(const RedArgs a) {
  const int nx = a.nx, ny = a.ny;
  const long nel = (long)nx * ny;
  const long K = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (K >= nel) return;
  const int i = (int)(K % nx), j = (int)(K / nx);
  const T* __restrict__ z = (const T*)a.z;
  const T* __restrict__ cv = (const T*)a.cvec;
  T* __restrict__ y = (T*)a.y;
  const T al = (T)a.alpha, be = (T)a.beta;
  // y = A v, y = c - A v and y = c + A v take no multiply
  const int form = (al == T(1) && (!cv || be == T(0))) ? 0
                   : (cv && be == T(1) && al == T(-1)) ? 1 : (cv && be == T(1) && al == T(1)) ? 2 : 3;
  const long eW = i + (long)(nx + 1) * j, eS = (long)(nx + 1) * ny + i + (long)nx * j;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const bool bnd = side == 0 ? (i == 0) : (j == 0);
    const long e = side == 0 ? eW : eS;
    const int fo = side == 0 ? 0 : 2;                    // own face W / S
    const long Kn = side == 0 ? K - 1 : K - nx;           // neighbour across it
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      const size_t o = (size_t)e * N1 + q;
      T val = T(0);
      if (!bnd) {
        const T s = z[(size_t)(fo * N1 + q) * nel + K] + z[(size_t)((fo + 1) * N1 + q) * nel + Kn];
        if (form == 0) val = s;
        else if (form == 1) val = cv[o] - s;
        else if (form == 2) val = cv[o] + s;
        else {
          val = al * s;
          if (cv) val = fma(be, cv[o], val);
        }
      }
      y[o] = val;
    }
  }
  if (i == nx - 1) {
#pragma unroll
    for (int q = 0; q < N1; ++q) y[(eW + 1) * N1 + q] = T(0);
  }
  if (j == ny - 1) {
#pragma unroll
    for (int q = 0; q < N1; ++q) y[(eS + nx) * N1 + q] = T(0);
  }
}

template <int N1, typename TS, typename T, bool DIFF>
cudaError_t red_launch(const RedArgs& a, long nel, cudaStream_t s) {
  const unsigned g1 = (unsigned)((nel + 127) / 128), g2 = (unsigned)((nel + 255) / 256);
  reduced_elem_kernel<N1, TS, T, DIFF><<<g1, 128, 0, s>>>(a);
  HDG_CUDA_TRY(cudaGetLastError());
  reduced_face_kernel<N1, T><<<g2, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename TS, typename T, bool DIFF>
cudaError_t red_dispatch(int n1, const RedArgs& a, long nel, cudaStream_t s) {
  switch (n1) {
    case 1: return red_launch<1, TS, T, DIFF>(a, nel, s);
    case 2: return red_launch<2, TS, T, DIFF>(a, nel, s);
    case 3: return red_launch<3, TS, T, DIFF>(a, nel, s);
    case 4: return red_launch<4, TS, T, DIFF>(a, nel, s);
    case 5: return red_launch<5, TS, T, DIFF>(a, nel, s);
    case 6: return red_launch<6, TS, T, DIFF>(a, nel, s);
    case 7: return red_launch<7, TS, T, DIFF>(a, nel, s);
    case 8: return red_launch<8, TS, T, DIFF>(a, nel, s);
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
                                      float* __restrict__ R32) {
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
    R64[t] = val;
    if (R32) R32[t] = (float)val;
  }
}

}  // namespace

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
  reduced_blocks_kernel<<<blocks, 256, 0, s>>>(c->nel, L.n1, L.Sdense, L.R64, L.R32);
  return cudaGetLastError();
}

cudaError_t launch_reduced_apply(Context* c, int p, int prec, const void* v, const void* cvec, void* y,
                                 double alpha, double beta, cudaStream_t s) {
  PLevel& L = c->plev[p];
  RedArgs a{};
  a.v = v; a.cvec = cvec; a.y = y; a.z = c->red_z;
  a.alpha = alpha; a.beta = beta;
  a.nx = c->mesh.nx; a.ny = c->mesh.ny;
  const long nel = c->nel;
  if (prec_double(prec)) {   // FP64 (and the double-vector F32X2 cycles): FP64 blocks
    if (!L.R64) return cudaErrorInvalidValue;
    a.R = L.R64;
    return red_dispatch<double, double, false>(L.n1, a, nel, s);
  }
  // FP32 / BF16 cycles (float vectors): FP32 blocks applied to v - mean
  if (!L.R32) return cudaErrorInvalidValue;
  a.R = L.R32;
  return red_dispatch<float, float, true>(L.n1, a, nel, s);
}

}  // namespace hdg
