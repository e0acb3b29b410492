// Nested p/h multigrid (Sec. 6, Algs. 1 and 2) and multigrid-preconditioned CG.
//
// p-levels k..1 : element-block operators (records), weighted additive Schwarz
//                 smoothing, per-edge transfers P (Eq. eq_mg_pro), R = P^T.
// p = 0         : top of the h-hierarchy; Jacobi-preconditioned Chebyshev.
// Q1 levels     : interior vertices of nested N, N/2, ... meshes; 9-point
//                 stencils (conforming Q1 stiffness on the finest mesh, Galerkin
//                 triple products below), Chebyshev smoothing, bilinear P and
//                 R = P^T; P_J / P_J^T (edge means, Eq. eq_h_mg_pro) between the
//                 finest Q1 level and p = 0; FP64 Cholesky on the coarsest mesh.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "hdg_internal.h"

namespace hdg {

constexpr int kRedBlocks = 304;   // fixed reduction grid (deterministic sums)
constexpr int kCgScalars = 12;    // per-column scalars of the batched CG
constexpr int kColRedBlocks = 608; // fixed grid of the per-column dot products

// ---------------------------------------------------------------------------
// Deterministic dot products: fixed grid of partial sums, then one block sums
// the partials in a fixed order.
template <typename T>
__global__ void dots_kernel(size_t n, const T* __restrict__ a0, const T* __restrict__ b0,
                            const T* __restrict__ a1, const T* __restrict__ b1, const T* __restrict__ a2,
                            const T* __restrict__ b2, double* __restrict__ part) {
  __shared__ double sh[3][256];
  // four independent partial sums per thread (loads of four strides in flight),
  // combined in a fixed order
  double p0[4] = {0.0, 0.0, 0.0, 0.0}, p1[4] = {0.0, 0.0, 0.0, 0.0}, p2[4] = {0.0, 0.0, 0.0, 0.0};
  const size_t step = (size_t)gridDim.x * blockDim.x;
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (; t + 3 * step < n; t += 4 * step) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const size_t o = t + u * step;
      p0[u] += (double)a0[o] * (double)b0[o];
      if (a1) p1[u] += (double)a1[o] * (double)b1[o];
      if (a2) p2[u] += (double)a2[o] * (double)b2[o];
    }
  }
  for (; t < n; t += step) {
    p0[0] += (double)a0[t] * (double)b0[t];
    if (a1) p1[0] += (double)a1[t] * (double)b1[t];
    if (a2) p2[0] += (double)a2[t] * (double)b2[t];
  }
  const double s0 = (p0[0] + p0[1]) + (p0[2] + p0[3]);
  const double s1 = (p1[0] + p1[1]) + (p1[2] + p1[3]);
  const double s2 = (p2[0] + p2[1]) + (p2[2] + p2[3]);
  sh[0][threadIdx.x] = s0; sh[1][threadIdx.x] = s1; sh[2][threadIdx.x] = s2;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) part[q * kRedBlocks + blockIdx.x] = sh[q][0];
}

__global__ void dots_finalize_kernel(const double* __restrict__ part, int nd, double* __restrict__ out) {
  __shared__ double sh[3][512];
  for (int q = 0; q < 3; ++q) {
    double v = 0.0;
    for (int t = threadIdx.x; t < kRedBlocks; t += 512) v += part[q * kRedBlocks + t];
    sh[q][threadIdx.x] = v;
  }
  __syncthreads();
  for (int w = 256; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < nd; ++q) out[q] = sh[q][0];
}

template <typename T>
static cudaError_t dots(Context* c, size_t n, const T* a0, const T* b0, const T* a1, const T* b1, const T* a2,
                        const T* b2, double* out, cudaStream_t s) {
  dots_kernel<T><<<kRedBlocks, 256, 0, s>>>(n, a0, b0, a1, b1, a2, b2, c->red);
  HDG_CUDA_TRY(cudaGetLastError());
  const int nd = a2 ? 3 : (a1 ? 2 : 1);
  dots_finalize_kernel<<<1, 512, 0, s>>>(c->red, nd, out);
  return cudaGetLastError();
}

cudaError_t vec_dot(Context* c, const double* a, const double* b, int n, double* out_dev, cudaStream_t s) {
  return dots<double>(c, (size_t)n, a, b, nullptr, nullptr, nullptr, nullptr, out_dev, s);
}

// ---------------------------------------------------------------------------
// Elementwise helpers
template <typename T>
__global__ void scale_kernel(size_t n, T* __restrict__ x, const double* __restrict__ sc, double mult) {
  const double f = mult / sc[0];
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    x[t] = (T)((double)x[t] * f);
}

template <typename T>
__global__ void mul_kernel(size_t n, const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ y) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    y[t] = a[t] * b[t];
}

template <typename TI, typename TO>
__global__ void copy_convert_kernel(size_t n, const TI* __restrict__ a, TO* __restrict__ b) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    b[t] = (TO)a[t];
}

// t -> (t / d, t % d) with 32-bit division when t fits (64-bit division by a
// runtime value costs far more than the memory traffic of these kernels)
__device__ __forceinline__ size_t divmod(size_t t, int d, int* rem) {
  if (d == 1) { *rem = 0; return t; }
  if (t <= 0xffffffffull) {
    const unsigned tt = (unsigned)t, q = tt / (unsigned)d;
    *rem = (int)(tt - q * (unsigned)d);
    return q;
  }
  *rem = (int)(t % (size_t)d);
  return t / (size_t)d;
}

static int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  if (b > 2048) b = 2048;
  if (b < 1) b = 1;
  return (int)b;
}

// Chebyshev steps: first step from x = 0 (x = d = c0 * dinv .* f), first step
// with x given (d = c0 * dinv .* t; x += d), later steps (d = a1 d + a2 dinv .* t;
// x += d). Vectors hold nb right-hand sides per unknown (right-hand side
// fastest); n counts unknowns x columns.
// The per-entry bodies are device functions shared by the one-launch-per-step
// kernels and the fused coarse-level kernel; their vector arguments carry no
// __restrict__ (the fused kernel reads in one phase what it wrote in the last).
template <typename T>
__device__ __forceinline__ void cheb_first_zero_at(size_t t, int nb, const T* dinv, const T* f, T* x, T* d, T c0) {
  int col;
  const T v = c0 * dinv[divmod(t, nb, &col)] * f[t];
  x[t] = v;
  d[t] = v;
}
template <typename T>
__device__ __forceinline__ void cheb_step_at(size_t t, int nb, const T* dinv, const T* r, T* x, T* d, T a1, T a2) {
  int col;
  const T v = a1 * d[t] + a2 * dinv[divmod(t, nb, &col)] * r[t];
  d[t] = v;
  x[t] += v;
}
template <typename T>
__global__ void cheb_first_zero_kernel(size_t n, int nb, const T* __restrict__ dinv, const T* __restrict__ f,
                                       T* __restrict__ x, T* __restrict__ d, T c0) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    cheb_first_zero_at<T>(t, nb, dinv, f, x, d, c0);
}
template <typename T>
__global__ void cheb_step_kernel(size_t n, int nb, const T* __restrict__ dinv, const T* __restrict__ r,
                                 T* __restrict__ x, T* __restrict__ d, T a1, T a2) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    cheb_step_at<T>(t, nb, dinv, r, x, d, a1, a2);
}

// ---------------------------------------------------------------------------
// p-transfers per edge. P is [(pc+2) x (pc+1)] row-major: fine node a', coarse a.
// One thread per (edge, column) loads the edge's NF fine (or NC coarse) values
// once and writes all its outputs; NC = pc + 1 is a template constant so the
// loads issue back to back.
template <typename T, int NC>
__global__ void restrict_p_kernel(int n_edges, int nb, const T* __restrict__ P, const T* __restrict__ rf,
                                  T* __restrict__ rc) {
  constexpr int NF = NC + 1;
  const size_t total = (size_t)n_edges * nb;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    int col;
    const size_t e = divmod(t, nb, &col);
    T v[NF];
#pragma unroll
    for (int b = 0; b < NF; ++b) v[b] = rf[(e * NF + b) * nb + col];
#pragma unroll
    for (int a = 0; a < NC; ++a) {
      T s = 0;
#pragma unroll
      for (int b = 0; b < NF; ++b) s += __ldg(&P[b * NC + a]) * v[b];
      rc[(e * NC + a) * nb + col] = s;
    }
  }
}
template <typename T, int NC>
__global__ void prolong_p_add_kernel(int n_edges, int nb, const T* __restrict__ P, const T* __restrict__ xc,
                                     T* __restrict__ xf) {
  constexpr int NF = NC + 1;
  const size_t total = (size_t)n_edges * nb;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    int col;
    const size_t e = divmod(t, nb, &col);
    T v[NC], o[NF];
#pragma unroll
    for (int b = 0; b < NC; ++b) v[b] = xc[(e * NC + b) * nb + col];
#pragma unroll
    for (int a = 0; a < NF; ++a) o[a] = xf[(e * NF + a) * nb + col];
#pragma unroll
    for (int a = 0; a < NF; ++a) {
      T s = 0;
#pragma unroll
      for (int b = 0; b < NC; ++b) s += __ldg(&P[a * NC + b]) * v[b];
      xf[(e * NF + a) * nb + col] = o[a] + s;
    }
  }
}
template <typename T>
static cudaError_t p_transfer(bool restrict_, int n1c, int n_edges, int nb, const T* P, const T* in, T* out,
                              cudaStream_t s) {
  const int g = grid_for((size_t)n_edges * nb);
#define HDG_PT(NCv)                                                                              \
  case NCv:                                                                                      \
    if (restrict_) restrict_p_kernel<T, NCv><<<g, 256, 0, s>>>(n_edges, nb, P, in, out);         \
    else prolong_p_add_kernel<T, NCv><<<g, 256, 0, s>>>(n_edges, nb, P, in, out);                \
    break;
  switch (n1c) {
    HDG_PT(1) HDG_PT(2) HDG_PT(3) HDG_PT(4) HDG_PT(5) HDG_PT(6) HDG_PT(7)
    default: return cudaErrorInvalidValue;
  }
#undef HDG_PT
  return cudaGetLastError();
}

// P_J^T: interior vertex (I, J) gets half the sum of its 4 edges' residuals.
template <typename T>
__global__ void restrict_J_kernel(int nx, int ny, int nb, const T* __restrict__ r0, T* __restrict__ rq) {
  const int nvx = nx - 1;
  const size_t nv = (size_t)(nx + 1) * ny, total = (size_t)(nx - 1) * (ny - 1) * nb;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    int col;
    const int u = (int)divmod(t, nb, &col);
    const size_t I = u % nvx + 1, J = u / nvx + 1;
    const T s = r0[(I + (nx + 1) * (J - 1)) * nb + col] + r0[(I + (nx + 1) * J) * nb + col] +
                r0[(nv + (I - 1) + nx * J) * nb + col] + r0[(nv + I + nx * J) * nb + col];
    rq[t] = T(0.5) * s;
  }
}
// P_J: every edge gets the mean of its two end vertices (boundary vertices 0);
// boundary edges stay 0.
template <typename T>
__global__ void prolong_J_add_kernel(int nx, int ny, int nb, const T* __restrict__ xq, T* __restrict__ x0) {
  const int nvx = nx - 1;
  const int nv = (nx + 1) * ny, ne = nv + nx * (ny + 1);
  const size_t total = (size_t)ne * nb;
  for (size_t tt = blockIdx.x * (size_t)blockDim.x + threadIdx.x; tt < total; tt += (size_t)gridDim.x * blockDim.x) {
    int col;
    const int t = (int)divmod(tt, nb, &col);
    int I0, J0, I1, J1;
    bool interior;
    if (t < nv) {
      const int i = t % (nx + 1), j = t / (nx + 1);
      I0 = i; J0 = j; I1 = i; J1 = j + 1;
      interior = (i > 0 && i < nx);
    } else {
      const int u = t - nv, i = u % nx, j = u / nx;
      I0 = i; J0 = j; I1 = i + 1; J1 = j;
      interior = (j > 0 && j < ny);
    }
    if (!interior) continue;
    T s = 0;
    if (I0 > 0 && I0 < nx && J0 > 0 && J0 < ny) s += xq[((size_t)(I0 - 1) + nvx * (J0 - 1)) * nb + col];
    if (I1 > 0 && I1 < nx && J1 > 0 && J1 < ny) s += xq[((size_t)(I1 - 1) + nvx * (J1 - 1)) * nb + col];
    x0[tt] += T(0.5) * s;
  }
}

// ---------------------------------------------------------------------------
// Q1 stencil levels. Stencil [9][nv], offset o = (dy+1)*3 + (dx+1).
// y = beta c + alpha A x. With `rsum` (row sums of A, low-precision levels)
// the product is taken in difference form, sum_{o != centre} a_o (x_{v+o} - x_v)
// + rsum_v x_v: exact in exact arithmetic, and the rounded stencil then sees the
// variation of x around v rather than its (smooth, large) value.
// (A x)_v for vertex t, column col of a Q1 stencil level (difference form with
// row sums when rsum is given)
template <typename T>
__device__ __forceinline__ T stencil_row(int nvx, int nvy, int nb, int t, int col, const T* st, const T* x,
                                         const T* rsum) {
  const int nvert = nvx * nvy;
  const int I = t % nvx, J = t / nvx;
  const T xc = x[(size_t)t * nb + col];
  T s = rsum ? rsum[t] * xc : T(0);
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int I2 = I + dx, J2 = J + dy;
      if (I2 < 0 || J2 < 0 || I2 >= nvx || J2 >= nvy) continue;
      const T a = st[((dy + 1) * 3 + dx + 1) * (size_t)nvert + t];
      const T xn = x[((size_t)I2 + (size_t)nvx * J2) * nb + col];
      if (rsum) {
        if (dx != 0 || dy != 0) s += a * (xn - xc);
      } else {
        s += a * xn;
      }
    }
  return s;
}

template <typename T>
__device__ __forceinline__ void stencil_apply_at(size_t tt, int nx, int ny, int nb, const T* st, const T* x,
                                                 const T* c, T* y, T alpha, T beta, const T* rsum) {
  int col;
  const int t = (int)divmod(tt, nb, &col);
  T v = alpha * stencil_row<T>(nx - 1, ny - 1, nb, t, col, st, x, rsum);
  if (c) v += beta * c[tt];
  y[tt] = v;
}
template <typename T>
__global__ void stencil_apply_kernel(int nx, int ny, int nb, const T* __restrict__ st, const T* __restrict__ x,
                                     const T* __restrict__ c, T* __restrict__ y, T alpha, T beta,
                                     const T* __restrict__ rsum) {
  const size_t total = (size_t)(nx - 1) * (ny - 1) * nb;
  for (size_t tt = blockIdx.x * (size_t)blockDim.x + threadIdx.x; tt < total; tt += (size_t)gridDim.x * blockDim.x)
    stencil_apply_at<T>(tt, nx, ny, nb, st, x, c, y, alpha, beta, rsum);
}

// Fused Chebyshev steps on a Q1 level (stencil A, Jacobi D), two launches per
// degree-2 step instead of four:
//   cheb_resid: r = f - A x, d = c0 D^-1 r             (x is not touched)
//   cheb_next:  r' = rin - A d, d' = a1 d + a2 D^-1 r',
//               x += d' (+ d when x does not hold d yet); d' goes to a second
//               buffer, so no thread writes what its neighbours read
template <typename T>
__device__ __forceinline__ void cheb_resid_at(size_t tt, int nx, int ny, int nb, const T* st, const T* rsum,
                                              const T* dinv, const T* f, const T* x, T* r, T* d, T c0) {
  int col;
  const int t = (int)divmod(tt, nb, &col);
  const T rv = f[tt] - stencil_row<T>(nx - 1, ny - 1, nb, t, col, st, x, rsum);
  r[tt] = rv;
  d[tt] = c0 * dinv[t] * rv;
}
template <typename T>
__device__ __forceinline__ void cheb_next_at(size_t tt, int nx, int ny, int nb, const T* st, const T* rsum,
                                             const T* dinv, const T* rin, T* rout, const T* d, T* dn, T* x, T a1,
                                             T a2, int add_d) {
  int col;
  const int t = (int)divmod(tt, nb, &col);
  const T rv = rin[tt] - stencil_row<T>(nx - 1, ny - 1, nb, t, col, st, d, rsum);
  const T dv = d[tt];
  const T dnv = a1 * dv + a2 * dinv[t] * rv;
  rout[tt] = rv;
  dn[tt] = dnv;
  x[tt] += add_d ? dv + dnv : dnv;
}
template <typename T>
__global__ void cheb_resid_kernel(int nx, int ny, int nb, const T* __restrict__ st, const T* __restrict__ rsum,
                                  const T* __restrict__ dinv, const T* __restrict__ f, const T* __restrict__ x,
                                  T* __restrict__ r, T* __restrict__ d, T c0) {
  const size_t total = (size_t)(nx - 1) * (ny - 1) * nb;
  for (size_t tt = blockIdx.x * (size_t)blockDim.x + threadIdx.x; tt < total; tt += (size_t)gridDim.x * blockDim.x)
    cheb_resid_at<T>(tt, nx, ny, nb, st, rsum, dinv, f, x, r, d, c0);
}
template <typename T>
__global__ void cheb_next_kernel(int nx, int ny, int nb, const T* __restrict__ st, const T* __restrict__ rsum,
                                 const T* __restrict__ dinv, const T* rin, T* rout, const T* __restrict__ d,
                                 T* __restrict__ dn, T* __restrict__ x, T a1, T a2, int add_d) {
  const size_t total = (size_t)(nx - 1) * (ny - 1) * nb;
  for (size_t tt = blockIdx.x * (size_t)blockDim.x + threadIdx.x; tt < total; tt += (size_t)gridDim.x * blockDim.x)
    cheb_next_at<T>(tt, nx, ny, nb, st, rsum, dinv, rin, rout, d, dn, x, a1, a2, add_d);
}

// row sums of a stencil level (FP64), stored in float for the difference form
__global__ void stencil_rowsum_kernel(int nvert, const double* __restrict__ st, float* __restrict__ rs) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nvert; t += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int o = 0; o < 9; ++o) s += st[o * (size_t)nvert + t];
    rs[t] = (float)s;
  }
}

// full weighting R = P^T of bilinear interpolation
template <typename T>
__device__ __forceinline__ void restrict_q_at(size_t tt, int nxc, int nyc, int nb, const T* rf, T* rc) {
  const int nxf = 2 * nxc, nyf = 2 * nyc;
  const int nvxc = nxc - 1, nvxf = nxf - 1;
  int col;
  const int t = (int)divmod(tt, nb, &col);
  const int I = t % nvxc + 1, J = t / nvxc + 1;
  T s = 0;
  for (int b = -1; b <= 1; ++b)
    for (int a = -1; a <= 1; ++a) {
      const int i = 2 * I + a, j = 2 * J + b;
      if (i <= 0 || j <= 0 || i >= nxf || j >= nyf) continue;
      const T w = (a == 0 ? T(1) : T(0.5)) * (b == 0 ? T(1) : T(0.5));
      s += w * rf[((size_t)(i - 1) + (size_t)nvxf * (j - 1)) * nb + col];
    }
  rc[tt] = s;
}
template <typename T>
__global__ void restrict_q_kernel(int nxc, int nyc, int nb, const T* __restrict__ rf, T* __restrict__ rc) {
  const size_t total = (size_t)(nxc - 1) * (nyc - 1) * nb;
  for (size_t tt = blockIdx.x * (size_t)blockDim.x + threadIdx.x; tt < total; tt += (size_t)gridDim.x * blockDim.x)
    restrict_q_at<T>(tt, nxc, nyc, nb, rf, rc);
}

template <typename T>
__device__ __forceinline__ void prolong_q_add_at(size_t tt, int nxc, int nyc, int nb, const T* xc, T* xf) {
  const int nxf = 2 * nxc;
  const int nvxf = nxf - 1, nvxc = nxc - 1;
  int col;
  const int t = (int)divmod(tt, nb, &col);
  const int i = t % nvxf + 1, j = t / nvxf + 1;
  const int i0 = i / 2, j0 = j / 2;
  const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1;
  const T wx = (i & 1) ? T(0.5) : T(1), wy = (j & 1) ? T(0.5) : T(1);
  T s = 0;
  for (int b = 0; b < nj; ++b)
    for (int a = 0; a < ni; ++a) {
      const int I = i0 + a, J = j0 + b;
      if (I <= 0 || J <= 0 || I >= nxc || J >= nyc) continue;
      s += wx * wy * xc[((size_t)(I - 1) + (size_t)nvxc * (J - 1)) * nb + col];
    }
  xf[tt] += s;
}
template <typename T>
__global__ void prolong_q_add_kernel(int nxc, int nyc, int nb, const T* __restrict__ xc, T* __restrict__ xf) {
  const size_t total = (size_t)(2 * nxc - 1) * (2 * nyc - 1) * nb;
  for (size_t tt = blockIdx.x * (size_t)blockDim.x + threadIdx.x; tt < total; tt += (size_t)gridDim.x * blockDim.x)
    prolong_q_add_at<T>(tt, nxc, nyc, nb, xc, xf);
}

// conforming Q1 stiffness (kappa grad u, grad v) on the finest mesh:
// element matrix kappa * ((hy/hx) Kx + (hx/hy) Ky) with the bilinear patterns
// Kx = 1/6 [[2,-2,1,-1],[-2,2,-1,1],[1,-1,2,-2],[-1,1,-2,2]] (vertex order
// (0,0), (1,0), (0,1), (1,1)) and Ky its x/y transpose.
__global__ void q1_stencil_kernel(int nx, int ny, double hx, double hy, const double* __restrict__ kappa,
                                  double* __restrict__ st) {
  const int nvx = nx - 1, nvert = (nx - 1) * (ny - 1);
  const double ax = hy / hx / 6.0, ay = hx / hy / 6.0;
  const double Kx[4][4] = {{2, -2, 1, -1}, {-2, 2, -1, 1}, {1, -1, 2, -2}, {-1, 1, -2, 2}};
  const double Ky[4][4] = {{2, 1, -2, -1}, {1, 2, -1, -2}, {-2, -1, 2, 1}, {-1, -2, 1, 2}};
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nvert; t += gridDim.x * blockDim.x) {
    const int I = t % nvx + 1, J = t / nvx + 1;
    double acc[9];
    for (int o = 0; o < 9; ++o) acc[o] = 0.0;
    for (int ej = J - 1; ej <= J; ++ej)
      for (int ei = I - 1; ei <= I; ++ei) {
        const double kap = kappa[ei + nx * ej];
        const int la = (I - ei) + 2 * (J - ej);          // local index of (I, J)
        for (int lb = 0; lb < 4; ++lb) {
          const int I2 = ei + (lb & 1), J2 = ej + (lb >> 1);
          if (I2 <= 0 || J2 <= 0 || I2 >= nx || J2 >= ny) continue;
          const int o = (J2 - J + 1) * 3 + (I2 - I + 1);
          acc[o] += kap * (ax * Kx[la][lb] + ay * Ky[la][lb]);
        }
      }
    for (int o = 0; o < 9; ++o) st[o * (size_t)nvert + t] = acc[o];
  }
}

// Galerkin coarse stencil A_c = P^T A_f P for bilinear P.
__global__ void galerkin_stencil_kernel(int nxc, int nyc, const double* __restrict__ stf,
                                        double* __restrict__ stc) {
  const int nxf = 2 * nxc, nyf = 2 * nyc;
  const int nvxc = nxc - 1, nvertc = (nxc - 1) * (nyc - 1);
  const int nvxf = nxf - 1, nvertf = (nxf - 1) * (nyf - 1);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nvertc * 9; t += gridDim.x * blockDim.x) {
    const int v = t % nvertc, o = t / nvertc;
    const int I = v % nvxc + 1, J = v / nvxc + 1;
    const int dx = o % 3 - 1, dy = o / 3 - 1;
    const int I2 = I + dx, J2 = J + dy;
    double s = 0.0;
    if (I2 > 0 && J2 > 0 && I2 < nxc && J2 < nyc) {
      for (int b = -1; b <= 1; ++b)
        for (int a = -1; a <= 1; ++a) {
          const int ui = 2 * I + a, uj = 2 * J + b;
          if (ui <= 0 || uj <= 0 || ui >= nxf || uj >= nyf) continue;
          const double wu = (a == 0 ? 1.0 : 0.5) * (b == 0 ? 1.0 : 0.5);
          for (int b2 = -1; b2 <= 1; ++b2)
            for (int a2 = -1; a2 <= 1; ++a2) {
              const int vi = 2 * I2 + a2, vj = 2 * J2 + b2;
              if (vi <= 0 || vj <= 0 || vi >= nxf || vj >= nyf) continue;
              const int ox = vi - ui, oy = vj - uj;
              if (ox < -1 || ox > 1 || oy < -1 || oy > 1) continue;
              const double wv = (a2 == 0 ? 1.0 : 0.5) * (b2 == 0 ? 1.0 : 0.5);
              s += wu * wv * stf[((oy + 1) * 3 + ox + 1) * (size_t)nvertf + (ui - 1) + nvxf * (uj - 1)];
            }
        }
    }
    stc[o * (size_t)nvertc + v] = s;
  }
}

__global__ void stencil_diag_kernel(int nvert, const double* __restrict__ st, double* __restrict__ dinv64,
                                    float* __restrict__ dinv32) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nvert; t += gridDim.x * blockDim.x) {
    const double v = 1.0 / st[4 * (size_t)nvert + t];
    dinv64[t] = v;
    if (dinv32) dinv32[t] = (float)v;
  }
}

// ---------------------------------------------------------------------------
// Coarsest level: dense FP64 matrix from the stencil, Cholesky (one block),
// and the per-cycle triangular solves (one block).
__global__ void dense_from_stencil_kernel(int nx, int ny, const double* __restrict__ st, double* __restrict__ A) {
  const int nvx = nx - 1, n = (nx - 1) * (ny - 1);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * n; t += gridDim.x * blockDim.x) A[t] = 0.0;
  __syncthreads();
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int I = t % nvx, J = t / nvx;
    for (int o = 0; o < 9; ++o) {
      const int I2 = I + o % 3 - 1, J2 = J + o / 3 - 1;
      if (I2 < 0 || J2 < 0 || I2 >= nvx || J2 >= ny - 1) continue;
      A[(size_t)t * n + I2 + nvx * J2] = st[o * (size_t)n + t];
    }
  }
}

__global__ void cholesky_block_kernel(int n, double* __restrict__ A, int* err) {
  for (int j = 0; j < n; ++j) {
    __syncthreads();
    const double ajj = A[(size_t)j * n + j];
    if (!(ajj > 0.0) && threadIdx.x == 0) atomicExch(err, 4);
    const double d = sqrt(fmax(ajj, 1e-300));
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[(size_t)i * n + j] /= d;
    __syncthreads();
    if (threadIdx.x == 0) A[(size_t)j * n + j] = d;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const double lij = A[(size_t)i * n + j];
      for (int l = j + 1; l <= i; ++l) A[(size_t)i * n + l] -= lij * A[(size_t)l * n + j];
    }
  }
}

// one CTA per right-hand side (column blockIdx.x of [n][nb]); w: [nb][n] scratch
template <typename T>
__global__ void coarse_solve_kernel(int n, int nb, const double* __restrict__ L, const T* __restrict__ r,
                                    T* __restrict__ x, double* __restrict__ w) {
  const int col = blockIdx.x;
  w += (size_t)col * n;
  // forward then backward substitution, rows in parallel over threads
  for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = (double)r[(size_t)i * nb + col];
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) w[j] /= L[(size_t)j * n + j];
    __syncthreads();
    const double wj = w[j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) w[i] -= L[(size_t)i * n + j] * wj;
    __syncthreads();
  }
  for (int j = n - 1; j >= 0; --j) {
    if (threadIdx.x == 0) w[j] /= L[(size_t)j * n + j];
    __syncthreads();
    const double wj = w[j];
    for (int i = threadIdx.x; i < j; i += blockDim.x) w[i] -= L[(size_t)j * n + i] * wj;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[(size_t)i * nb + col] = (T)w[i];
}

// column j of the coarsest operator's inverse (L L^T)^-1 e_j for the fused
// coarse cycle: one CTA per column, the substitutions of coarse_solve_kernel on
// the unit vector in shared memory; stored transposed, AinvT[j][i] = (A^-1)_ij
__global__ void coarse_inverse_kernel(int n, const double* __restrict__ L, double* __restrict__ AinvT) {
  extern __shared__ double cw[];
  const int col = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) cw[i] = (i == col) ? 1.0 : 0.0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) cw[j] /= L[(size_t)j * n + j];
    __syncthreads();
    const double wj = cw[j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) cw[i] -= L[(size_t)i * n + j] * wj;
    __syncthreads();
  }
  for (int j = n - 1; j >= 0; --j) {
    if (threadIdx.x == 0) cw[j] /= L[(size_t)j * n + j];
    __syncthreads();
    const double wj = cw[j];
    for (int i = threadIdx.x; i < j; i += blockDim.x) cw[i] -= L[(size_t)j * n + i] * wj;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) AinvT[(size_t)col * n + i] = cw[i];
}

// ---------------------------------------------------------------------------
// Coarse Q1 levels in one launch. From the first Q1 level whose data, with
// every coarser level's, fits in one CTA's shared memory, the rest of Alg. 1
// -- Chebyshev pre-smoothing, residual, restriction, the coarsest solve,
// prolongation and post-smoothing on the way up -- runs in one CTA: stencils,
// diagonals and vectors of those levels are staged in shared memory, and every
// step is a phase over the level's entries with the per-entry arithmetic of
// the one-launch-per-step kernels, phases separated by __syncthreads. On
// meshes of a few hundred vertices each step is launch-latency bound as its own
// kernel; here it costs a barrier and shared-memory latency. The coarsest solve
// is x = A_c^-1 r with the inverse formed at set-up from the Cholesky factor
// (its 2n dependent substitution steps would cost more than the whole cycle).
constexpr int kHfMaxLevels = 8;
constexpr int kHfMaxCoef = 7;         // cheb_degree <= 8
constexpr int kHfThreads = 512;
constexpr int kHfMaxCoarse = 1024;    // largest coarsest system solved through its inverse

// one fused level: global sources of its read-only data, offsets (in entries
// of T) of its arrays in the shared-memory image, Chebyshev coefficients
template <typename T>
struct HfLevel {
  int nx, ny;
  const T* st_g;                       // stencil [9][nv] (global)
  const T* rs_g;                       // row sums (float levels) or null
  const T* dinv_g;                     // Jacobi diagonal inverse
  int o_st, o_rs, o_dinv;              // shared offsets (o_rs < 0: none)
  int o_r, o_x, o_t, o_d, o_d2;        // vectors [nv][nb]
  T c0, a1[kHfMaxCoef], a2[kHfMaxCoef];
};
template <typename T>
struct HfArgs {
  int nlev, nb, nu1, nu2, ncoef, nc;   // fused levels (the last is the coarsest), coarsest unknowns
  const double* AinvT;                 // [nc][nc] transposed inverse of the coarsest operator
  const T* r_top;                      // right-hand side of the top fused level (global)
  T* x_top;                            // its correction (global)
  HfLevel<T> L[kHfMaxLevels];
};

// shared-memory view of a fused level
template <typename T>
struct HfView {
  int nx, ny;
  const T *st, *rs, *dinv;
  T *r, *x, *t, *d, *d2;
};
template <typename T>
__device__ __forceinline__ HfView<T> hf_view(const HfLevel<T>& L, T* sm) {
  HfView<T> v;
  v.nx = L.nx; v.ny = L.ny;
  v.st = sm + L.o_st; v.rs = L.o_rs >= 0 ? sm + L.o_rs : nullptr; v.dinv = sm + L.o_dinv;
  v.r = sm + L.o_r; v.x = sm + L.o_x; v.t = sm + L.o_t; v.d = sm + L.o_d; v.d2 = sm + L.o_d2;
  return v;
}

// nu Chebyshev steps on a fused level (the phases of cheb_smooth's Q1 branch)
template <typename T>
__device__ void hf_smooth(const HfView<T>& L, const HfLevel<T>& C, int nb, int ncoef, bool x_zero, int nu) {
  const size_t n = (size_t)(L.nx - 1) * (L.ny - 1) * nb;
  T* da = L.d;
  T* db = L.d2;
  for (int step = 0; step < nu; ++step) {
    const T* rin;
    int add_d;
    if (step == 0 && x_zero) {
      for (size_t tt = threadIdx.x; tt < n; tt += blockDim.x) cheb_first_zero_at<T>(tt, nb, L.dinv, L.r, L.x, da, C.c0);
      rin = L.r;
      add_d = 0;
    } else {
      for (size_t tt = threadIdx.x; tt < n; tt += blockDim.x)
        cheb_resid_at<T>(tt, L.nx, L.ny, nb, L.st, L.rs, L.dinv, L.r, L.x, L.t, da, C.c0);
      rin = L.t;
      add_d = 1;
    }
    __syncthreads();
    for (int i = 0; i < ncoef; ++i) {
      for (size_t tt = threadIdx.x; tt < n; tt += blockDim.x)
        cheb_next_at<T>(tt, L.nx, L.ny, nb, L.st, L.rs, L.dinv, rin, L.t, da, db, L.x, C.a1[i], C.a2[i], add_d);
      __syncthreads();
      T* tmp = da; da = db; db = tmp;
      rin = L.t;
      add_d = 0;
    }
    if (add_d) {   // degree 1: x += d
      for (size_t tt = threadIdx.x; tt < n; tt += blockDim.x) cheb_step_at<T>(tt, nb, L.dinv, L.t, L.x, da, T(1), T(0));
      __syncthreads();
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kHfThreads, 1) hcoarse_kernel(const __grid_constant__ HfArgs<T> A) {
  extern __shared__ __align__(16) unsigned char hf_smem[];
  T* sm = reinterpret_cast<T*>(hf_smem);
  const int nb = A.nb;
  // stage the levels' stencils and diagonals and the top right-hand side
  for (int l = 0; l + 1 < A.nlev; ++l) {
    const HfLevel<T>& C = A.L[l];
    const int nv = (C.nx - 1) * (C.ny - 1);
    for (int i = threadIdx.x; i < 9 * nv; i += blockDim.x) sm[C.o_st + i] = C.st_g[i];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
      sm[C.o_dinv + i] = C.dinv_g[i];
      if (C.o_rs >= 0) sm[C.o_rs + i] = C.rs_g[i];
    }
  }
  {
    const HfLevel<T>& C = A.L[0];
    const int n = (C.nx - 1) * (C.ny - 1) * nb;
    for (int i = threadIdx.x; i < n; i += blockDim.x) sm[C.o_r + i] = A.r_top[i];
  }
  __syncthreads();
  for (int l = 0; l + 1 < A.nlev; ++l) {                  // down: smooth, residual, restrict
    const HfView<T> L = hf_view(A.L[l], sm);
    const HfView<T> Lc = hf_view(A.L[l + 1], sm);
    hf_smooth<T>(L, A.L[l], nb, A.ncoef, true, A.nu1);
    const size_t n = (size_t)(L.nx - 1) * (L.ny - 1) * nb;
    for (size_t tt = threadIdx.x; tt < n; tt += blockDim.x)
      stencil_apply_at<T>(tt, L.nx, L.ny, nb, L.st, L.x, L.r, L.t, T(-1), T(1), L.rs);
    __syncthreads();
    const size_t nc = (size_t)(Lc.nx - 1) * (Lc.ny - 1) * nb;
    for (size_t tt = threadIdx.x; tt < nc; tt += blockDim.x) restrict_q_at<T>(tt, Lc.nx, Lc.ny, nb, L.t, Lc.r);
    __syncthreads();
  }
  {                                                       // coarsest: x = A_c^-1 r in FP64
    const HfView<T> Lc = hf_view(A.L[A.nlev - 1], sm);
    const int n = A.nc;
    for (size_t tt = threadIdx.x; tt < (size_t)n * nb; tt += blockDim.x) {
      const int i = (int)(tt / nb), col = (int)(tt - (size_t)i * nb);
      double acc = 0.0;
      for (int j = 0; j < n; ++j) acc += A.AinvT[(size_t)j * n + i] * (double)Lc.r[(size_t)j * nb + col];
      Lc.x[tt] = (T)acc;
    }
    __syncthreads();
  }
  for (int l = A.nlev - 2; l >= 0; --l) {                 // up: prolong, smooth
    const HfView<T> L = hf_view(A.L[l], sm);
    const HfView<T> Lc = hf_view(A.L[l + 1], sm);
    const size_t n = (size_t)(L.nx - 1) * (L.ny - 1) * nb;
    for (size_t tt = threadIdx.x; tt < n; tt += blockDim.x) prolong_q_add_at<T>(tt, Lc.nx, Lc.ny, nb, Lc.x, L.x);
    __syncthreads();
    hf_smooth<T>(L, A.L[l], nb, A.ncoef, false, A.nu2);
  }
  {
    const HfLevel<T>& C = A.L[0];
    const int n = (C.nx - 1) * (C.ny - 1) * nb;
    for (int i = threadIdx.x; i < n; i += blockDim.x) A.x_top[i] = sm[C.o_x + i];
  }
}

// ---------------------------------------------------------------------------
// Power-iteration start vector s_i = ((7919 i) mod 1009) / 1009 - 1/2 over the
// interior unknowns in increasing order (for p = 0: interior edges, vertical
// ones before horizontal ones).
__global__ void power_start_edges_kernel(int nx, int ny, double* __restrict__ x) {
  const int nv = (nx + 1) * ny, ne = nv + nx * (ny + 1);
  const int nvi = (nx - 1) * ny;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ne; t += gridDim.x * blockDim.x) {
    long idx = -1;
    if (t < nv) {
      const int i = t % (nx + 1), j = t / (nx + 1);
      if (i > 0 && i < nx) idx = (long)j * (nx - 1) + (i - 1);
    } else {
      const int u = t - nv, i = u % nx, j = u / nx;
      if (j > 0 && j < ny) idx = nvi + (long)(j - 1) * nx + i;
    }
    x[t] = idx < 0 ? 0.0 : (double)((7919L * idx) % 1009L) / 1009.0 - 0.5;
  }
}
__global__ void power_start_verts_kernel(int n, double* __restrict__ x) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
    x[t] = (double)((7919L * t) % 1009L) / 1009.0 - 0.5;
}

// ---------------------------------------------------------------------------
// Level operators used by the V-cycle, generic over the vector type; nb
// right-hand sides per unknown.
static cudaError_t p0_apply(Context* c, int prec, const void* v, const void* cv, void* y, double al, double be,
                            int nb, cudaStream_t s) {
  return launch_apply(c, 0, 0, prec, v, cv, y, al, be, nb, s);
}

template <typename T>
static cudaError_t q_apply(HLevel& H, const T* st, const T* x, const T* cv, T* y, double al, double be, int nb,
                           cudaStream_t s) {
  // float levels use the difference form (rowsum32), double levels the plain one
  const T* rs = (sizeof(T) == 4) ? (const T*)(const void*)H.rsum32 : nullptr;
  stencil_apply_kernel<T><<<grid_for((size_t)H.nv * nb), 256, 0, s>>>(H.nx, H.ny, nb, st, x, cv, y, (T)al, (T)be, rs);
  return cudaGetLastError();
}

struct ChebCoef {
  double c0;
  std::vector<double> a1, a2;
};
static ChebCoef cheb_coefficients(double lmax, int degree) {
  const double a = 0.1 * lmax, b = 1.1 * lmax;
  const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
  ChebCoef cc;
  cc.c0 = 1.0 / theta;
  double rho = 1.0 / sigma;
  for (int i = 1; i < degree; ++i) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    cc.a1.push_back(rn * rho);
    cc.a2.push_back(2.0 * rn / delta);
    rho = rn;
  }
  return cc;
}

// nu Chebyshev smoothing steps on one h-level (the p = 0 level when H == nullptr).
template <typename T>
static cudaError_t cheb_smooth(Context* c, int prec, HLevel* H, const T* f, T* x, T* t, T* d, T* d2, bool x_zero,
                               int nu, int nb, cudaStream_t s) {
  const bool p0 = (H == nullptr);
  if (!p0) {   // Q1 level: fused stencil + update kernels
    const int n = H->nv * nb;
    const int g = grid_for((size_t)n);
    const T* dinv = (const T*)(prec_double(prec) ? (const void*)H->dinv64 : (const void*)H->dinv32);
    const T* st = (const T*)(prec_double(prec) ? (const void*)H->st64 : (const void*)H->st32);
    const T* rs = (sizeof(T) == 4) ? (const T*)(const void*)H->rsum32 : nullptr;
    const ChebCoef cc = cheb_coefficients(H->lmax, c->opt.cheb_degree);
    T* da = d;
    T* db = d2;
    for (int step = 0; step < nu; ++step) {
      const T* rin;
      bool add_d;
      if (step == 0 && x_zero) {
        cheb_first_zero_kernel<T><<<g, 256, 0, s>>>((size_t)n, nb, dinv, f, x, da, (T)cc.c0);
        rin = f;
        add_d = false;           // x already holds d
      } else {
        cheb_resid_kernel<T><<<g, 256, 0, s>>>(H->nx, H->ny, nb, st, rs, dinv, f, x, t, da, (T)cc.c0);
        rin = t;
        add_d = true;
      }
      HDG_CUDA_TRY(cudaGetLastError());
      for (size_t i = 0; i < cc.a1.size(); ++i) {
        cheb_next_kernel<T><<<g, 256, 0, s>>>(H->nx, H->ny, nb, st, rs, dinv, rin, t, da, db, x, (T)cc.a1[i],
                                              (T)cc.a2[i], add_d ? 1 : 0);
        HDG_CUDA_TRY(cudaGetLastError());
        T* tmp = da; da = db; db = tmp;
        rin = t;
        add_d = false;
      }
      if (add_d) {               // degree 1: x += d
        cheb_step_kernel<T><<<g, 256, 0, s>>>((size_t)n, nb, dinv, t, x, da, (T)1, (T)0);
        HDG_CUDA_TRY(cudaGetLastError());
      }
    }
    return cudaSuccess;
  }
  PLevel& L0 = c->plev[0];
  const size_t n = (p0 ? (size_t)c->n_edges : (size_t)H->nv) * nb;
  const T* dinv = p0 ? (const T*)(prec_double(prec) ? (const void*)L0.dinv64 : (const void*)L0.dinv32)
                     : (const T*)(prec_double(prec) ? (const void*)H->dinv64 : (const void*)H->dinv32);
  const T* st = p0 ? nullptr : (const T*)(prec_double(prec) ? (const void*)H->st64 : (const void*)H->st32);
  const ChebCoef cc = cheb_coefficients(p0 ? L0.lmax : H->lmax, c->opt.cheb_degree);
  auto A = [&](const T* v, const T* cv, T* y, double al, double be) -> cudaError_t {
    if (p0) return p0_apply(c, prec, v, cv, y, al, be, nb, s);
    return q_apply<T>(*H, st, v, cv, y, al, be, nb, s);
  };
  const int g = grid_for(n);
  for (int step = 0; step < nu; ++step) {
    const T* rsrc;
    if (step == 0 && x_zero) {
      cheb_first_zero_kernel<T><<<g, 256, 0, s>>>(n, nb, dinv, f, x, d, (T)cc.c0);
      HDG_CUDA_TRY(cudaGetLastError());
      rsrc = f;
    } else {
      HDG_CUDA_TRY(A(x, f, t, -1.0, 1.0));                    // t = f - A x
      cheb_step_kernel<T><<<g, 256, 0, s>>>(n, nb, dinv, t, x, d, (T)0, (T)cc.c0);   // d = c0 D^-1 t
      HDG_CUDA_TRY(cudaGetLastError());
      rsrc = t;
    }
    for (size_t i = 0; i < cc.a1.size(); ++i) {
      HDG_CUDA_TRY(A(d, rsrc, t, -1.0, 1.0));                 // t = r - A d
      cheb_step_kernel<T><<<g, 256, 0, s>>>(n, nb, dinv, t, x, d, (T)cc.a1[i], (T)cc.a2[i]);
      HDG_CUDA_TRY(cudaGetLastError());
      rsrc = t;
    }
  }
  return cudaSuccess;
}

// Shared-memory image of the fused levels l0..nh-1 for nb right-hand sides in
// vector type T: per smoothed level the stencil, diagonal (and row sums for
// float), and r, x, t, d, d2; r and x of the coarsest. Offsets in entries of T,
// each array starting on a 16-byte boundary. Returns the image's size in bytes.
template <typename T>
static size_t hfuse_layout(const Context* c, int l0, int nb, HfLevel<T>* L) {
  const int nh = (int)c->hlev.size();
  size_t off = 0;
  auto take = [&](size_t n) {
    const size_t o = off;
    off += (n * sizeof(T) + 15) / 16 * 16 / sizeof(T);
    return (int)o;
  };
  for (int l = l0; l < nh; ++l) {
    const HLevel& H = c->hlev[l];
    const size_t nv = (size_t)H.nv, nvb = nv * nb;
    HfLevel<T> z{};
    HfLevel<T>& C = L ? L[l - l0] : z;
    C.nx = H.nx;
    C.ny = H.ny;
    C.o_st = C.o_rs = C.o_dinv = C.o_t = C.o_d = C.o_d2 = -1;
    if (l < nh - 1) {
      C.o_st = take(9 * nv);
      C.o_dinv = take(nv);
      if (sizeof(T) == 4) C.o_rs = take(nv);
      C.o_t = take(nvb);
      C.o_d = take(nvb);
      C.o_d2 = take(nvb);
    }
    C.o_r = take(nvb);
    C.o_x = take(nvb);
  }
  return off * sizeof(T);
}

// First Q1 level of the fused coarse cycle for nb right-hand sides (-1: none):
// the first level whose image with all coarser levels fits in shared memory,
// at most kHfMaxLevels from the coarsest, and above it (a lone coarsest solve
// gains nothing). Double levels also keep to kHfMaxDoubleEntries entries: one
// SM retires only about two FP64 FMAs per clock on this GPU, so a 961-vertex
// level costs ~3 us per phase in one CTA, more than a launch of its own.
constexpr long kHfMaxDoubleEntries = 512;
template <typename T>
static int hfuse_level(const Context* c, int nb, size_t* bytes) {
  const int nh = (int)c->hlev.size();
  if (!c->opt.coarse_fuse || !c->coarse_AinvT || nh < 2) return -1;
  const size_t budget = (size_t)c->smem_optin;
  for (int l0 = std::max(0, nh - kHfMaxLevels); l0 <= nh - 2; ++l0) {
    if (sizeof(T) == 8 && (long)c->hlev[l0].nv * nb > kHfMaxDoubleEntries) continue;
    const size_t b = hfuse_layout<T>(c, l0, nb, nullptr);
    if (b <= budget) {
      if (bytes) *bytes = b;
      return l0;
    }
  }
  return -1;
}

// The cycle below Q1 level l0 in one launch (hcoarse_kernel): r, x are level
// l0's vectors; the coarser levels live in the kernel's shared memory.
template <typename T>
static cudaError_t launch_hcoarse(Context* c, int prec, int l0, size_t bytes, int nb, const T* r, T* x,
                                  cudaStream_t s) {
  const int nh = (int)c->hlev.size();
  HfArgs<T> A{};
  A.nlev = nh - l0;
  A.nb = nb;
  A.nu1 = c->opt.nu1;
  A.nu2 = c->opt.nu2;
  A.nc = c->coarse_dim;
  A.AinvT = c->coarse_AinvT;
  A.r_top = r;
  A.x_top = x;
  hfuse_layout<T>(c, l0, nb, A.L);
  for (int i = 0; i + 1 < A.nlev; ++i) {
    const HLevel& H = c->hlev[l0 + i];
    HfLevel<T>& L = A.L[i];
    L.st_g = (const T*)(prec_double(prec) ? (const void*)H.st64 : (const void*)H.st32);
    L.rs_g = (sizeof(T) == 4) ? (const T*)(const void*)H.rsum32 : nullptr;
    L.dinv_g = (const T*)(prec_double(prec) ? (const void*)H.dinv64 : (const void*)H.dinv32);
    const ChebCoef cc = cheb_coefficients(H.lmax, c->opt.cheb_degree);
    if ((int)cc.a1.size() > kHfMaxCoef) return cudaErrorInvalidValue;
    L.c0 = (T)cc.c0;
    A.ncoef = (int)cc.a1.size();
    for (size_t j = 0; j < cc.a1.size(); ++j) {
      L.a1[j] = (T)cc.a1[j];
      L.a2[j] = (T)cc.a2[j];
    }
  }
  HDG_CUDA_TRY(cudaFuncSetAttribute(hcoarse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  hcoarse_kernel<T><<<1, kHfThreads, bytes, s>>>(A);
  return cudaGetLastError();
}

// Alg. 1 on the h-levels: level l = -1 is the p = 0 HDG space, l >= 0 the Q1
// levels (finest first); the last Q1 level is solved directly.
template <typename T>
static cudaError_t hmg(Context* c, VWork& w, int prec, int l, const T* r, T* x, cudaStream_t s) {
  const int nh = (int)c->hlev.size();
  const int nb = w.nb;
  if (l >= 0) {
    size_t hb = 0;
    if (l == hfuse_level<T>(c, nb, &hb)) return launch_hcoarse<T>(c, prec, l, hb, nb, r, x, s);
  }
  if (l == nh - 1) {
    HLevel& H = c->hlev[l];
    coarse_solve_kernel<T><<<nb, 256, 0, s>>>(H.nv, nb, c->coarse_L, r, x, w.coarse_w);
    return cudaGetLastError();
  }
  const bool p0 = (l < 0);
  HLevel* H = p0 ? nullptr : &c->hlev[l];
  T* t = (T*)(p0 ? w.pt[0] : w.ht[l]);
  T* d = (T*)(p0 ? w.p0d : w.hd[l]);
  T* d2 = p0 ? nullptr : (T*)w.hd2[l];
  HDG_CUDA_TRY(cheb_smooth<T>(c, prec, H, r, x, t, d, d2, true, c->opt.nu1, nb, s));
  // residual and restriction to the next (coarser) Q1 level
  HLevel& Hc = c->hlev[l + 1];
  T* rc = (T*)w.hr[l + 1];
  T* xc = (T*)w.hx[l + 1];
  if (p0) {
    HDG_CUDA_TRY(p0_apply(c, prec == HDG_PREC_BF16 ? HDG_PREC_FP32 : prec, x, r, t, -1.0, 1.0, nb, s));
    restrict_J_kernel<T><<<grid_for((size_t)Hc.nv * nb), 256, 0, s>>>(c->mesh.nx, c->mesh.ny, nb, t, rc);
  } else {
    const T* st = (const T*)(prec_double(prec) ? (const void*)H->st64 : (const void*)H->st32);
    HDG_CUDA_TRY(q_apply<T>(*H, st, x, r, t, -1.0, 1.0, nb, s));
    restrict_q_kernel<T><<<grid_for((size_t)Hc.nv * nb), 256, 0, s>>>(Hc.nx, Hc.ny, nb, t, rc);
  }
  HDG_CUDA_TRY(cudaGetLastError());
  HDG_CUDA_TRY(hmg<T>(c, w, prec, l + 1, rc, xc, s));
  if (p0)
    prolong_J_add_kernel<T><<<grid_for((size_t)c->n_edges * nb), 256, 0, s>>>(c->mesh.nx, c->mesh.ny, nb, xc, x);
  else
    prolong_q_add_kernel<T><<<grid_for((size_t)H->nv * nb), 256, 0, s>>>(Hc.nx, Hc.ny, nb, xc, x);
  HDG_CUDA_TRY(cudaGetLastError());
  return cheb_smooth<T>(c, prec, H, r, x, t, d, d2, false, c->opt.nu2, nb, s);
}

// Finest level of a float V-cycle: its correction x is accumulated as a
// double-float pair hi + lo (two floats, ~48 significant bits), hi being the
// float vector the level's kernels read. A float cycle that rounds x to float
// after every update converges markedly slower on fine meshes (51 against 36
// CG iterations at 512^2, k = 4): x is the sum of the prolongated coarse
// correction and the smoothing increments, and its float rounding loses the
// smaller, oscillatory part that the outer CG needs. Every operator of the
// cycle stays in float; only this sum is kept wider.
// (hi, lo) = (set ? 0 : (hi, lo)) + u, by Knuth's two-sum and a renormalisation
__global__ void df_acc_kernel(size_t n, const float* __restrict__ u, float* __restrict__ hi, float* __restrict__ lo,
                              int set) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const float ut = u[t];
    if (set) {
      hi[t] = ut;
      lo[t] = 0.0f;
      continue;
    }
    const float a = hi[t];
    const float sum = __fadd_rn(a, ut);
    const float bv = __fsub_rn(sum, a);
    const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(sum, bv)), __fsub_rn(ut, bv));
    const float l = __fadd_rn(lo[t], err);
    const float h2 = __fadd_rn(sum, l);
    hi[t] = h2;
    lo[t] = __fsub_rn(l, __fsub_rn(h2, sum));
  }
}
// z = hi + lo in double (a float z: hi)
__global__ void df_out_kernel(size_t n, const float* __restrict__ hi, const float* __restrict__ lo,
                              double* __restrict__ z) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    z[t] = (double)hi[t] + (double)lo[t];
}
// (hi, lo) += P xc on the finest level of a float cycle, in double-float
// arithmetic: P = Phi + Plo (the FP64 weights as two floats), every product
// ph x split exactly by an FMA, the sums by two-sum. The prolongated correction
// must not be rounded to float: its rounding (of the weights or of the result)
// is a rough perturbation of the smooth coarse correction that the level
// operator amplifies (a float prolongation here costs 51 instead of 36 CG
// iterations at 512^2, k = 4, even with the rest of the sum kept wide).
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}
template <int NC>
__global__ void prolong_p_df_kernel(int n_edges, int nb, const float* __restrict__ Phi, const float* __restrict__ Plo,
                                    const float* __restrict__ xc, float* __restrict__ hi, float* __restrict__ lo) {
  constexpr int NF = NC + 1;
  const size_t total = (size_t)n_edges * nb;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    int col;
    const size_t e = divmod(t, nb, &col);
    float v[NC];
#pragma unroll
    for (int b = 0; b < NC; ++b) v[b] = xc[(e * NC + b) * nb + col];
#pragma unroll
    for (int a = 0; a < NF; ++a) {
      float sh = 0.0f, sl = 0.0f;
#pragma unroll
      for (int b = 0; b < NC; ++b) {
        const float ph = __ldg(&Phi[a * NC + b]), pl = __ldg(&Plo[a * NC + b]);
        const float pr = __fmul_rn(ph, v[b]);
        float er = __fmaf_rn(ph, v[b], -pr);     // ph v = pr + er exactly
        er = __fmaf_rn(pl, v[b], er);
        float s2, e2;
        df_two_sum(sh, pr, s2, e2);
        sh = s2;
        sl = __fadd_rn(sl, __fadd_rn(e2, er));
      }
      const size_t o = (e * NF + a) * nb + col;
      float s2, e2;
      df_two_sum(hi[o], sh, s2, e2);
      const float l = __fadd_rn(lo[o], __fadd_rn(sl, e2));
      const float h2 = __fadd_rn(s2, l);
      hi[o] = h2;
      lo[o] = __fsub_rn(l, __fsub_rn(h2, s2));
    }
  }
}
static cudaError_t p_prolong_df(int n1c, int n_edges, int nb, const float* Phi, const float* Plo, const float* xc,
                                float* hi, float* lo, cudaStream_t s) {
  if (!Phi || !Plo) return cudaErrorInvalidValue;
  const int g = grid_for((size_t)n_edges * nb);
  switch (n1c) {
    case 1: prolong_p_df_kernel<1><<<g, 256, 0, s>>>(n_edges, nb, Phi, Plo, xc, hi, lo); break;
    case 2: prolong_p_df_kernel<2><<<g, 256, 0, s>>>(n_edges, nb, Phi, Plo, xc, hi, lo); break;
    case 3: prolong_p_df_kernel<3><<<g, 256, 0, s>>>(n_edges, nb, Phi, Plo, xc, hi, lo); break;
    case 4: prolong_p_df_kernel<4><<<g, 256, 0, s>>>(n_edges, nb, Phi, Plo, xc, hi, lo); break;
    case 5: prolong_p_df_kernel<5><<<g, 256, 0, s>>>(n_edges, nb, Phi, Plo, xc, hi, lo); break;
    case 6: prolong_p_df_kernel<6><<<g, 256, 0, s>>>(n_edges, nb, Phi, Plo, xc, hi, lo); break;
    case 7: prolong_p_df_kernel<7><<<g, 256, 0, s>>>(n_edges, nb, Phi, Plo, xc, hi, lo); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Alg. 2 on p-level p >= 1 (zero initial guess): r, x are level-p vectors.
template <typename T>
static cudaError_t pmg(Context* c, VWork& w, int prec, int p, const T* r, T* x, cudaStream_t s) {
  PLevel& L = c->plev[p];
  PLevel& Lc = c->plev[p - 1];
  const int nb = w.nb;
  T* t = (T*)w.pt[p];
  const int nu1 = c->opt.nu1, nu2 = c->opt.nu2;
  // finest level of a float cycle: x = hi (this x) + lo, every update u = M v
  // (or the prolongated correction) added by df_acc_kernel; a BF16 cycle runs
  // this level with the FP32 blocks (its BF16 Schwarz blocks there cost 46
  // instead of 36 CG iterations at 512^2, k = 4, more than they save) and the
  // coarser p-levels with the BF16 blocks
  const bool dfx = sizeof(T) == 4 && p == c->k && w.top_lo && w.top_u;
  const int mprec = (dfx && prec == HDG_PREC_BF16) ? HDG_PREC_FP32 : prec;
  // smoother M of this level: x_out = x_add + M v (Schwarz blocks, or G^T G)
  auto smooth1 = [&](const T* v, const T* xadd, T* xout) -> cudaError_t {
    if (c->opt.smoother == 1) return launch_fsai_smooth(c, p, prec, v, xadd, xout, w.pw[p], nb, s);
    return launch_apply(c, p, 1, mprec, v, xadd, xout, 1.0, xadd ? 1.0 : 0.0, nb, s);
  };
  const size_t nn = (size_t)c->n_edges * L.n1 * nb;
  auto dfacc = [&](const float* u, bool set) -> cudaError_t {
    df_acc_kernel<<<grid_for(nn), 256, 0, s>>>(nn, u, (float*)x, w.top_lo, set ? 1 : 0);
    return cudaGetLastError();
  };
  auto smooth = [&](const T* v, const T* xadd, T* xout) -> cudaError_t {
    if (!dfx) return smooth1(v, xadd, xout);
    HDG_CUDA_TRY(smooth1(v, nullptr, (T*)w.top_u));
    return dfacc(w.top_u, xadd == nullptr);
  };
  // pre-smoothing: x = M r, then x += M (r - A x)
  HDG_CUDA_TRY(smooth(r, nullptr, x));
  for (int i = 1; i < nu1; ++i) {
    HDG_CUDA_TRY(launch_apply(c, p, 0, mprec, x, r, t, -1.0, 1.0, nb, s));
    HDG_CUDA_TRY(smooth(t, x, x));
  }
  // restricted residual; a BF16 cycle takes it with the FP32 blocks: its smooth
  // part drives the coarse correction, and BF16 rounding (2^-9) of the blocks
  // would swamp it on fine meshes
  const int rprec = prec == HDG_PREC_BF16 ? HDG_PREC_FP32 : prec;
  HDG_CUDA_TRY(launch_apply(c, p, 0, rprec, x, r, t, -1.0, 1.0, nb, s));
  T* rc = (T*)w.pr[p - 1];
  T* xc = (T*)w.px[p - 1];
  const T* Pp = (const T*)(prec_double(prec) ? (const void*)L.Pp : (const void*)L.Pp32);
  HDG_CUDA_TRY(p_transfer<T>(true, Lc.n1, c->n_edges, nb, Pp, t, rc, s));
  if (p - 1 == 0) HDG_CUDA_TRY(hmg<T>(c, w, prec, -1, rc, xc, s));
  else HDG_CUDA_TRY(pmg<T>(c, w, prec, p - 1, rc, xc, s));
  if (dfx) {
    // the prolongated correction in double-float arithmetic with the
    // double-float weights, added to (hi, lo) unrounded
    HDG_CUDA_TRY(p_prolong_df(Lc.n1, c->n_edges, nb, L.Pp32, L.Pplo, (const float*)xc, (float*)x, w.top_lo, s));
  } else {
    HDG_CUDA_TRY(p_transfer<T>(false, Lc.n1, c->n_edges, nb, Pp, xc, x, s));
  }
  for (int i = 0; i < nu2; ++i) {
    HDG_CUDA_TRY(launch_apply(c, p, 0, mprec, x, r, t, -1.0, 1.0, nb, s));
    HDG_CUDA_TRY(smooth(t, x, x));
  }
  return cudaSuccess;
}

// V-cycle body on the work's top-level buffers r -> x of level k.
template <typename T>
static cudaError_t vcycle_body(Context* c, VWork& w, int prec, cudaStream_t s) {
  const T* r = (const T*)w.pr[c->k];
  T* x = (T*)w.px[c->k];
  if (c->k == 0) return hmg<T>(c, w, prec, -1, r, x, s);
  return pmg<T>(c, w, prec, c->k, r, x, s);
}

static cudaError_t vcycle_body_any(Context* c, VWork& w, int prec, cudaStream_t s) {
  if (prec_double(prec)) return vcycle_body<double>(c, w, prec, s);
  return vcycle_body<float>(c, w, prec, s);
}

// whether a float cycle on work w keeps its finest correction as hi + lo
static bool top_df(const Context* c, const VWork& w) { return !w.dbl && c->k >= 1 && w.top_lo && w.top_u; }

// z = V r on work w. r and z are double for FP64 / F32X2, float otherwise
// (device, [ndof][w.nb]); r_double: r and z are double for a float cycle.
static cudaError_t vcycle_typed(Context* c, VWork& w, int prec, const void* r, void* z, bool r_double,
                                cudaStream_t s) {
  const size_t n = (size_t)c->ndof * w.nb;
  const int g = grid_for(n);
  void* wr = w.pr[c->k];
  void* wx = w.px[c->k];
  if (prec_double(prec)) {
    HDG_CUDA_TRY(cudaMemcpyAsync(wr, r, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else if (r_double) {
    copy_convert_kernel<double, float><<<g, 256, 0, s>>>(n, (const double*)r, (float*)wr);
    HDG_CUDA_TRY(cudaGetLastError());
  } else {
    HDG_CUDA_TRY(cudaMemcpyAsync(wr, r, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  }
  const int gi = prec;
  if (c->opt.use_graphs) {
    if (w.graph[gi] == nullptr || w.gstream[gi] != s) {
      if (w.graph[gi]) { cudaGraphExecDestroy(w.graph[gi]); w.graph[gi] = nullptr; }
      cudaStream_t cap = s;
      bool own = false;
      if (cap == 0) {  // the legacy stream cannot be captured: capture on a private stream
        HDG_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        own = true;
      }
      cudaGraph_t g0;
      HDG_CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
      cudaError_t eb = vcycle_body_any(c, w, prec, cap);
      cudaError_t ee = cudaStreamEndCapture(cap, &g0);
      if (own) cudaStreamDestroy(cap);
      HDG_CUDA_TRY(eb);
      HDG_CUDA_TRY(ee);
      HDG_CUDA_TRY(cudaGraphInstantiate(&w.graph[gi], g0, 0));
      size_t nn = 0;
      HDG_CUDA_TRY(cudaGraphGetNodes(g0, nullptr, &nn));
      std::vector<cudaGraphNode_t> nodes(nn);
      HDG_CUDA_TRY(cudaGraphGetNodes(g0, nodes.data(), &nn));
      int nk = 0;
      for (auto nd : nodes) {
        cudaGraphNodeType ty;
        HDG_CUDA_TRY(cudaGraphNodeGetType(nd, &ty));
        if (ty == cudaGraphNodeTypeKernel) ++nk;
      }
      c->vcycle_kernels = nk;
      cudaGraphDestroy(g0);
      w.gstream[gi] = s;
    }
    HDG_CUDA_TRY(cudaGraphLaunch(w.graph[gi], s));
  } else {
    HDG_CUDA_TRY(vcycle_body_any(c, w, prec, s));
  }
  if (prec_double(prec)) {
    HDG_CUDA_TRY(cudaMemcpyAsync(z, wx, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else if (r_double) {
    if (top_df(c, w)) df_out_kernel<<<g, 256, 0, s>>>(n, (const float*)wx, w.top_lo, (double*)z);
    else copy_convert_kernel<float, double><<<g, 256, 0, s>>>(n, (const float*)wx, (double*)z);
    HDG_CUDA_TRY(cudaGetLastError());
  } else {
    HDG_CUDA_TRY(cudaMemcpyAsync(z, wx, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Works: the single-vector ones point into the levels' buffers; batched ones
// are allocated when first asked for with a given nb (and replaced when nb
// changes).
static void release_work(VWork& w) {
  for (int g = 0; g < 4; ++g) {
    if (w.graph[g]) cudaGraphExecDestroy(w.graph[g]);
    w.graph[g] = nullptr;
    w.gstream[g] = nullptr;
  }
  for (void* p : w.own) cudaFree(p);
  w.own.clear();
  if (w.h_sc) cudaFreeHost(w.h_sc);
  w.h_sc = nullptr;
}

void release_works(Context* c) {
  for (int g = 0; g < 4; ++g) {
    if (c->cg_graph[g]) cudaGraphExecDestroy(c->cg_graph[g]);
    c->cg_graph[g] = nullptr;
  }
  if (c->h_cg) cudaFreeHost(c->h_cg);
  c->h_cg = nullptr;
  for (int f = 0; f < 2; ++f) {
    release_work(c->w1[f]);
    if (c->wb[f]) {
      release_work(*c->wb[f]);
      delete c->wb[f];
      c->wb[f] = nullptr;
    }
  }
}

static void single_works(Context* c) {
  for (int f = 0; f < 2; ++f) {
    VWork& w = c->w1[f];
    const bool dbl = (f == 0);
    w.nb = 1;
    w.dbl = dbl;
    w.pr.clear(); w.px.clear(); w.pt.clear(); w.pw.clear();
    for (int p = 0; p <= c->k; ++p) {
      PLevel& L = c->plev[p];
      w.pr.push_back(dbl ? (void*)L.r64 : (void*)L.r32);
      w.px.push_back(dbl ? (void*)L.x64 : (void*)L.x32);
      w.pt.push_back(dbl ? (void*)L.t64 : (void*)L.t32);
      w.pw.push_back(dbl ? (void*)L.w64 : (void*)L.w32);
    }
    w.p0d = dbl ? (void*)c->plev[0].d64 : (void*)c->plev[0].d32;
    w.hr.clear(); w.hx.clear(); w.ht.clear(); w.hd.clear(); w.hd2.clear();
    for (HLevel& H : c->hlev) {
      w.hr.push_back(dbl ? (void*)H.r64 : (void*)H.r32);
      w.hx.push_back(dbl ? (void*)H.x64 : (void*)H.x32);
      w.ht.push_back(dbl ? (void*)H.t64 : (void*)H.t32);
      w.hd.push_back(dbl ? (void*)H.d64 : (void*)H.d32);
      w.hd2.push_back(dbl ? (void*)H.e64 : (void*)H.e32);
    }
    w.coarse_w = c->coarse_rhs;
    w.top_lo = dbl ? nullptr : c->top_lo32;
    w.top_u = dbl ? nullptr : c->top_u32;
  }
}

static void* work_alloc(VWork* w, size_t bytes) {
  void* p = nullptr;
  if (w->own_bytes + bytes > w->cap) return nullptr;   // the context's memory cap
  if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  w->own.push_back(p);
  w->own_bytes += bytes;
  return p;
}

// the batched CG vectors and scalars of a work (allocated once)
static cudaError_t work_cg(Context* c, VWork* w) {
  if (w->cg_r) return cudaSuccess;
  const size_t n = (size_t)c->ndof * w->nb * sizeof(double);
  w->cg_r = (double*)work_alloc(w, n); w->cg_z = (double*)work_alloc(w, n);
  w->cg_p = (double*)work_alloc(w, n); w->cg_q = (double*)work_alloc(w, n);
  w->cg_zold = (double*)work_alloc(w, n);
  w->cg_sc = (double*)work_alloc(w, (size_t)kCgScalars * w->nb * sizeof(double));
  w->cg_part = (double*)work_alloc(w, (size_t)2 * kColRedBlocks * w->nb * sizeof(double));
  bool ok = w->cg_r && w->cg_z && w->cg_p && w->cg_q && w->cg_zold && w->cg_sc && w->cg_part;
  if (ok) ok = cudaMallocHost((void**)&w->h_sc, 3 * (size_t)w->nb * sizeof(double)) == cudaSuccess;
  if (!ok) { cudaGetLastError(); w->cg_r = nullptr; return cudaErrorMemoryAllocation; }
  return cudaSuccess;
}

static cudaError_t batched_work(Context* c, int nb, bool dbl, VWork** out) {
  const int f = dbl ? 0 : 1;
  if (c->wb[f] && c->wb[f]->nb == nb) { *out = c->wb[f]; return cudaSuccess; }
  if (c->wb[f]) { release_work(*c->wb[f]); delete c->wb[f]; c->wb[f] = nullptr; }
  VWork* w = new VWork();
  w->nb = nb;
  w->dbl = dbl;
  if (c->opt.max_device_bytes) {
    // what the cap leaves after the set-up data and the other batched work
    size_t used = c->bytes;
    if (c->wb[1 - f]) used += c->wb[1 - f]->own_bytes;
    w->cap = c->opt.max_device_bytes > used ? c->opt.max_device_bytes - used : 0;
  }
  const size_t es = dbl ? sizeof(double) : sizeof(float);
  bool ok = true;
  for (int p = 0; p <= c->k && ok; ++p) {
    const size_t n = (size_t)c->n_edges * c->plev[p].n1 * nb * es;
    void *a = work_alloc(w, n), *b = work_alloc(w, n), *d = work_alloc(w, n);
    ok = a && b && d;
    w->pr.push_back(a); w->px.push_back(b); w->pt.push_back(d);
    void* fw = nullptr;
    if (ok && p >= 1 && c->opt.smoother == 1) { fw = work_alloc(w, n); ok = fw != nullptr; }
    w->pw.push_back(fw);
  }
  if (ok) { w->p0d = work_alloc(w, (size_t)c->n_edges * nb * es); ok = w->p0d != nullptr; }
  for (size_t l = 0; l < c->hlev.size() && ok; ++l) {
    const size_t n = (size_t)c->hlev[l].nv * nb * es;
    void *a = work_alloc(w, n), *b = work_alloc(w, n), *d = work_alloc(w, n), *e = work_alloc(w, n);
    void* e2 = work_alloc(w, n);
    ok = a && b && d && e && e2;
    w->hr.push_back(a); w->hx.push_back(b); w->ht.push_back(d); w->hd.push_back(e); w->hd2.push_back(e2);
  }
  if (ok) {
    w->coarse_w = (double*)work_alloc(w, (size_t)c->coarse_dim * nb * sizeof(double));
    ok = w->coarse_w != nullptr;
  }
  if (ok && !dbl && c->opt.top_accum && c->k >= 1) {   // hi + lo correction of the finest level
    const size_t n = (size_t)c->ndof * nb * sizeof(float);
    w->top_lo = (float*)work_alloc(w, n);
    w->top_u = (float*)work_alloc(w, n);
    ok = w->top_lo && w->top_u;
  }
  if (ok && c->opt.reduced == 1) {   // double-sized: the batched CG's outer apply is FP64 in every mode
    w->red_z = work_alloc(w, (size_t)c->nel * c->ref.m * nb * sizeof(double));
    ok = w->red_z != nullptr;
  }
  if (!ok) {
    release_work(*w);
    delete w;
    return cudaErrorMemoryAllocation;
  }
  c->wb[f] = w;
  *out = w;
  return cudaSuccess;
}

static void set_cols_scratch(Context* c, const VWork* w) {
  c->cur_zb = w->red_z;
  c->cur_zb_bytes = w->red_z ? (size_t)c->nel * c->ref.m * w->nb * sizeof(double) : 0;
}

cudaError_t use_batched_work(Context* c, int nb, int prec) {
  VWork* w = nullptr;
  HDG_CUDA_TRY(batched_work(c, nb, prec_double(prec), &w));
  set_cols_scratch(c, w);
  return cudaSuccess;
}

static cudaError_t alloc_vecs_d(Context* c, size_t n, std::initializer_list<double**> ps);

__global__ void fmg_add_kernel(size_t n, const double* __restrict__ z, double* __restrict__ x) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    x[t] += z[t];
}

// Full multigrid (Sec. 7) with FP64 V-cycles, one right-hand side: b restricted
// to every level, a direct solve on the coarsest mesh, then upwards level by
// level the coarser solution interpolated as the start and `cycles` V-cycles of
// that level's own hierarchy (hmg on the p = 0 and Q1 levels, pmg on the
// p-levels) applied to its residual. The per-level right-hand sides, solutions,
// residuals and corrections live in the context's FMG work (allocated on the
// first call); the V-cycles use the single-vector work as usual.
cudaError_t fmg_solve(Context* c, const double* b, double* x_out, int cycles, cudaStream_t s) {
  FmgWork& f = c->fmg;
  const int k = c->k, nh = (int)c->hlev.size();
  const size_t ne = (size_t)c->n_edges;
  if (!f.ready) {
    f.bp.assign(k + 1, nullptr); f.xp.assign(k + 1, nullptr); f.rp.assign(k + 1, nullptr); f.zp.assign(k + 1, nullptr);
    f.bh.assign(nh, nullptr); f.xh.assign(nh, nullptr); f.rh.assign(nh, nullptr); f.zh.assign(nh, nullptr);
    for (int p = 0; p <= k; ++p)
      HDG_CUDA_TRY(alloc_vecs_d(c, ne * c->plev[p].n1, {&f.bp[p], &f.xp[p], &f.rp[p], &f.zp[p]}));
    for (int l = 0; l < nh; ++l)
      HDG_CUDA_TRY(alloc_vecs_d(c, (size_t)c->hlev[l].nv, {&f.bh[l], &f.xh[l], &f.rh[l], &f.zh[l]}));
    f.ready = true;
  }
  VWork& w = c->w1[0];
  const int prec = HDG_PREC_FP64;
  // right-hand sides on every level (R = P^T)
  HDG_CUDA_TRY(cudaMemcpyAsync(f.bp[k], b, ne * (k + 1) * sizeof(double), cudaMemcpyDeviceToDevice, s));
  for (int p = k; p >= 1; --p)
    HDG_CUDA_TRY(p_transfer<double>(true, c->plev[p - 1].n1, c->n_edges, 1, c->plev[p].Pp, f.bp[p], f.bp[p - 1], s));
  restrict_J_kernel<double><<<grid_for((size_t)c->hlev[0].nv), 256, 0, s>>>(c->mesh.nx, c->mesh.ny, 1, f.bp[0],
                                                                           f.bh[0]);
  HDG_CUDA_TRY(cudaGetLastError());
  for (int l = 0; l + 1 < nh; ++l) {
    HLevel& Hc = c->hlev[l + 1];
    restrict_q_kernel<double><<<grid_for((size_t)Hc.nv), 256, 0, s>>>(Hc.nx, Hc.ny, 1, f.bh[l], f.bh[l + 1]);
    HDG_CUDA_TRY(cudaGetLastError());
  }
  // coarsest mesh: direct solve
  HDG_CUDA_TRY(hmg<double>(c, w, prec, nh - 1, f.bh[nh - 1], f.xh[nh - 1], s));
  // up the Q1 levels
  for (int l = nh - 2; l >= 0; --l) {
    HLevel& H = c->hlev[l];
    HLevel& Hc = c->hlev[l + 1];
    HDG_CUDA_TRY(cudaMemsetAsync(f.xh[l], 0, (size_t)H.nv * sizeof(double), s));
    prolong_q_add_kernel<double><<<grid_for((size_t)H.nv), 256, 0, s>>>(Hc.nx, Hc.ny, 1, f.xh[l + 1], f.xh[l]);
    HDG_CUDA_TRY(cudaGetLastError());
    for (int it = 0; it < cycles; ++it) {
      HDG_CUDA_TRY(q_apply<double>(H, H.st64, f.xh[l], f.bh[l], f.rh[l], -1.0, 1.0, 1, s));
      HDG_CUDA_TRY(hmg<double>(c, w, prec, l, f.rh[l], f.zh[l], s));
      fmg_add_kernel<<<grid_for((size_t)H.nv), 256, 0, s>>>((size_t)H.nv, f.zh[l], f.xh[l]);
      HDG_CUDA_TRY(cudaGetLastError());
    }
  }
  // the p = 0 level
  HDG_CUDA_TRY(cudaMemsetAsync(f.xp[0], 0, ne * sizeof(double), s));
  prolong_J_add_kernel<double><<<grid_for(ne), 256, 0, s>>>(c->mesh.nx, c->mesh.ny, 1, f.xh[0], f.xp[0]);
  HDG_CUDA_TRY(cudaGetLastError());
  for (int it = 0; it < cycles; ++it) {
    HDG_CUDA_TRY(p0_apply(c, prec, f.xp[0], f.bp[0], f.rp[0], -1.0, 1.0, 1, s));
    HDG_CUDA_TRY(hmg<double>(c, w, prec, -1, f.rp[0], f.zp[0], s));
    fmg_add_kernel<<<grid_for(ne), 256, 0, s>>>(ne, f.zp[0], f.xp[0]);
    HDG_CUDA_TRY(cudaGetLastError());
  }
  // up the p-levels
  for (int p = 1; p <= k; ++p) {
    const size_t n = ne * c->plev[p].n1;
    HDG_CUDA_TRY(cudaMemsetAsync(f.xp[p], 0, n * sizeof(double), s));
    HDG_CUDA_TRY(p_transfer<double>(false, c->plev[p - 1].n1, c->n_edges, 1, c->plev[p].Pp, f.xp[p - 1], f.xp[p], s));
    for (int it = 0; it < cycles; ++it) {
      HDG_CUDA_TRY(launch_apply(c, p, 0, prec, f.xp[p], f.bp[p], f.rp[p], -1.0, 1.0, 1, s));
      HDG_CUDA_TRY(pmg<double>(c, w, prec, p, f.rp[p], f.zp[p], s));
      fmg_add_kernel<<<grid_for(n), 256, 0, s>>>(n, f.zp[p], f.xp[p]);
      HDG_CUDA_TRY(cudaGetLastError());
    }
  }
  HDG_CUDA_TRY(cudaMemcpyAsync(x_out, f.xp[k], ne * (k + 1) * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return cudaSuccess;
}

cudaError_t vcycle(Context* c, int prec, const void* r, void* z, int nb, cudaStream_t s) {
  const bool dbl = prec_double(prec);
  if (nb == 1) return vcycle_typed(c, c->w1[dbl ? 0 : 1], prec, r, z, false, s);
  VWork* w = nullptr;
  HDG_CUDA_TRY(batched_work(c, nb, dbl, &w));
  set_cols_scratch(c, w);
  return vcycle_typed(c, *w, prec, r, z, false, s);
}

// ---------------------------------------------------------------------------
// Hierarchy construction (after the p-level blocks exist).
static cudaError_t alloc_vecs_d(Context* c, size_t n, std::initializer_list<double**> ps) {
  for (double** p : ps) HDG_CUDA_TRY(ctx_alloc(c, (void**)p, n * sizeof(double)));
  return cudaSuccess;
}
static cudaError_t alloc_vecs_f(Context* c, size_t n, std::initializer_list<float**> ps) {
  for (float** p : ps) HDG_CUDA_TRY(ctx_alloc(c, (void**)p, n * sizeof(float)));
  return cudaSuccess;
}

// lambda_max(D^-1 A) by 10 power iterations from the fixed pattern (FP64).
static cudaError_t power_iteration(Context* c, HLevel* H, double* out, cudaStream_t s) {
  const bool p0 = (H == nullptr);
  const size_t n = p0 ? (size_t)c->n_edges : (size_t)H->nv;
  double *x, *y;
  HDG_CUDA_TRY(cudaMallocAsync((void**)&x, n * sizeof(double), s));
  HDG_CUDA_TRY(cudaMallocAsync((void**)&y, n * sizeof(double), s));
  const int g = grid_for(n);
  if (p0) power_start_edges_kernel<<<g, 256, 0, s>>>(c->mesh.nx, c->mesh.ny, x);
  else power_start_verts_kernel<<<g, 256, 0, s>>>((int)n, x);
  HDG_CUDA_TRY(cudaGetLastError());
  const double* dinv = p0 ? c->plev[0].dinv64 : H->dinv64;
  double* sc = c->scal + 16;
  HDG_CUDA_TRY(dots<double>(c, n, x, x, nullptr, nullptr, nullptr, nullptr, sc, s));
  // x /= |x|: scale by 1/sqrt(sc[0]) -- done on the host-visible value below
  double h_nrm2 = 0.0;
  HDG_CUDA_TRY(cudaMemcpyAsync(&h_nrm2, sc, sizeof(double), cudaMemcpyDeviceToHost, s));
  HDG_CUDA_TRY(cudaStreamSynchronize(s));
  double* scale_dev = c->scal + 20;
  double one_over = std::sqrt(h_nrm2);
  HDG_CUDA_TRY(cudaMemcpyAsync(scale_dev, &one_over, sizeof(double), cudaMemcpyHostToDevice, s));
  scale_kernel<double><<<g, 256, 0, s>>>(n, x, scale_dev, 1.0);
  HDG_CUDA_TRY(cudaGetLastError());
  double lam = 0.0;
  for (int it = 0; it < 10; ++it) {
    if (p0) HDG_CUDA_TRY(p0_apply(c, HDG_PREC_FP64, x, nullptr, y, 1.0, 0.0, 1, s));
    else HDG_CUDA_TRY(q_apply<double>(*H, H->st64, x, nullptr, y, 1.0, 0.0, 1, s));
    mul_kernel<double><<<g, 256, 0, s>>>(n, y, dinv, y);
    HDG_CUDA_TRY(cudaGetLastError());
    HDG_CUDA_TRY(dots<double>(c, n, y, y, nullptr, nullptr, nullptr, nullptr, sc, s));
    HDG_CUDA_TRY(cudaMemcpyAsync(&h_nrm2, sc, sizeof(double), cudaMemcpyDeviceToHost, s));
    HDG_CUDA_TRY(cudaStreamSynchronize(s));
    lam = std::sqrt(h_nrm2);
    HDG_CUDA_TRY(cudaMemcpyAsync(scale_dev, &lam, sizeof(double), cudaMemcpyHostToDevice, s));
    scale_kernel<double><<<g, 256, 0, s>>>(n, y, scale_dev, 1.0);
    HDG_CUDA_TRY(cudaGetLastError());
    std::swap(x, y);
  }
  HDG_CUDA_TRY(cudaStreamSynchronize(s));
  *out = lam;
  HDG_CUDA_TRY(cudaFreeAsync(x, s));
  HDG_CUDA_TRY(cudaFreeAsync(y, s));
  return cudaSuccess;
}

cudaError_t build_hierarchy(Context* c, cudaStream_t s) {
  const bool mixed = c->opt.mixed != 0;
  const size_t ne = (size_t)c->n_edges;
  // p-level vectors
  for (int p = 0; p <= c->k; ++p) {
    PLevel& L = c->plev[p];
    const size_t n = ne * L.n1;
    HDG_CUDA_TRY(alloc_vecs_d(c, n, {&L.r64, &L.x64, &L.t64}));
    if (mixed) HDG_CUDA_TRY(alloc_vecs_f(c, n, {&L.r32, &L.x32, &L.t32}));
    if (p >= 1 && c->opt.smoother == 1) {
      HDG_CUDA_TRY(alloc_vecs_d(c, n, {&L.w64}));
      if (mixed) HDG_CUDA_TRY(alloc_vecs_f(c, n, {&L.w32}));
    }
  }
  // p = 0 Jacobi diagonal and Chebyshev direction vector
  PLevel& L0 = c->plev[0];
  HDG_CUDA_TRY(alloc_vecs_d(c, ne, {&L0.d64}));
  if (mixed) HDG_CUDA_TRY(alloc_vecs_f(c, ne, {&L0.d32}));
  HDG_CUDA_TRY(ctx_alloc(c, (void**)&L0.dinv64, ne * sizeof(double)));
  if (mixed) HDG_CUDA_TRY(ctx_alloc(c, (void**)&L0.dinv32, ne * sizeof(float)));
  HDG_CUDA_TRY(launch_p0_diag(c, s));
  if (mixed && c->opt.top_accum && c->k >= 1) {   // float cycles: hi + lo correction of the finest level
    HDG_CUDA_TRY(ctx_alloc(c, (void**)&c->top_lo32, (size_t)c->ndof * sizeof(float)));
    HDG_CUDA_TRY(ctx_alloc(c, (void**)&c->top_u32, (size_t)c->ndof * sizeof(float)));
  }
  // Q1 levels
  int nx = c->mesh.nx, ny = c->mesh.ny;
  c->hlev.clear();
  if (nx < 2 || ny < 2) return cudaErrorInvalidValue;
  {
    HLevel H; H.nx = nx; H.ny = ny; H.nv = (nx - 1) * (ny - 1);
    c->hlev.push_back(H);
  }
  const int cn = c->opt.coarse_n;
  while (nx % 2 == 0 && ny % 2 == 0 && nx / 2 >= cn && ny / 2 >= cn && nx > cn && nx / 2 >= 2 && ny / 2 >= 2) {
    nx /= 2; ny /= 2;
    HLevel H; H.nx = nx; H.ny = ny; H.nv = (nx - 1) * (ny - 1);
    c->hlev.push_back(H);
  }
  for (size_t l = 0; l < c->hlev.size(); ++l) {
    HLevel& H = c->hlev[l];
    const size_t n = (size_t)H.nv;
    HDG_CUDA_TRY(ctx_alloc(c, (void**)&H.st64, 9 * n * sizeof(double)));
    HDG_CUDA_TRY(alloc_vecs_d(c, n, {&H.dinv64, &H.r64, &H.x64, &H.t64, &H.d64, &H.e64}));
    if (mixed) {
      HDG_CUDA_TRY(ctx_alloc(c, (void**)&H.st32, 9 * n * sizeof(float)));
      HDG_CUDA_TRY(alloc_vecs_f(c, n, {&H.dinv32, &H.r32, &H.x32, &H.t32, &H.d32, &H.e32}));
    }
    if (l == 0) {
      q1_stencil_kernel<<<grid_for(n), 256, 0, s>>>(H.nx, H.ny, c->hx, c->hy, c->kappa, H.st64);
    } else {
      galerkin_stencil_kernel<<<grid_for(9 * n), 256, 0, s>>>(H.nx, H.ny, c->hlev[l - 1].st64, H.st64);
    }
    HDG_CUDA_TRY(cudaGetLastError());
    stencil_diag_kernel<<<grid_for(n), 256, 0, s>>>((int)n, H.st64, H.dinv64, H.dinv32);
    HDG_CUDA_TRY(cudaGetLastError());
    if (mixed) {
      copy_convert_kernel<double, float><<<grid_for(9 * n), 256, 0, s>>>(9 * n, H.st64, H.st32);
      HDG_CUDA_TRY(cudaGetLastError());
      HDG_CUDA_TRY(ctx_alloc(c, (void**)&H.rsum32, n * sizeof(float)));
      stencil_rowsum_kernel<<<grid_for(n), 256, 0, s>>>((int)n, H.st64, H.rsum32);
      HDG_CUDA_TRY(cudaGetLastError());
    }
  }
  // Chebyshev bounds on the smoothed levels (p = 0 and every Q1 level but the last)
  HDG_CUDA_TRY(power_iteration(c, nullptr, &L0.lmax, s));
  for (size_t l = 0; l + 1 < c->hlev.size(); ++l) HDG_CUDA_TRY(power_iteration(c, &c->hlev[l], &c->hlev[l].lmax, s));
  // coarsest dense Cholesky (FP64)
  HLevel& Hc = c->hlev.back();
  const int nc = Hc.nv;
  c->coarse_dim = nc;
  HDG_CUDA_TRY(ctx_alloc(c, (void**)&c->coarse_L, (size_t)nc * nc * sizeof(double)));
  HDG_CUDA_TRY(ctx_alloc(c, (void**)&c->coarse_rhs, (size_t)nc * sizeof(double)));
  dense_from_stencil_kernel<<<1, 256, 0, s>>>(Hc.nx, Hc.ny, Hc.st64, c->coarse_L);
  HDG_CUDA_TRY(cudaGetLastError());
  cholesky_block_kernel<<<1, 256, 0, s>>>(nc, c->coarse_L, c->err_flag);
  HDG_CUDA_TRY(cudaGetLastError());
  if (c->opt.coarse_fuse && nc <= kHfMaxCoarse && c->hlev.size() >= 2) {   // for the fused coarse cycle
    HDG_CUDA_TRY(ctx_alloc(c, (void**)&c->coarse_AinvT, (size_t)nc * nc * sizeof(double)));
    coarse_inverse_kernel<<<nc, 256, (size_t)nc * sizeof(double), s>>>(nc, c->coarse_L, c->coarse_AinvT);
    HDG_CUDA_TRY(cudaGetLastError());
  }
  single_works(c);
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Preconditioned CG on the FP64 trace system.
// scal layout: 0 rz, 1 pq, 2 rr, 3 r.zold, 4 bb, 8.. scratch
__global__ void cg_xr_kernel(size_t n, const double* __restrict__ scal, const double* __restrict__ p,
                             const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r) {
  const double alpha = scal[0] / scal[1];
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    x[t] += alpha * p[t];
    r[t] -= alpha * q[t];
  }
}
// p = z + beta p, beta = (r.z_new - r.z_old [flexible]) / rz_old; then rz <- r.z_new
__global__ void cg_p_kernel(size_t n, double* __restrict__ scal, const double* __restrict__ z,
                            double* __restrict__ p, int flexible) {
  const double rz_new = scal[8];
  const double num = flexible ? rz_new - scal[9] : rz_new;
  const double beta = num / scal[0];
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    p[t] = z[t] + beta * p[t];
}
__global__ void cg_commit_kernel(double* scal) { scal[0] = scal[8]; }

// ---------------------------------------------------------------------------
// Device-resident CG loop: the iterations of pcg_solve as the body of one
// conditional WHILE node of a CUDA graph, so that a solve is one graph launch
// with no host round trip per iteration. The body runs
//   [zold = z]; z = V r; rz_new = r.z [, r.zold]; p = z (first pass) or
//   z + beta p; rz = rz_new; q = A p; alpha = rz / p.q; x += alpha p;
//   r -= alpha q; rr = r.r; check (breakdown, rel <= rtol, maxit)
// -- the host loop's operations in its order (the host loop takes its first
// V-cycle before the loop, the device loop in its first pass), so both give
// the same iterates bit for bit. The graph reads only context buffers (its
// iterate is cg_x), so one graph per inner precision serves every call;
// rtol, |b| and maxit are device scalars set before each launch.
// scal slots: 16 rtol, 17 |b|, 19 relres; ctl: [0] iterations, [1] status
// (hdg_status, -1 while running), [2] maxit.
__global__ void cgd_init_kernel(double* scal, int* ctl, double rtol, int maxit) {
  scal[16] = rtol;
  scal[17] = sqrt(scal[4]);
  scal[19] = 1.0;
  ctl[0] = 0;
  ctl[1] = -1;
  ctl[2] = maxit;
}
__global__ void cgd_p_kernel(size_t n, const double* __restrict__ scal, const int* __restrict__ ctl,
                             const double* __restrict__ z, double* __restrict__ p, int flexible) {
  const bool first = ctl[0] == 0;
  double beta = 0.0;
  if (!first) {
    const double rz_new = scal[8];
    beta = (flexible ? rz_new - scal[9] : rz_new) / scal[0];
  }
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    p[t] = first ? z[t] : z[t] + beta * p[t];
}
__global__ void cgd_check_kernel(double* scal, int* ctl, double* hist, cudaGraphConditionalHandle h) {
  const int it = ctl[0] + 1;
  ctl[0] = it;
  const double pq = scal[1];
  int st = -1;
  double rel = scal[19];
  if (!(pq > 0.0) || !isfinite(pq)) {
    st = HDG_ERR_BREAKDOWN;
  } else {
    rel = sqrt(scal[2]) / scal[17];
    if (it < 256) hist[it] = rel;
    if (!isfinite(rel)) st = HDG_ERR_BREAKDOWN;
    else if (rel <= scal[16]) st = HDG_OK;
    else if (it >= ctl[2]) st = HDG_ERR_NOT_CONVERGED;
  }
  scal[19] = rel;
  ctl[1] = st;
  cudaGraphSetConditional(h, st < 0 ? 1u : 0u);
}

// z = V r for double r, z on the single-vector work, launched directly (no
// graph of its own: it is captured into the CG loop's body)
static cudaError_t vcycle_direct(Context* c, int prec, const double* r, double* z, cudaStream_t s) {
  VWork& w = c->w1[prec_double(prec) ? 0 : 1];
  const size_t n = (size_t)c->ndof;
  const int g = grid_for(n);
  if (prec_double(prec)) copy_convert_kernel<double, double><<<g, 256, 0, s>>>(n, r, (double*)w.pr[c->k]);
  else copy_convert_kernel<double, float><<<g, 256, 0, s>>>(n, r, (float*)w.pr[c->k]);
  HDG_CUDA_TRY(cudaGetLastError());
  HDG_CUDA_TRY(vcycle_body_any(c, w, prec, s));
  if (prec_double(prec)) copy_convert_kernel<double, double><<<g, 256, 0, s>>>(n, (const double*)w.px[c->k], z);
  else if (top_df(c, w)) df_out_kernel<<<g, 256, 0, s>>>(n, (const float*)w.px[c->k], w.top_lo, z);
  else copy_convert_kernel<float, double><<<g, 256, 0, s>>>(n, (const float*)w.px[c->k], z);
  return cudaGetLastError();
}

// the loop body on capture stream s
static cudaError_t cgd_body(Context* c, int inner, cudaGraphConditionalHandle h, cudaStream_t s) {
  const size_t n = (size_t)c->ndof;
  const int g = grid_for(n);
  const bool flexible = inner != HDG_PREC_FP64;
  const int outer = (inner == HDG_PREC_FP64) ? HDG_PREC_FP64 : HDG_PREC_F32X2;
  double* sc = c->scal;
  if (flexible) {
    copy_convert_kernel<double, double><<<g, 256, 0, s>>>(n, c->cg_z, c->cg_zold);
    HDG_CUDA_TRY(cudaGetLastError());
  }
  HDG_CUDA_TRY(vcycle_direct(c, inner, c->cg_r, c->cg_z, s));
  if (flexible) HDG_CUDA_TRY(dots<double>(c, n, c->cg_r, c->cg_z, c->cg_r, c->cg_zold, nullptr, nullptr, sc + 8, s));
  else HDG_CUDA_TRY(dots<double>(c, n, c->cg_r, c->cg_z, nullptr, nullptr, nullptr, nullptr, sc + 8, s));
  cgd_p_kernel<<<g, 256, 0, s>>>(n, sc, c->cg_ctl, c->cg_z, c->cg_p, flexible ? 1 : 0);
  HDG_CUDA_TRY(cudaGetLastError());
  cg_commit_kernel<<<1, 1, 0, s>>>(sc);
  HDG_CUDA_TRY(cudaGetLastError());
  HDG_CUDA_TRY(launch_apply(c, c->k, 0, outer, c->cg_p, nullptr, c->cg_q, 1.0, 0.0, 1, s));
  HDG_CUDA_TRY(dots<double>(c, n, c->cg_p, c->cg_q, nullptr, nullptr, nullptr, nullptr, sc + 1, s));
  cg_xr_kernel<<<g, 256, 0, s>>>(n, sc, c->cg_p, c->cg_q, c->cg_x, c->cg_r);
  HDG_CUDA_TRY(cudaGetLastError());
  HDG_CUDA_TRY(dots<double>(c, n, c->cg_r, c->cg_r, nullptr, nullptr, nullptr, nullptr, sc + 2, s));
  cgd_check_kernel<<<1, 1, 0, s>>>(sc, c->cg_ctl, c->cg_hist, h);
  return cudaGetLastError();
}

// graph: one WHILE node whose body is cgd_body (condition initially 1)
static cudaError_t build_cg_graph(Context* c, int inner, cudaGraphExec_t* out) {
  cudaGraph_t G = nullptr;
  HDG_CUDA_TRY(cudaGraphCreate(&G, 0));
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  cudaGraphConditionalHandle h;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, G, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams np = {};
  cudaGraphNode_t wn;
  if (e == cudaSuccess) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&wn, G, nullptr, nullptr, 0, &np);
  }
  if (e == cudaSuccess) {
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t eb = cgd_body(c, inner, h, cs);
      const cudaError_t ee = cudaStreamEndCapture(cs, &body);
      e = eb != cudaSuccess ? eb : ee;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, G, 0);
  cudaGraphDestroy(G);
  if (e == cudaSuccess) {
    // kernels of one V-cycle (hdg_info.vcycle_kernels): the cycle captured alone
    cudaGraph_t Gv = nullptr;
    VWork& w = c->w1[prec_double(inner) ? 0 : 1];
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t eb = vcycle_body_any(c, w, inner, cs);
      const cudaError_t ee = cudaStreamEndCapture(cs, &Gv);
      e = eb != cudaSuccess ? eb : ee;
    }
    size_t nn = 0;
    if (e == cudaSuccess) e = cudaGraphGetNodes(Gv, nullptr, &nn);
    if (e == cudaSuccess) {
      std::vector<cudaGraphNode_t> nodes(nn);
      e = cudaGraphGetNodes(Gv, nodes.data(), &nn);
      int nk = 0;
      for (size_t q = 0; q < nn && e == cudaSuccess; ++q) {
        cudaGraphNodeType ty;
        e = cudaGraphNodeGetType(nodes[q], &ty);
        if (ty == cudaGraphNodeTypeKernel) ++nk;
      }
      if (e == cudaSuccess) c->vcycle_kernels = nk;
    }
    if (Gv) cudaGraphDestroy(Gv);
  }
  if (cs) cudaStreamDestroy(cs);
  return e;
}

static int pcg_solve_impl(Context* c, const double* b, double* x, double rtol, int maxit, int inner,
                          hdg_solve_info* info, cudaStream_t s) {
  const size_t n = (size_t)c->ndof;
  const int g = grid_for(n);
  double* r = c->cg_r;
  double* z = c->cg_z;
  double* p = c->cg_p;
  double* q = c->cg_q;
  double* zold = c->cg_zold;
  double* sc = c->scal;
  double* h = c->h_scal;
  const bool flexible = inner != HDG_PREC_FP64;
  // plain FP64 mode applies FP64 blocks everywhere; the other modes compute the
  // outer residual with the double-float blocks (FP64 vectors, ~48-bit products)
  const int outer = (inner == HDG_PREC_FP64) ? HDG_PREC_FP64 : HDG_PREC_F32X2;
#define CK(expr) do { cudaError_t _e = (expr); if (_e != cudaSuccess) return HDG_ERR_CUDA; } while (0)
  CK(dots<double>(c, n, b, b, nullptr, nullptr, nullptr, nullptr, sc + 4, s));
  CK(cudaMemcpyAsync(h, sc + 4, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double bn = std::sqrt(h[0]);
  if (c->opt.fmg_start > 0 && bn > 0.0) {
    // start from one full multigrid cycle: x = FMG(b), r = b - A x
    const cudaError_t e = fmg_solve(c, b, x, c->opt.fmg_start, s);
    if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return HDG_ERR_OOM; }
    CK(e);
    CK(launch_apply(c, c->k, 0, outer, x, b, r, -1.0, 1.0, 1, s));
  } else {
    CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    CK(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  if (info) { info->iterations = 0; info->relres = 0.0; info->relres_history[0] = 1.0; }
  if (!(bn > 0.0)) {
    if (info) info->relres = 0.0;
    return (bn == 0.0) ? HDG_OK : HDG_ERR_INVALID_ARG;
  }
  if (x == c->cg_x && c->cg_graph[inner]) {
    // device-resident loop: one graph launch runs every iteration
    cgd_init_kernel<<<1, 1, 0, s>>>(sc, c->cg_ctl, rtol, maxit);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(z, 0, n * sizeof(double), s));
    CK(cudaGraphLaunch(c->cg_graph[inner], s));
    double* hc = c->h_cg;
    CK(cudaMemcpyAsync(hc, sc + 19, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hc + 1, c->cg_ctl, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hc + 8, c->cg_hist, 256 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int ctl[2];
    std::memcpy(ctl, hc + 1, sizeof(ctl));
    if (info) {
      info->iterations = ctl[0];
      info->relres = hc[0];
      for (int i = 1; i < 256 && i <= ctl[0]; ++i) info->relres_history[i] = hc[8 + i];
    }
    return ctl[1] < 0 ? HDG_ERR_CUDA : ctl[1];
  }
  CK(vcycle_typed(c, c->w1[prec_double(inner) ? 0 : 1], inner, r, z, true, s));
  CK(dots<double>(c, n, r, z, nullptr, nullptr, nullptr, nullptr, sc + 0, s));
  CK(cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  int it = 0;
  double rel = 1.0;
  int status = HDG_ERR_NOT_CONVERGED;
  for (it = 1; it <= maxit; ++it) {
    CK(launch_apply(c, c->k, 0, outer, p, nullptr, q, 1.0, 0.0, 1, s));
    CK(dots<double>(c, n, p, q, nullptr, nullptr, nullptr, nullptr, sc + 1, s));
    CK(cudaMemcpyAsync(h + 1, sc + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    cg_xr_kernel<<<g, 256, 0, s>>>(n, sc, p, q, x, r);
    CK(cudaGetLastError());
    CK(dots<double>(c, n, r, r, nullptr, nullptr, nullptr, nullptr, sc + 2, s));
    CK(cudaMemcpyAsync(h + 2, sc + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!(h[1] > 0.0) || !std::isfinite(h[1])) { status = HDG_ERR_BREAKDOWN; break; }
    rel = std::sqrt(h[2]) / bn;
    if (info && it < 256) info->relres_history[it] = rel;
    if (!std::isfinite(rel)) { status = HDG_ERR_BREAKDOWN; break; }
    if (rel <= rtol) { status = HDG_OK; break; }
    if (flexible) CK(cudaMemcpyAsync(zold, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(vcycle_typed(c, c->w1[prec_double(inner) ? 0 : 1], inner, r, z, true, s));
    if (flexible) CK(dots<double>(c, n, r, z, r, zold, nullptr, nullptr, sc + 8, s));
    else CK(dots<double>(c, n, r, z, nullptr, nullptr, nullptr, nullptr, sc + 8, s));
    cg_p_kernel<<<g, 256, 0, s>>>(n, sc, z, p, flexible ? 1 : 0);
    CK(cudaGetLastError());
    cg_commit_kernel<<<1, 1, 0, s>>>(sc);
    CK(cudaGetLastError());
  }
#undef CK
  if (it > maxit) it = maxit;
  if (info) { info->iterations = it; info->relres = rel; }
  return status;
}

// ---------------------------------------------------------------------------
// Several contexts' solves as one graph (hdg_solve_multi): per instance a
// chain prologue -> WHILE node (the body of the device-resident loop) ->
// epilogue, the chains independent, so one launch solves every instance and
// the GPU overlaps them. The prologue does on the device what pcg_solve's
// host part does (|b|, x = 0, r = b, z = 0, the control words); a zero b stops
// the loop before its first pass (condition 0, status OK, x = 0).
__global__ void cgd_init_multi_kernel(double* scal, int* ctl, double rtol, int maxit, cudaGraphConditionalHandle h) {
  const double bn = sqrt(scal[4]);
  scal[16] = rtol;
  scal[17] = bn;
  scal[19] = bn > 0.0 ? 1.0 : 0.0;
  ctl[0] = 0;
  ctl[1] = bn > 0.0 ? -1 : (bn == 0.0 ? HDG_OK : HDG_ERR_INVALID_ARG);
  ctl[2] = maxit;
  cudaGraphSetConditional(h, bn > 0.0 ? 1u : 0u);
}

// Adds instance c's chain to G (capture stream cs); solution to lambda.
cudaError_t cg_multi_add(Context* c, int inner, const double* b, double* lambda, double rtol, int maxit, cudaGraph_t G,
                         cudaStream_t cs) {
  if (!c->cg_x || !c->cg_ctl || !c->cg_hist || !c->h_cg) return cudaErrorInvalidValue;
  const size_t n = (size_t)c->ndof;
  const int g = grid_for(n);
  cudaGraphConditionalHandle h;
  HDG_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, G, 1, cudaGraphCondAssignDefault));
  // prologue
  HDG_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, G, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = dots<double>(c, n, b, b, nullptr, nullptr, nullptr, nullptr, c->scal + 4, cs);
  if (e == cudaSuccess) {
    cgd_init_multi_kernel<<<1, 1, 0, cs>>>(c->scal, c->cg_ctl, rtol, maxit, h);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = vec_fill(c->cg_x, HDG_PREC_FP64, n, cs);
  if (e == cudaSuccess) e = vec_fill(c->cg_z, HDG_PREC_FP64, n, cs);
  if (e == cudaSuccess) {
    copy_convert_kernel<double, double><<<g, 256, 0, cs>>>(n, b, c->cg_r);
    e = cudaGetLastError();
  }
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edata = nullptr;
  size_t ndeps = 0;
  std::vector<cudaGraphNode_t> dv;
  if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, &edata, &ndeps);
  if (e == cudaSuccess) dv.assign(deps, deps + ndeps);
  cudaGraph_t Gout = G;
  const cudaError_t ee = cudaStreamEndCapture(cs, &Gout);
  HDG_CUDA_TRY(e);
  HDG_CUDA_TRY(ee);
  // the loop
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t wn;
  HDG_CUDA_TRY(cudaGraphAddNode(&wn, G, dv.data(), nullptr, dv.size(), &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  HDG_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  e = cgd_body(c, inner, h, cs);
  const cudaError_t eb = cudaStreamEndCapture(cs, &body);
  HDG_CUDA_TRY(e);
  HDG_CUDA_TRY(eb);
  // epilogue
  HDG_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, G, &wn, nullptr, 1, cudaStreamCaptureModeThreadLocal));
  copy_convert_kernel<double, double><<<g, 256, 0, cs>>>(n, c->cg_x, lambda);
  e = cudaGetLastError();
  Gout = G;
  const cudaError_t e2 = cudaStreamEndCapture(cs, &Gout);
  HDG_CUDA_TRY(e);
  return e2;
}

// After the graph: copies of instance c's results to its pinned buffer (stream s)
cudaError_t cg_multi_fetch(Context* c, cudaStream_t s) {
  double* hc = c->h_cg;
  HDG_CUDA_TRY(cudaMemcpyAsync(hc, c->scal + 19, sizeof(double), cudaMemcpyDeviceToHost, s));
  HDG_CUDA_TRY(cudaMemcpyAsync(hc + 1, c->cg_ctl, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  return cudaMemcpyAsync(hc + 8, c->cg_hist, 256 * sizeof(double), cudaMemcpyDeviceToHost, s);
}
// ... and, once they have arrived, the status and the solve information
int cg_multi_result(Context* c, hdg_solve_info* info) {
  const double* hc = c->h_cg;
  int ctl[2];
  std::memcpy(ctl, hc + 1, sizeof(ctl));
  if (info) {
    info->iterations = ctl[0];
    info->relres = hc[0];
    info->relres_history[0] = 1.0;
    for (int i = 1; i < 256 && i <= ctl[0]; ++i) info->relres_history[i] = hc[8 + i];
  }
  return ctl[1] < 0 ? HDG_ERR_CUDA : ctl[1];
}

// One right-hand side: with CUDA graphs on, the device-resident loop (its
// buffers made at set-up, its graph on first use per inner precision; the host
// loop where conditional graph nodes are not available), iterating in cg_x and
// copied to x at the end.
int pcg_solve(Context* c, const double* b, double* x, double rtol, int maxit, int inner, hdg_solve_info* info,
              cudaStream_t s) {
  if (!c->opt.use_graphs || c->cg_graph_failed || !c->cg_x || !c->h_cg)
    return pcg_solve_impl(c, b, x, rtol, maxit, inner, info, s);
  if (!c->cg_graph[inner]) {
    const cudaError_t e = build_cg_graph(c, inner, &c->cg_graph[inner]);
    if (e != cudaSuccess) {
      // conditional nodes unavailable (driver): keep the host loop from now on
      cudaGetLastError();
      c->cg_graph[inner] = nullptr;
      c->cg_graph_failed = true;
      return pcg_solve_impl(c, b, x, rtol, maxit, inner, info, s);
    }
  }
  const int st = pcg_solve_impl(c, b, c->cg_x, rtol, maxit, inner, info, s);
  if (cudaMemcpyAsync(x, c->cg_x, (size_t)c->ndof * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return HDG_ERR_CUDA;
  return st;
}

// ---------------------------------------------------------------------------
// Batched CG: nb right-hand sides, vectors [n][nb], per-column scalars in
// sc[slot * nb + col]:
//   0 rz  1 pq  2 rr (first: bb)  3 r.zold  4 |b|  5 relres  6 active  7 breakdown
//   8 rz_new  9 alpha  10 beta
enum { kRz = 0, kPq, kRr, kRzOld, kBn, kRel, kAct, kErr, kRzNew, kAlpha, kBeta };

// per-column dot products of [n][nb] arrays (deterministic: fixed grid, fixed
// order): part[(q * gridDim.x + block) * nb + col]
__global__ void cdots_kernel(size_t n, int nb, const double* __restrict__ a0, const double* __restrict__ b0,
                             const double* __restrict__ a1, const double* __restrict__ b1,
                             double* __restrict__ part) {
  __shared__ double sh[2][256];
  const int cw = nb < 256 ? nb : 256;
  const int rl = 256 / cw;
  const int lc = threadIdx.x % cw, rowl = threadIdx.x / cw;
  for (int col0 = 0; col0 < nb; col0 += cw) {
    const int col = col0 + lc;
    double s0 = 0.0, s1 = 0.0;
    if (rowl < rl && col < nb) {
      // four independent partial sums (loads in flight), combined in a fixed order
      double p0[4] = {0.0, 0.0, 0.0, 0.0}, p1[4] = {0.0, 0.0, 0.0, 0.0};
      const size_t step = (size_t)gridDim.x * rl;
      size_t i = (size_t)blockIdx.x * rl + rowl;
      for (; i + 3 * step < n; i += 4 * step) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const size_t o = (i + u * step) * nb + col;
          p0[u] += a0[o] * b0[o];
          if (a1) p1[u] += a1[o] * b1[o];
        }
      }
      for (; i < n; i += step) {
        const size_t o = i * nb + col;
        p0[0] += a0[o] * b0[o];
        if (a1) p1[0] += a1[o] * b1[o];
      }
      s0 = (p0[0] + p0[1]) + (p0[2] + p0[3]);
      s1 = (p1[0] + p1[1]) + (p1[2] + p1[3]);
    }
    sh[0][threadIdx.x] = s0;
    sh[1][threadIdx.x] = s1;
    __syncthreads();
    if (rowl == 0 && col < nb) {
      double t0 = 0.0, t1 = 0.0;
      for (int q = 0; q < rl; ++q) { t0 += sh[0][q * cw + lc]; t1 += sh[1][q * cw + lc]; }
      part[(size_t)blockIdx.x * nb + col] = t0;
      part[((size_t)gridDim.x + blockIdx.x) * nb + col] = t1;
    }
    __syncthreads();
  }
}
// one warp per column: lanes take every 32nd partial, then a fixed shuffle tree
__global__ void cdots_finalize_kernel(int nb, int nblk, const double* __restrict__ part, double* __restrict__ out0,
                                      double* __restrict__ out1) {
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (col >= nb) return;
  double t0 = 0.0, t1 = 0.0;
  for (int b = lane; b < nblk; b += 32) {
    t0 += part[(size_t)b * nb + col];
    if (out1) t1 += part[((size_t)nblk + b) * nb + col];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    t0 += __shfl_xor_sync(0xffffffffu, t0, o);
    t1 += __shfl_xor_sync(0xffffffffu, t1, o);
  }
  if (lane == 0) {
    out0[col] = t0;
    if (out1) out1[col] = t1;
  }
}
static cudaError_t cdots(VWork* w, size_t n, const double* a0, const double* b0, const double* a1,
                         const double* b1, double* out0, double* out1, cudaStream_t s) {
  cdots_kernel<<<kColRedBlocks, 256, 0, s>>>(n, w->nb, a0, b0, a1, b1, w->cg_part);
  HDG_CUDA_TRY(cudaGetLastError());
  cdots_finalize_kernel<<<(w->nb + 7) / 8, 256, 0, s>>>(w->nb, kColRedBlocks, w->cg_part, out0, out1);
  return cudaGetLastError();
}

__global__ void cgb_init_kernel(int nb, double* __restrict__ sc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const double bn = sqrt(sc[kRr * nb + j]);
  sc[kBn * nb + j] = bn;
  sc[kAct * nb + j] = bn > 0.0 ? 1.0 : 0.0;
  sc[kRel * nb + j] = bn > 0.0 ? 1.0 : 0.0;
  sc[kErr * nb + j] = 0.0;
  sc[kAlpha * nb + j] = 0.0;
  sc[kBeta * nb + j] = 0.0;
}
__global__ void cgb_alpha_kernel(int nb, double* __restrict__ sc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  double a = 0.0;
  if (sc[kAct * nb + j] != 0.0) {
    const double pq = sc[kPq * nb + j];
    if (pq > 0.0 && isfinite(pq)) {
      a = sc[kRz * nb + j] / pq;
    } else {
      sc[kErr * nb + j] = 1.0;
      sc[kAct * nb + j] = 0.0;
    }
  }
  sc[kAlpha * nb + j] = a;
}
__global__ void cgb_xr_kernel(size_t n, int nb, const double* __restrict__ sc, const double* __restrict__ p,
                              const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r) {
  const double* al = sc + kAlpha * nb;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int col;
    (void)divmod(t, nb, &col);
    const double a = al[col];
    if (a != 0.0) {
      x[t] += a * p[t];
      r[t] -= a * q[t];
    }
  }
}
__global__ void cgb_status_kernel(int nb, double* __restrict__ sc, double rtol) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  if (sc[kAct * nb + j] == 0.0) return;
  const double rel = sqrt(sc[kRr * nb + j]) / sc[kBn * nb + j];
  sc[kRel * nb + j] = rel;
  if (!isfinite(rel)) { sc[kErr * nb + j] = 1.0; sc[kAct * nb + j] = 0.0; }
  else if (rel <= rtol) sc[kAct * nb + j] = 0.0;
}
__global__ void cgb_beta_kernel(int nb, double* __restrict__ sc, int flexible) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  double b = 0.0;
  if (sc[kAct * nb + j] != 0.0) {
    const double rzn = sc[kRzNew * nb + j];
    b = (flexible ? rzn - sc[kRzOld * nb + j] : rzn) / sc[kRz * nb + j];
    sc[kRz * nb + j] = rzn;
  }
  sc[kBeta * nb + j] = b;
}
__global__ void cgb_p_kernel(size_t n, int nb, const double* __restrict__ sc, const double* __restrict__ z,
                             double* __restrict__ p) {
  const double* act = sc + kAct * nb;
  const double* be = sc + kBeta * nb;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    int j;
    (void)divmod(t, nb, &j);
    if (act[j] != 0.0) p[t] = z[t] + be[j] * p[t];
  }
}

int pcg_solve_batched(Context* c, const double* b, double* x, int nb, double rtol, int maxit, int inner,
                      hdg_solve_info* info, cudaStream_t s) {
  VWork* w = nullptr;
  if (batched_work(c, nb, prec_double(inner), &w) != cudaSuccess) return HDG_ERR_OOM;
  if (work_cg(c, w) != cudaSuccess) return HDG_ERR_OOM;
  set_cols_scratch(c, w);
  const size_t n = (size_t)c->ndof * nb;
  const int g = grid_for(n);
  const int gs = (nb + 255) / 256;
  double *r = w->cg_r, *z = w->cg_z, *p = w->cg_p, *q = w->cg_q, *zold = w->cg_zold, *sc = w->cg_sc;
  double* h = w->h_sc;
  const bool flexible = inner != HDG_PREC_FP64;
  const int outer = (inner == HDG_PREC_FP64) ? HDG_PREC_FP64 : HDG_PREC_F32X2;
  const bool use_tc = c->opt.tensor_apply && c->oz_B && nb % 64 == 0 && nb <= 2048;
  auto S = [&](int slot) { return sc + (size_t)slot * nb; };
#define CK(expr) do { cudaError_t _e = (expr); if (_e != cudaSuccess) return HDG_ERR_CUDA; } while (0)
  CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  CK(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cdots(w, (size_t)c->ndof, b, b, nullptr, nullptr, S(kRr), nullptr, s));
  cgb_init_kernel<<<gs, 256, 0, s>>>(nb, sc);
  CK(cudaGetLastError());
  CK(vcycle_typed(c, *w, inner, r, z, true, s));
  CK(cdots(w, (size_t)c->ndof, r, z, nullptr, nullptr, S(kRz), nullptr, s));
  CK(cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (info) { info->iterations = 0; info->relres = 0.0; info->relres_history[0] = 1.0; }
  int it = 0;
  double relmax = 0.0;
  int status = HDG_ERR_NOT_CONVERGED;
  for (it = 1; it <= maxit; ++it) {
    // the outer operator on the tensor cores (FP64 by exact slice splitting) when
    // every element shares one block and the columns come in groups of 64
    if (use_tc) CK(launch_ozaki_apply(c, p, q, nb, s));
    else CK(launch_apply(c, c->k, 0, outer, p, nullptr, q, 1.0, 0.0, nb, s));
    CK(cdots(w, (size_t)c->ndof, p, q, nullptr, nullptr, S(kPq), nullptr, s));
    cgb_alpha_kernel<<<gs, 256, 0, s>>>(nb, sc);
    CK(cudaGetLastError());
    cgb_xr_kernel<<<g, 256, 0, s>>>(n, nb, sc, p, q, x, r);
    CK(cudaGetLastError());
    CK(cdots(w, (size_t)c->ndof, r, r, nullptr, nullptr, S(kRr), nullptr, s));
    cgb_status_kernel<<<gs, 256, 0, s>>>(nb, sc, rtol);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h, S(kRel), 3 * (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    relmax = 0.0;
    int active = 0, err = 0;
    for (int j = 0; j < nb; ++j) {
      relmax = std::max(relmax, h[j]);
      active += h[nb + j] != 0.0;
      err += h[2 * nb + j] != 0.0;
    }
    if (info && it < 256) info->relres_history[it] = relmax;
    if (err) { status = HDG_ERR_BREAKDOWN; break; }
    if (active == 0) { status = HDG_OK; break; }
    if (it == maxit) break;
    if (flexible) CK(cudaMemcpyAsync(zold, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(vcycle_typed(c, *w, inner, r, z, true, s));
    if (flexible) CK(cdots(w, (size_t)c->ndof, r, z, r, zold, S(kRzNew), S(kRzOld), s));
    else CK(cdots(w, (size_t)c->ndof, r, z, nullptr, nullptr, S(kRzNew), nullptr, s));
    cgb_beta_kernel<<<gs, 256, 0, s>>>(nb, sc, flexible ? 1 : 0);
    CK(cudaGetLastError());
    cgb_p_kernel<<<g, 256, 0, s>>>(n, nb, sc, z, p);
    CK(cudaGetLastError());
  }
#undef CK
  if (it > maxit) it = maxit;
  if (info) { info->iterations = it; info->relres = relmax; }
  return status;
}

}  // namespace hdg
