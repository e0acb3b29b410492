// Device code of the reduced-block apply shared by the one-mesh launches
// (apply_reduced.cu, where the method is described) and the one-launch apply
// over several meshes (apply_multi.cu).
#pragma once
#include "apply_impl.cuh"

namespace hdg {
namespace red {

// Double-float arithmetic for the reduced product of the double-vector
// (F32X2) applies: a value is hi + lo (two floats, lo below half an ulp of hi
// after every operation), products are split exactly by an FMA and sums by
// Knuth's two-sum, so the element product keeps about 46 significant bits on
// the FP32 pipe (the FP64 pipe of this GPU is ~60x slower). Blocks are float2
// pairs (hi, lo) of the FP64 reduced blocks; vectors stay double.
struct dd {
  float hi, lo;
  __device__ __forceinline__ dd() {}
  __device__ __forceinline__ explicit dd(int v) : hi((float)v), lo(0.0f) {}
  __device__ __forceinline__ explicit dd(float v) : hi(v), lo(0.0f) {}
  __device__ __forceinline__ dd(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ dd(float2 v) : hi(v.x), lo(v.y) {}
};
__device__ __forceinline__ dd dd_norm(float s, float l) {
  const float h = __fadd_rn(s, l);
  return dd(h, __fsub_rn(l, __fsub_rn(h, s)));
}
__device__ __forceinline__ dd operator+(dd a, dd b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bv = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bv)), __fsub_rn(b.hi, bv));
  return dd_norm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + dd(-b.hi, -b.lo); }
// u + b t in each arithmetic (named apart from fma so that double and float
// calls inside this namespace never meet the double-float overload)
__device__ __forceinline__ double madd(double b, double t, double u) { return ::fma(b, t, u); }
__device__ __forceinline__ float madd(float b, float t, float u) { return fmaf(b, t, u); }
__device__ __forceinline__ dd madd(dd b, dd t, dd u) {
  const float p = __fmul_rn(b.hi, t.hi);
  float e = __fmaf_rn(b.hi, t.hi, -p);
  e = __fmaf_rn(b.hi, t.lo, e);
  e = __fmaf_rn(b.lo, t.hi, e);
  const float s = __fadd_rn(u.hi, p);
  const float bv = __fsub_rn(s, u.hi);
  const float e2 = __fadd_rn(__fsub_rn(u.hi, __fsub_rn(s, bv)), __fsub_rn(p, bv));
  return dd_norm(s, __fadd_rn(u.lo, __fadd_rn(e, e2)));
}
// vector entries in the arithmetic type: double vectors are split into
// (hi, lo) with integer operations for the double-float product
template <typename T>
__device__ __forceinline__ T vload(const void* v, size_t i) { return __ldg((const T*)v + i); }
template <>
__device__ __forceinline__ dd vload<dd>(const void* v, size_t i) {
  const dfloat f = split_double(__ldg((const double*)v + i));
  return dd(f.hi, f.lo);
}
// the vector type of an arithmetic type, and the conversion of a result
template <typename T> struct VecT { using type = T; };
template <> struct VecT<dd> { using type = double; };
template <typename T>
__device__ __forceinline__ T to_vec(T a) { return a; }
__device__ __forceinline__ double to_vec(dd a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

template <int N1>
struct Red {
  static constexpr int se = N1 / 2 + (N1 & 1), so = N1 / 2;                 // even / odd node parts
  static constexpr int d0 = 2 * se, d1 = so + se, d2 = se + so, d3 = 2 * so;   // block dimensions
  static constexpr int q0 = 0, q1 = d0 * (d0 + 1) / 2, q2 = q1 + d1 * (d1 + 1) / 2, q3 = q2 + d2 * (d2 + 1) / 2;
  static constexpr int Q = q3 + d3 * (d3 + 1) / 2;                            // entries per element
};

// Block layout: warp-sized chunks, entry q of element K at
// [((K / 32) * Q + q) * 32 + K % 32] — the 32 consecutive elements of a warp
// read entry q as one 128 / 256-byte run, and all of a warp's entries form one
// contiguous chunk (Q runs in a row, so DRAM pages are read sequentially).
__device__ __forceinline__ size_t red_base(long K, int Q) { return ((size_t)(K >> 5) * Q) * 32 + (K & 31); }

// FP32 blocks: the same chunks in groups of four entries, entry q of element K
// at [((K / 32) * ceil(Q / 4) + q / 4) * 128 + (K % 32) * 4 + q % 4], so a
// thread reads its entries as float4 (one 512-byte run per warp and group) and
// has ceil(Q/4) wide loads in flight before any arithmetic
__host__ __device__ constexpr int red_groups(int Q) { return (Q + 3) / 4; }
__device__ __forceinline__ size_t red_index32(long K, int Q, int q) {
  return ((size_t)(K >> 5) * red_groups(Q) + (q >> 2)) * 128 + (K & 31) * 4 + (q & 3);
}

// u = B t for one block whose entries are already in registers (bq: the
// element's entries from the block's first on)
template <int D, typename T>
__device__ __forceinline__ void sym_block_reg(const float* bq, const T (&t)[D > 0 ? D : 1], T (&u)[D > 0 ? D : 1]) {
#pragma unroll
  for (int i = 0; i < D; ++i) u[i] = T(0);
  int q = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int j = i; j < D; ++j, ++q) {
      const T b = (T)bq[q];
      if (j == i) {
        u[i] = madd(b, t[i], u[i]);
      } else {
        u[i] = madd(b, t[j], u[i]);
        u[j] = madd(b, t[i], u[j]);
      }
    }
  }
}

// u = B t for one symmetric block of dimension D stored as a packed upper
// triangle (row-major) from entry qoff on (base = red_base(K, Q))
template <int D, typename T, typename TS>
__device__ __forceinline__ void sym_block(const TS* __restrict__ R, int qoff, size_t base, const T (&t)[D > 0 ? D : 1],
                                          T (&u)[D > 0 ? D : 1]) {
#pragma unroll
  for (int i = 0; i < D; ++i) u[i] = T(0);
  int q = qoff;
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int j = i; j < D; ++j, ++q) {
      const T b = (T)__ldcs(R + base + (size_t)q * 32);
      if (j == i) {
        u[i] = madd(b, t[i], u[i]);
      } else {
        u[i] = madd(b, t[j], u[i]);
        u[j] = madd(b, t[i], u[j]);
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
  const void* R;       // reduced blocks in warp chunks (type TS; see red_base / red_index32)
  const void* v;       // input vector (type T)
  const void* cvec;    // addend or nullptr
  void* y;             // output
  void* z;             // element products [4 n1][nel] (type T)
  double alpha, beta;
  int nx, ny;
};

// z_K = S_K v_K for element K = (i, j) by the reduced product; the four face
// outputs in zw, ze, zs, zn (boundary faces of v read as zero)
// (v: column `col` of nb right-hand sides stored right-hand side fastest)
template <int N1, typename TS, typename T, bool DIFF>
__device__ __forceinline__ void elem_product(const RedArgs& a, long nel, long K, int i, int j, T (&zw)[N1],
                                             T (&ze)[N1], T (&zs)[N1], T (&zn)[N1], int nb = 1, int col = 0) {
  using RD = Red<N1>;
  constexpr int se = RD::se, so = RD::so;
  // FP32 blocks: every entry of the element loaded first, as float4
  constexpr bool kVec = sizeof(TS) == 4;
  constexpr int G = kVec ? red_groups(RD::Q) : 1;
  float bq[4 * G];
  if constexpr (kVec) {
    const float4* __restrict__ R4 = (const float4*)a.R;
    const size_t g0 = ((size_t)(K >> 5) * G) * 32 + (K & 31);
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const float4 w = __ldcs(R4 + g0 + (size_t)g * 32);
      bq[4 * g] = w.x; bq[4 * g + 1] = w.y; bq[4 * g + 2] = w.z; bq[4 * g + 3] = w.w;
    }
  }
  const int nx = a.nx, ny = a.ny;
  const void* v = a.v;
  const long eW = i + (long)(nx + 1) * j, eS = (long)(nx + 1) * ny + i + (long)nx * j;
  const bool hW = i > 0, hE = i < nx - 1, hS = j > 0, hN = j < ny - 1;
  T xw[N1], xe[N1], xs[N1], xn[N1];
#pragma unroll
  for (int q = 0; q < N1; ++q) {
    xw[q] = hW ? vload<T>(v, (eW * N1 + q) * nb + col) : T(0);
    xe[q] = hE ? vload<T>(v, ((eW + 1) * N1 + q) * nb + col) : T(0);
    xs[q] = hS ? vload<T>(v, (eS * N1 + q) * nb + col) : T(0);
    xn[q] = hN ? vload<T>(v, ((eS + nx) * N1 + q) * nb + col) : T(0);
  }
  if constexpr (DIFF) {   // S_K has zero row sums: apply it to v_K - mean(v_K)
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
  if constexpr (kVec) {
    sym_block_reg<RD::d0, T>(bq + RD::q0, t0, u0);
    sym_block_reg<RD::d1, T>(bq + RD::q1, t1, u1);
    sym_block_reg<RD::d2, T>(bq + RD::q2, t2, u2);
    sym_block_reg<RD::d3, T>(bq + RD::q3, t3, u3);
  } else {
    const size_t base = red_base(K, RD::Q);
    sym_block<RD::d0, T>(R, RD::q0, base, t0, u0);
    sym_block<RD::d1, T>(R, RD::q1, base, t1, u1);
    sym_block<RD::d2, T>(R, RD::q2, base, t2, u2);
    sym_block<RD::d3, T>(R, RD::q3, base, t3, u3);
  }
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
#pragma unroll
  for (int q = 0; q < N1; ++q) {
    zw[q] = Po[q] + Mo[q];
    ze[q] = Po[q] - Mo[q];
    zs[q] = Ppo[q] + Mpo[q];
    zn[q] = Ppo[q] - Mpo[q];
  }
}

// epilogue y = beta c + alpha s; y = A v, y = c - A v and y = c + A v take no
// multiply (FP64 operations are slow on this GPU)
template <typename T>
struct Form {
  int f;
  T al, be;
  const T* __restrict__ cv;
  __device__ __forceinline__ Form(const RedArgs& a) : al((T)a.alpha), be((T)a.beta), cv((const T*)a.cvec) {
    f = (al == T(1) && (!cv || be == T(0))) ? 0
        : (cv && be == T(1) && al == T(-1)) ? 1 : (cv && be == T(1) && al == T(1)) ? 2 : 3;
  }
  __device__ __forceinline__ T operator()(T s, size_t o) const {
    if (f == 0) return s;
    if (f == 1) return cv[o] - s;
    if (f == 2) return cv[o] + s;
    T val = al * s;
    if (cv) val = fma(be, cv[o], val);
    return val;
  }
  // the same with the addend c already loaded (any value when cv is null)
  __device__ __forceinline__ T with(T s, T c) const {
    if (f == 0) return s;
    if (f == 1) return c - s;
    if (f == 2) return c + s;
    T val = al * s;
    if (cv) val = fma(be, c, val);
    return val;
  }
};

// Pass 1 of the two-launch form for element K: z_K = S_K v_K into the scratch.
template <int N1, typename TS, typename T, bool DIFF>
__device__ __forceinline__ void elem_body(const RedArgs& a, long K) {
  const int nx = a.nx, ny = a.ny;
  const long nel = (long)nx * ny;
  if (K >= nel) return;
  const int i = (int)(K % nx), j = (int)(K / nx);
  T zw[N1], ze[N1], zs[N1], zn[N1];
  elem_product<N1, TS, T, DIFF>(a, nel, K, i, j, zw, ze, zs, zn);
  T* __restrict__ z = (T*)a.z;
#pragma unroll
  for (int q = 0; q < N1; ++q) {
    z[(size_t)(0 * N1 + q) * nel + K] = zw[q];
    z[(size_t)(1 * N1 + q) * nel + K] = ze[q];
    z[(size_t)(2 * N1 + q) * nel + K] = zs[q];
    z[(size_t)(3 * N1 + q) * nel + K] = zn[q];
  }
}

constexpr int kElemThreads = 128, kFaceThreads = 256;

// Pass 2 for the kFaceThreads elements from K0 (t = thread index; every
// thread of the CTA calls it): each owned face from its two contributions.
// The face sums are staged in shared memory (sw, ss: kFaceThreads * N1 each)
// so that y (and the addend) are then written / read in dof order: the W (and
// S) edges of consecutive elements of a row are consecutive, so each warp
// store is one contiguous run instead of 32 runs of n1 values.
template <int N1, typename T>
__device__ __forceinline__ void face_body(const RedArgs& a, long K0, int t, T* sw, T* ss) {
  const int nx = a.nx, ny = a.ny;
  const long nel = (long)nx * ny;
  const long K = K0 + t;
  using VT = typename VecT<T>::type;
  const T* __restrict__ z = (const T*)a.z;
  VT* __restrict__ y = (VT*)a.y;
  const long nv = (long)(nx + 1) * ny;
  if (K < nel) {
    const int i = (int)(K % nx), j = (int)(K / nx);
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      sw[t * N1 + q] = i > 0 ? z[(size_t)(0 * N1 + q) * nel + K] + z[(size_t)(1 * N1 + q) * nel + K - 1] : T(0);
      ss[t * N1 + q] = j > 0 ? z[(size_t)(2 * N1 + q) * nel + K] + z[(size_t)(3 * N1 + q) * nel + K - nx] : T(0);
    }
    // the E / N domain-boundary edges have no owner element: zero them here
    if (i == nx - 1) {
#pragma unroll
      for (int q = 0; q < N1; ++q) y[(i + 1 + (long)(nx + 1) * j) * N1 + q] = VT(0);
    }
    if (j == ny - 1) {
#pragma unroll
      for (int q = 0; q < N1; ++q) y[(nv + i + (long)nx * (j + 1)) * N1 + q] = VT(0);
    }
  }
  __syncthreads();
  const Form<VT> form(a);
  const int cnt = (int)((nel - K0) < kFaceThreads ? (nel - K0) : kFaceThreads);
  // every thread has at most N1 outputs of each face type: their addends are
  // all loaded before the first store, so the loads overlap
  size_t ow[N1], os[N1];
  bool hw[N1], hs[N1];
  VT cw[N1], cs[N1];
#pragma unroll
  for (int u = 0; u < N1; ++u) {
    const int idx = t + u * kFaceThreads;
    hw[u] = false;
    hs[u] = false;
    ow[u] = os[u] = 0;
    cw[u] = cs[u] = VT(0);
    if (idx < cnt * N1) {
      const int tt = idx / N1, q = idx - tt * N1;
      const long Kt = K0 + tt;
      const int i = (int)(Kt % nx), j = (int)(Kt / nx);
      ow[u] = (size_t)(i + (long)(nx + 1) * j) * N1 + q;
      os[u] = (size_t)(nv + i + (long)nx * j) * N1 + q;
      hw[u] = i > 0;
      hs[u] = j > 0;
      if (form.cv) {
        cw[u] = form.cv[ow[u]];
        cs[u] = form.cv[os[u]];
      }
    }
  }
#pragma unroll
  for (int u = 0; u < N1; ++u) {
    const int idx = t + u * kFaceThreads;
    if (idx < cnt * N1) {
      y[ow[u]] = hw[u] ? form.with(to_vec(sw[idx]), cw[u]) : VT(0);
      y[os[u]] = hs[u] ? form.with(to_vec(ss[idx]), cs[u]) : VT(0);
    }
  }
}

// Many right-hand sides (v, y: [ndof][nb], right-hand side fastest): element K
// and column col per thread, a warp over 32 consecutive columns of one element
// (the block entries it reads are the same for the whole warp: one broadcast
// load each, reused by 32 columns). Scratch z: [4 n1][nel][nb].
template <int N1, typename TS, typename T, bool DIFF>
__device__ __forceinline__ void cols_elem_body(const RedArgs& a, long K, int nb, int col) {
  const int nx = a.nx, ny = a.ny;
  const long nel = (long)nx * ny;
  if (K >= nel || col >= nb) return;
  const int i = (int)(K % nx), j = (int)(K / nx);
  T zw[N1], ze[N1], zs[N1], zn[N1];
  elem_product<N1, TS, T, DIFF>(a, nel, K, i, j, zw, ze, zs, zn, nb, col);
  T* __restrict__ z = (T*)a.z;
#pragma unroll
  for (int q = 0; q < N1; ++q) {
    z[((size_t)(0 * N1 + q) * nel + K) * nb + col] = zw[q];
    z[((size_t)(1 * N1 + q) * nel + K) * nb + col] = ze[q];
    z[((size_t)(2 * N1 + q) * nel + K) * nb + col] = zs[q];
    z[((size_t)(3 * N1 + q) * nel + K) * nb + col] = zn[q];
  }
}

template <int N1, typename T>
__device__ __forceinline__ void cols_face_body(const RedArgs& a, long K, int nb, int col) {
  const int nx = a.nx, ny = a.ny;
  const long nel = (long)nx * ny;
  if (K >= nel || col >= nb) return;
  const int i = (int)(K % nx), j = (int)(K / nx);
  using VT = typename VecT<T>::type;
  const T* __restrict__ z = (const T*)a.z;
  VT* __restrict__ y = (VT*)a.y;
  const Form<VT> form(a);
  const long nv = (long)(nx + 1) * ny;
  const long eW = i + (long)(nx + 1) * j, eS = nv + i + (long)nx * j;
#pragma unroll
  for (int q = 0; q < N1; ++q) {
    const size_t ow = (size_t)(eW * N1 + q) * nb + col, os = (size_t)(eS * N1 + q) * nb + col;
    y[ow] = i > 0 ? form(to_vec(z[((size_t)(0 * N1 + q) * nel + K) * nb + col] +
                                z[((size_t)(1 * N1 + q) * nel + K - 1) * nb + col]), ow)
                  : VT(0);
    y[os] = j > 0 ? form(to_vec(z[((size_t)(2 * N1 + q) * nel + K) * nb + col] +
                                z[((size_t)(3 * N1 + q) * nel + K - nx) * nb + col]), os)
                  : VT(0);
    if (i == nx - 1) y[((eW + 1) * N1 + q) * nb + col] = VT(0);
    if (j == ny - 1) y[((eS + nx) * N1 + q) * nb + col] = VT(0);
  }
}

}  // namespace red
}  // namespace hdg
