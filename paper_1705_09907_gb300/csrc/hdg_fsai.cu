// Factorized sparse approximate inverse (FSAI) smoother of Sec. 6.4.1 for the
// p-levels: M = G^T G ~ A^-1, G lower triangular on the pattern of the
// assembled p-level operator A (interior trace dofs in global order, dof =
// edge * (p+1) + a), each row normalised so that G A G^T has a unit diagonal.
// A smoothing step is x += G^T G (f - A x).
//
// Pattern of a row (edge e, node a): the columns of A in the row that are <= it
// are the nodes 0..a of e itself and every node of the interior edges of e's
// two elements that are numbered before e. Vertical edges come first in the
// numbering, so
//   vertical e = v(i, j):   slots (v(i-1, j), self)
//   horizontal e = h(i, j): slots (v(i, j-1), v(i+1, j-1), v(i, j), v(i+1, j),
//                                  h(i, j-1), self)
// (a slot whose edge is on the boundary or off the mesh is empty). G is stored
// per row edge and slot as dense (p+1) x (p+1) blocks, [edge][slot][a][b],
// vertical rows with 2 slots, horizontal rows with 6; entries of empty slots
// and of self-slot columns b > a are 0.
//
// Set-up (one warp per row): A[J, J] is summed from the element blocks S_K of
// the level, Cholesky-factored (A[J, J] = L L^T), and since i is the last index
// of J the normalised row is G[i, J] = L^-T e_last (A g = e_i gives g =
// L^-T e_last / L_nn and g_i = 1 / L_nn^2).
// Apply: w = G t (one thread per row dof and column), then z = c + G^T w (one
// thread per column dof and column, summing over the rows that hold it in a
// fixed order): each output written once, no atomics.
#include "hdg_internal.h"

namespace hdg {

namespace {

constexpr int kFsaiVSlots = 2, kFsaiHSlots = 6;

struct FsaiMesh {
  int nx, ny, n1;
  __device__ __forceinline__ int nv() const { return (nx + 1) * ny; }
  __device__ __forceinline__ int vedge(int i, int j) const { return i + (nx + 1) * j; }
  __device__ __forceinline__ int hedge(int i, int j) const { return nv() + i + nx * j; }
  // interior vertical / horizontal edges (the trace is zero on the others)
  __device__ __forceinline__ bool vin(int i, int j) const { return i >= 1 && i <= nx - 1 && j >= 0 && j < ny; }
  __device__ __forceinline__ bool hin(int i, int j) const { return j >= 1 && j <= ny - 1 && i >= 0 && i < nx; }
  // edge of slot s of row edge e (-1: empty); rows on the boundary have none
  __device__ __forceinline__ int slot_edge(int e, int s) const {
    if (e < nv()) {
      const int i = e % (nx + 1), j = e / (nx + 1);
      if (!vin(i, j)) return -1;
      if (s == 0) return vin(i - 1, j) ? vedge(i - 1, j) : -1;
      return e;
    }
    const int hh = e - nv(), i = hh % nx, j = hh / nx;
    if (!hin(i, j)) return -1;
    switch (s) {
      case 0: return vin(i, j - 1) ? vedge(i, j - 1) : -1;
      case 1: return vin(i + 1, j - 1) ? vedge(i + 1, j - 1) : -1;
      case 2: return vin(i, j) ? vedge(i, j) : -1;
      case 3: return vin(i + 1, j) ? vedge(i + 1, j) : -1;
      case 4: return hin(i, j - 1) ? hedge(i, j - 1) : -1;
      default: return e;
    }
  }
  // the (up to two) elements of an edge with the edge's face in each
  __device__ __forceinline__ int edge_elems(int e, int (&K)[2], int (&f)[2]) const {
    int n = 0;
    if (e < nv()) {
      const int i = e % (nx + 1), j = e / (nx + 1);
      if (i >= 1) { K[n] = (i - 1) + nx * j; f[n] = 1; ++n; }
      if (i < nx) { K[n] = i + nx * j; f[n] = 0; ++n; }
    } else {
      const int hh = e - nv(), i = hh % nx, j = hh / nx;
      if (j >= 1) { K[n] = i + nx * (j - 1); f[n] = 3; ++n; }
      if (j < ny) { K[n] = i + nx * j; f[n] = 2; ++n; }
    }
    return n;
  }
  // face of edge e in element K (-1 if e is not one of K's faces)
  __device__ __forceinline__ int face_in(int K, int e) const {
    const int ki = K % nx, kj = K / nx;
    if (e == vedge(ki, kj)) return 0;
    if (e == vedge(ki + 1, kj)) return 1;
    if (e == hedge(ki, kj)) return 2;
    if (e == hedge(ki, kj + 1)) return 3;
    return -1;
  }
};

// G blocks of row edge e: vertical rows at Gv + e * 2 n1^2, horizontal rows at
// Gh + (e - nv) * 6 n1^2
template <typename T>
__device__ __forceinline__ T* fsai_row(T* Gv, T* Gh, const FsaiMesh& m, int e) {
  const int b2 = m.n1 * m.n1;
  return e < m.nv() ? Gv + (size_t)e * kFsaiVSlots * b2 : Gh + (size_t)(e - m.nv()) * kFsaiHSlots * b2;
}

// One warp per row dof (e, a): A[J, J] from the element blocks S [nel][m][m],
// its Cholesky factor, and G[i, J] = L^-T e_last.
__global__ void fsai_setup_kernel(FsaiMesh m, const double* __restrict__ S, double* __restrict__ Gv,
                                  double* __restrict__ Gh, int* err) {
  extern __shared__ double fsai_smem[];
  const int n1 = m.n1, mm = 4 * n1, nmax = kFsaiHSlots * n1;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* A = fsai_smem + (size_t)wib * (nmax * nmax + 2 * nmax);
  double* y = A + nmax * nmax;
  int* Je = reinterpret_cast<int*>(y + nmax);      // column edge and node of J
  int* Jn = Je + nmax;                             // (2 nmax ints fit in nmax doubles)
  const int n_edges = m.nv() + m.nx * (m.ny + 1);
  const long rows = (long)n_edges * n1;
  const long w0 = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = ((long)gridDim.x * blockDim.x) >> 5;
  for (long row = w0; row < rows; row += nw) {
    const int e = (int)(row / n1), a = (int)(row % n1);
    const int nslots = e < m.nv() ? kFsaiVSlots : kFsaiHSlots;
    double* Grow = fsai_row(Gv, Gh, m, e) + (size_t)a * n1;   // + s * n1^2 + b
    if (m.slot_edge(e, nslots - 1) < 0) {
      // boundary row: G row is zero
      for (int idx = lane; idx < nslots * n1; idx += 32) Grow[(idx / n1) * n1 * n1 + idx % n1] = 0.0;
      continue;
    }
    // J in ascending global order: the slots in order, then the own nodes 0..a
    int nJ = 0;
    if (lane == 0) {
      for (int s = 0; s < nslots; ++s) {
        const int ec = m.slot_edge(e, s);
        if (ec < 0) continue;
        const int nb = (s == nslots - 1) ? a + 1 : n1;
        for (int b = 0; b < nb; ++b) { Je[nJ] = ec; Jn[nJ] = b; ++nJ; }
      }
    }
    nJ = __shfl_sync(0xffffffffu, nJ, 0);
    __syncwarp();
    // A[J, J]: sum over the elements of the row's edge that also hold the column's
    for (int idx = lane; idx < nJ * nJ; idx += 32) {
      const int r = idx / nJ, cc = idx % nJ;
      const int er = Je[r], ec = Je[cc];
      int K[2], f[2];
      const int nk = m.edge_elems(er, K, f);
      double v = 0.0;
      for (int q = 0; q < nk; ++q) {
        const int fc = m.face_in(K[q], ec);
        if (fc >= 0) v += S[((size_t)K[q] * mm + f[q] * n1 + Jn[r]) * mm + fc * n1 + Jn[cc]];
      }
      A[r * nJ + cc] = v;
    }
    __syncwarp();
    // Cholesky, lower triangle in place
    bool bad = false;
    for (int jj = 0; jj < nJ; ++jj) {
      const double ajj = A[jj * nJ + jj];
      if (!(ajj > 0.0)) bad = true;
      const double d = sqrt(fmax(ajj, 1e-300));
      __syncwarp();
      for (int r = jj + 1 + lane; r < nJ; r += 32) A[r * nJ + jj] /= d;
      if (lane == 0) A[jj * nJ + jj] = d;
      __syncwarp();
      for (int r = jj + 1; r < nJ; ++r) {
        const double lrj = A[r * nJ + jj];
        for (int l = jj + 1 + lane; l <= r; l += 32) A[r * nJ + l] -= lrj * A[l * nJ + jj];
      }
      __syncwarp();
    }
    if (bad && lane == 0) atomicExch(err, 1);
    // y = L^-T e_last by back substitution (one lane; n <= 48)
    if (lane == 0) {
      for (int r = nJ - 1; r >= 0; --r) {
        double acc = (r == nJ - 1) ? 1.0 : 0.0;
        for (int l = r + 1; l < nJ; ++l) acc -= A[l * nJ + r] * y[l];
        y[r] = acc / A[r * nJ + r];
      }
    }
    __syncwarp();
    // scatter into the slot blocks (zeros where J has no entry)
    for (int idx = lane; idx < nslots * n1; idx += 32) Grow[(idx / n1) * n1 * n1 + idx % n1] = 0.0;
    __syncwarp();
    if (lane == 0) {
      int r = 0;
      for (int s = 0; s < nslots; ++s) {
        if (m.slot_edge(e, s) < 0) continue;
        const int nb = (s == nslots - 1) ? a + 1 : n1;
        for (int b = 0; b < nb; ++b, ++r) Grow[(size_t)s * n1 * n1 + b] = y[r];
      }
    }
    __syncwarp();
  }
}

// Index tables of the apply (built once per mesh at set-up, the same for every
// p-level): rowslots[e][s] = the column edge of slot s of row edge e (-1:
// empty), colrows[e'][q] = 8 * (row edge) + slot for the q-th row whose pattern
// holds edge e' (own row first, -1 after the last), so the apply kernels read
// their neighbours instead of computing them.
__global__ void fsai_tables_kernel(FsaiMesh m, int* __restrict__ rowslots, int* __restrict__ colrows) {
  const int nv = m.nv(), n_edges = nv + m.nx * (m.ny + 1);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_edges; e += gridDim.x * blockDim.x) {
    const int nslots = e < nv ? kFsaiVSlots : kFsaiHSlots;
    for (int s = 0; s < kFsaiHSlots; ++s) rowslots[e * kFsaiHSlots + s] = s < nslots ? m.slot_edge(e, s) : -1;
    int re[6], rs[6], nr = 0;
    if (e < nv) {
      const int i = e % (m.nx + 1), j = e / (m.nx + 1);
      if (m.vin(i, j)) {
        re[nr] = e; rs[nr] = 1; ++nr;
        if (m.vin(i + 1, j)) { re[nr] = m.vedge(i + 1, j); rs[nr] = 0; ++nr; }
        if (m.hin(i, j + 1)) { re[nr] = m.hedge(i, j + 1); rs[nr] = 0; ++nr; }
        if (m.hin(i - 1, j + 1)) { re[nr] = m.hedge(i - 1, j + 1); rs[nr] = 1; ++nr; }
        if (m.hin(i, j)) { re[nr] = m.hedge(i, j); rs[nr] = 2; ++nr; }
        if (m.hin(i - 1, j)) { re[nr] = m.hedge(i - 1, j); rs[nr] = 3; ++nr; }
      }
    } else {
      const int hh = e - nv, i = hh % m.nx, j = hh / m.nx;
      if (m.hin(i, j)) {
        re[nr] = e; rs[nr] = 5; ++nr;
        if (m.hin(i, j + 1)) { re[nr] = m.hedge(i, j + 1); rs[nr] = 4; ++nr; }
      }
    }
    for (int q = 0; q < 6; ++q) colrows[e * 6 + q] = q < nr ? 8 * re[q] + rs[q] : -1;
  }
}

// w = G t for nb columns ([dof][nb], column fastest): one thread per (row dof,
// column); boundary rows give 0.
template <int N1, typename TG, typename T>
__global__ void __launch_bounds__(256) fsai_g_kernel(int nv, int n_edges, const int* __restrict__ rowslots,
                                                     const TG* __restrict__ Gv, const TG* __restrict__ Gh,
                                                     const T* __restrict__ t, T* __restrict__ w, int nb) {
  constexpr int B2 = N1 * N1;
  const size_t total = (size_t)n_edges * N1 * nb;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    size_t rowd = idx;
    int col = 0;
    if (nb > 1) { rowd = idx / (size_t)nb; col = (int)(idx - rowd * nb); }
    const int e = (int)(rowd / N1), a = (int)(rowd - (size_t)e * N1);
    const bool vert = e < nv;
    const int nslots = vert ? kFsaiVSlots : kFsaiHSlots;
    const TG* Grow = (vert ? Gv + (size_t)e * kFsaiVSlots * B2 : Gh + (size_t)(e - nv) * kFsaiHSlots * B2) + a * N1;
    const int* tab = rowslots + (size_t)e * kFsaiHSlots;
    T acc = T(0);
#pragma unroll
    for (int s = 0; s < kFsaiHSlots; ++s) {
      if (s >= nslots) break;
      const int ec = __ldg(tab + s);
      if (ec < 0) continue;
      const TG* g = Grow + s * B2;
      const T* tc = t + (size_t)ec * N1 * nb + col;
      const int nbn = (s == nslots - 1) ? a + 1 : N1;
#pragma unroll
      for (int b = 0; b < N1; ++b)
        if (b < nbn) acc += (T)__ldg(g + b) * __ldg(tc + (size_t)b * nb);
    }
    w[idx] = acc;
  }
}

// z = c + G^T w (c may be null; z may alias c): one thread per (column dof
// (e', b), column) sums G[i, (e', b)] w_i over the rows i whose pattern holds
// e' (colrows, own row first), each over its nodes a (a >= b on the own row).
template <int N1, typename TG, typename T>
__global__ void __launch_bounds__(256) fsai_gt_kernel(int nv, int n_edges, const int* __restrict__ colrows,
                                                      const TG* __restrict__ Gv, const TG* __restrict__ Gh,
                                                      const T* __restrict__ w, const T* c, T* z, int nb) {
  constexpr int B2 = N1 * N1;
  const size_t total = (size_t)n_edges * N1 * nb;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    size_t cold = idx;
    int col = 0;
    if (nb > 1) { cold = idx / (size_t)nb; col = (int)(idx - cold * nb); }
    const int ep = (int)(cold / N1), b = (int)(cold - (size_t)ep * N1);
    const int* tab = colrows + (size_t)ep * 6;
    const int first = __ldg(tab);
    T acc = T(0);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const int code = q == 0 ? first : __ldg(tab + q);
      if (code < 0) break;
      const int re = code >> 3, sl = code & 7;
      const TG* g = (re < nv ? Gv + (size_t)re * kFsaiVSlots * B2 : Gh + (size_t)(re - nv) * kFsaiHSlots * B2) +
                    sl * B2 + b;
      const T* wr = w + (size_t)re * N1 * nb + col;
      const int a0 = (q == 0) ? b : 0;                                       // own row: a >= b
#pragma unroll
      for (int aa = 0; aa < N1; ++aa)
        if (aa >= a0) acc += (T)__ldg(g + aa * N1) * __ldg(wr + (size_t)aa * nb);
    }
    const T base = c ? c[idx] : T(0);
    z[idx] = first >= 0 ? base + acc : T(0);
  }
}

__global__ void fsai_d2f_kernel(size_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    b[t] = (float)a[t];
}

int fsai_grid(size_t n, int num_sms) {
  size_t b = (n + 255) / 256;
  const size_t cap = (size_t)num_sms * 16;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

// G of level p (p >= 1) from its element blocks (plev[p].Sdense, FP64); FP32
// copy for the float V-cycles when the context is mixed.
cudaError_t launch_fsai_setup(Context* c, int p, cudaStream_t s) {
  PLevel& L = c->plev[p];
  const int n1 = L.n1, nmax = kFsaiHSlots * n1;
  const size_t nvr = (size_t)(c->mesh.nx + 1) * c->mesh.ny, nhr = (size_t)c->mesh.nx * (c->mesh.ny + 1);
  const size_t ent = (nvr * kFsaiVSlots + nhr * kFsaiHSlots) * n1 * n1;
  if (!c->fsai_rowslots) {
    HDG_CUDA_TRY(ctx_alloc(c, (void**)&c->fsai_rowslots, (size_t)c->n_edges * kFsaiHSlots * sizeof(int)));
    HDG_CUDA_TRY(ctx_alloc(c, (void**)&c->fsai_colrows, (size_t)c->n_edges * 6 * sizeof(int)));
    FsaiMesh m0{c->mesh.nx, c->mesh.ny, n1};
    fsai_tables_kernel<<<fsai_grid((size_t)c->n_edges, c->num_sms), 256, 0, s>>>(m0, c->fsai_rowslots,
                                                                                c->fsai_colrows);
    HDG_CUDA_TRY(cudaGetLastError());
  }
  HDG_CUDA_TRY(ctx_alloc(c, (void**)&L.G64, ent * sizeof(double)));
  if (c->opt.mixed) HDG_CUDA_TRY(ctx_alloc(c, (void**)&L.G32, ent * sizeof(float)));
  L.fsai_entries = ent;
  FsaiMesh m{c->mesh.nx, c->mesh.ny, n1};
  const size_t per_warp = (size_t)(nmax * nmax + 2 * nmax) * sizeof(double);
  int wpb = (int)((64 * 1024) / per_warp);
  if (wpb < 1) wpb = 1;
  if (wpb > 8) wpb = 8;
  const size_t smem = per_warp * wpb;
  if ((size_t)c->smem_optin < smem) return cudaErrorInvalidValue;
  HDG_CUDA_TRY(cudaFuncSetAttribute(fsai_setup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const long rows = (long)(nvr + nhr) * n1;
  long blocks = (rows + wpb - 1) / wpb;
  if (blocks > (long)c->num_sms * 32) blocks = (long)c->num_sms * 32;
  fsai_setup_kernel<<<(int)blocks, 32 * wpb, smem, s>>>(m, L.Sdense, L.G64, L.G64 + nvr * kFsaiVSlots * n1 * n1,
                                                        c->err_flag);
  HDG_CUDA_TRY(cudaGetLastError());
  if (L.G32) {
    fsai_d2f_kernel<<<fsai_grid(ent, c->num_sms), 256, 0, s>>>(ent, L.G64, L.G32);
    HDG_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

template <int N1, typename TG, typename T>
static void fsai_pair(const Context* c, const TG* G, size_t off, const T* in, const T* add, T* out, T* wbuf, int nb,
                      cudaStream_t s) {
  const int nv = (c->mesh.nx + 1) * c->mesh.ny;
  const size_t n = (size_t)c->n_edges * N1 * nb;
  const int g = fsai_grid(n, c->num_sms);
  fsai_g_kernel<N1, TG, T><<<g, 256, 0, s>>>(nv, c->n_edges, c->fsai_rowslots, G, G + off, in, wbuf, nb);
  fsai_gt_kernel<N1, TG, T><<<g, 256, 0, s>>>(nv, c->n_edges, c->fsai_colrows, G, G + off, wbuf, add, out, nb);
}

template <typename TG, typename T>
static cudaError_t fsai_dispatch(const Context* c, int n1, const TG* G, size_t off, const T* in, const T* add, T* out,
                                 T* wbuf, int nb, cudaStream_t s) {
  switch (n1) {
    case 2: fsai_pair<2>(c, G, off, in, add, out, wbuf, nb, s); break;
    case 3: fsai_pair<3>(c, G, off, in, add, out, wbuf, nb, s); break;
    case 4: fsai_pair<4>(c, G, off, in, add, out, wbuf, nb, s); break;
    case 5: fsai_pair<5>(c, G, off, in, add, out, wbuf, nb, s); break;
    case 6: fsai_pair<6>(c, G, off, in, add, out, wbuf, nb, s); break;
    case 7: fsai_pair<7>(c, G, off, in, add, out, wbuf, nb, s); break;
    case 8: fsai_pair<8>(c, G, off, in, add, out, wbuf, nb, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// out = add + G^T G in (add may be null or alias out) on level p for nb columns,
// through the scratch wbuf ([ndof_p][nb], the vector type); double vectors use
// the FP64 factor, float vectors the FP32 one.
cudaError_t launch_fsai_smooth(Context* c, int p, int prec, const void* in, const void* add, void* out, void* wbuf,
                               int nb, cudaStream_t s) {
  PLevel& L = c->plev[p];
  const size_t nvr = (size_t)(c->mesh.nx + 1) * c->mesh.ny;
  const size_t off = nvr * kFsaiVSlots * L.n1 * L.n1;
  if (!c->fsai_rowslots || !c->fsai_colrows) return cudaErrorInvalidValue;
  if (prec_double(prec)) {
    if (!L.G64) return cudaErrorInvalidValue;
    return fsai_dispatch<double, double>(c, L.n1, L.G64, off, (const double*)in, (const double*)add, (double*)out,
                                         (double*)wbuf, nb, s);
  }
  if (!L.G32) return cudaErrorInvalidValue;
  return fsai_dispatch<float, float>(c, L.n1, L.G32, off, (const float*)in, (const float*)add, (float*)out,
                                     (float*)wbuf, nb, s);
}

}  // namespace hdg
