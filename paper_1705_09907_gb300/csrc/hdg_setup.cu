// Setup kernels: local HDG solvers and condensed blocks (Sec. 3 procedure (i),
// Eqs. shur0/shur1), Galerkin p-coarsening, the owner-record layout used by the
// trace apply (Alg. 3), Schwarz patch inverses (Sec. 6.4.2) and the p = 0
// Jacobi diagonal. All arithmetic here is FP64.
#include <cstdio>

#include "hdg_internal.h"

namespace hdg {

cudaError_t ctx_alloc(Context* c, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  // the caller's memory cap (hdg_options.max_device_bytes) fails like a full device
  if (c->opt.max_device_bytes && c->bytes + bytes > c->opt.max_device_bytes) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return e;
  c->allocs.push_back(*p);
  c->bytes += bytes;
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Index helpers (mesh numbering documented in hdg.h)
__device__ __forceinline__ int vedge(int i, int j, int nx) { return i + (nx + 1) * j; }
__device__ __forceinline__ int hedge(int i, int j, int nx, int ny) { return (nx + 1) * ny + i + nx * j; }

// ---------------------------------------------------------------------------
// Local solver on the finest level: one warp per element.
//   A_u = kappa P + tau Mb, W = kappa Z + tau Eb, A_u = L L^T,
//   V = L^-1 W, S = kappa Y + tau diag(Ml) - V^T V,
// and for the element-local operations around the solve A_u^-1 = L^-T L^-1 and
// G = A_u^-1 W = L^-T V (no triangular solves are left for those kernels).
struct LocalTables {
  const double *P, *Mb, *Z, *Eb, *Y, *Ml;
};

__global__ void local_setup_kernel(int nel, int n, int m, double tau, int tau_kappa, const double* __restrict__ kappa,
                                   LocalTables tb, double* __restrict__ Sout, double* __restrict__ Ainv_out,
                                   double* __restrict__ Gout, int* err) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  double* A = sm + (size_t)wid * (2 * n * n + n * m);
  double* W = A + n * n;
  double* X = W + n * m;                     // A_u^-1, one column per lane
  for (int e = blockIdx.x * wpb + wid; e < nel; e += gridDim.x * wpb) {
    const double kap = kappa[e];
    const double te = tau_kappa ? kap : tau;          // tau_K
    for (int idx = lane; idx < n * n; idx += 32) A[idx] = kap * tb.P[idx] + te * tb.Mb[idx];
    for (int idx = lane; idx < n * m; idx += 32) W[idx] = kap * tb.Z[idx] + te * tb.Eb[idx];
    __syncwarp();
    // right-looking Cholesky, lower triangle in place
    bool bad = false;
    for (int j = 0; j < n; ++j) {
      const double ajj = A[j * n + j];
      if (!(ajj > 0.0)) bad = true;
      const double d = sqrt(fmax(ajj, 1e-300));
      __syncwarp();
      for (int i = j + 1 + lane; i < n; i += 32) A[i * n + j] /= d;
      if (lane == 0) A[j * n + j] = d;
      __syncwarp();
      for (int i = j + 1; i < n; ++i) {
        const double lij = A[i * n + j];
        for (int l = j + 1 + lane; l <= i; l += 32) A[i * n + l] -= lij * A[l * n + j];
      }
      __syncwarp();
    }
    if (bad && lane == 0) atomicExch(err, 1);
    // V = L^-1 W, one column per lane
    for (int c = lane; c < m; c += 32) {
      for (int i = 0; i < n; ++i) {
        double s = W[i * m + c];
        for (int l = 0; l < i; ++l) s -= A[i * n + l] * W[l * m + c];
        W[i * m + c] = s / A[i * n + i];
      }
    }
    __syncwarp();
    // S = kappa Y + tau Ml - V^T V
    double* S = Sout + (size_t)e * m * m;
    for (int idx = lane; idx < m * m; idx += 32) {
      const int r = idx / m, c = idx % m;
      double s = kap * tb.Y[idx] + ((r == c) ? te * tb.Ml[r] : 0.0);
      for (int i = 0; i < n; ++i) s -= W[i * m + r] * W[i * m + c];
      S[idx] = s;
    }
    // A_u^-1 column j (lane j, j + 32): L^-1 e_j forward, then L^-T backward
    for (int j = lane; j < n; j += 32) {
      for (int i = 0; i < n; ++i) {
        double s = (i == j) ? 1.0 : 0.0;
        for (int l = j; l < i; ++l) s -= A[i * n + l] * X[l * n + j];
        X[i * n + j] = i < j ? 0.0 : s / A[i * n + i];
      }
      for (int i = n - 1; i >= 0; --i) {
        double s = X[i * n + j];
        for (int l = i + 1; l < n; ++l) s -= A[l * n + i] * X[l * n + j];
        X[i * n + j] = s / A[i * n + i];
      }
    }
    // G = L^-T V, one column per lane, in place (after every lane's S entries
    // have read V)
    __syncwarp();
    for (int c = lane; c < m; c += 32) {
      for (int i = n - 1; i >= 0; --i) {
        double s = W[i * m + c];
        for (int l = i + 1; l < n; ++l) s -= A[l * n + i] * W[l * m + c];
        W[i * m + c] = s / A[i * n + i];
      }
    }
    __syncwarp();
    if (Ainv_out) {
      double* Ao = Ainv_out + (size_t)e * n * n;
      for (int idx = lane; idx < n * n; idx += 32) Ao[idx] = X[idx];
    }
    if (Gout) {
      double* G = Gout + (size_t)e * n * m;
      for (int idx = lane; idx < n * m; idx += 32) G[idx] = W[idx];
    }
    __syncwarp();
  }
}

cudaError_t launch_local_setup(Context* c, cudaStream_t s) {
  const int n = c->ref.n, m = c->ref.m;
  const size_t per_warp = (size_t)(2 * n * n + n * m) * sizeof(double);
  int wpb = (int)((96 * 1024) / per_warp);
  if (wpb < 1) wpb = 1;
  if (wpb > 8) wpb = 8;
  const size_t smem = per_warp * wpb;
  HDG_CUDA_TRY(cudaFuncSetAttribute(local_setup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, c->smem_optin));
  LocalTables tb{c->d_ref + c->off_P, c->d_ref + c->off_Mb, c->d_ref + c->off_Z,
                 c->d_ref + c->off_Eb, c->d_ref + c->off_Y, c->d_ref + c->off_Ml};
  int blocks = (c->nel + wpb - 1) / wpb;
  const int cap = c->num_sms * 16;
  if (blocks > cap) blocks = cap;
  local_setup_kernel<<<blocks, 32 * wpb, smem, s>>>(c->nel, n, m, c->opt.tau, c->opt.tau_kappa, c->kappa, tb,
                                                    c->plev[c->k].Sdense, c->Ainv, c->Gfac, c->err_flag);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Galerkin p-coarsening per element: S^{p-1} = P_K^T S^p P_K, P_K = diag(P1 x 4).
__global__ void galerkin_kernel(int nel, int n1f, const double* __restrict__ Pp,
                                const double* __restrict__ Sf, double* __restrict__ Sc) {
  const int n1c = n1f - 1, mf = 4 * n1f, mc = 4 * n1c;
  const long total = (long)nel * mc * mc;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int e = (int)(t / (mc * mc));
    const int rc = (int)(t % (mc * mc));
    const int r = rc / mc, cc = rc % mc;
    const int fr = r / n1c, ar = r % n1c, fc = cc / n1c, ac = cc % n1c;
    const double* S = Sf + (size_t)e * mf * mf;
    double sum = 0.0;
    for (int a = 0; a < n1f; ++a) {
      const double pa = Pp[a * n1c + ar];
      double inner = 0.0;
      for (int b = 0; b < n1f; ++b) inner += S[(fr * n1f + a) * mf + fc * n1f + b] * Pp[b * n1c + ac];
      sum += pa * inner;
    }
    Sc[t] = sum;
  }
}

cudaError_t launch_galerkin_coarsen(Context* c, int p_fine, cudaStream_t s) {
  const PLevel& f = c->plev[p_fine];
  PLevel& g = c->plev[p_fine - 1];
  const long total = (long)c->nel * g.m * g.m;
  int blocks = (int)((total + 255) / 256);
  if (blocks > c->num_sms * 32) blocks = c->num_sms * 32;
  galerkin_kernel<<<blocks, 256, 0, s>>>(c->nel, f.n1, f.Pp, f.Sdense, g.Sdense);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Owner-record layout from dense element blocks (see PLevel in hdg_internal.h).
__global__ void records_kernel(int nx, int ny, int n1, const double* __restrict__ dense,
                               double* __restrict__ rec, long total) {
  const int m = 4 * n1, R = 4 * n1 * m;
  const int spr = (nx + kSeg - 1) / kSeg;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int lane = (int)(t % kSeg);
    const long sr = t / kSeg;
    const int r = (int)(sr % R);
    const int seg = (int)(sr / R);
    const int j = seg / spr, i = (seg % spr) * kSeg + lane;
    const int slot = r / (n1 * m), a = (r / m) % n1, col = r % m;
    double v = 0.0;
    if (i < nx && j < ny) {
      int ki = i, kj = j, face;
      switch (slot) {
        case 0: face = 0; break;               // own W rows
        case 1: ki = i - 1; face = 1; break;   // west neighbour's E rows
        case 2: face = 2; break;               // own S rows
        default: kj = j - 1; face = 3; break;  // south neighbour's N rows
      }
      if (ki >= 0 && kj >= 0) {
        const long K = ki + (long)nx * kj;
        v = dense[(K * m + face * n1 + a) * m + col];
      }
    }
    rec[t] = v;
  }
}

template <typename T>
__global__ void convert_kernel(const double* __restrict__ in, T* __restrict__ out, long n);
// double -> (hi, lo) float pair: hi = fl(v), lo = fl(v - hi)
template <>
__global__ void convert_kernel<float2>(const double* __restrict__ in, float2* __restrict__ out, long n) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    const double v = in[t];
    const float hi = (float)v;
    out[t] = make_float2(hi, (float)(v - (double)hi));
  }
}
template <>
__global__ void convert_kernel<float>(const double* __restrict__ in, float* __restrict__ out, long n) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    out[t] = (float)in[t];
}
template <>
__global__ void convert_kernel<__nv_bfloat16>(const double* __restrict__ in, __nv_bfloat16* __restrict__ out,
                                              long n) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    out[t] = __float2bfloat16_rn((float)in[t]);
}

static cudaError_t write_records(Context* c, int p, const double* dense, double* r64, float* r32,
                                 __nv_bfloat16* r16, float2* r2, cudaStream_t s) {
  PLevel& L = c->plev[p];
  const long total = (long)L.rec_entries;
  int blocks = (int)((total + 255) / 256);
  if (blocks > c->num_sms * 32) blocks = c->num_sms * 32;
  records_kernel<<<blocks, 256, 0, s>>>(c->mesh.nx, c->mesh.ny, L.n1, dense, r64, total);
  HDG_CUDA_TRY(cudaGetLastError());
  if (r32) { convert_kernel<float><<<blocks, 256, 0, s>>>(r64, r32, total); HDG_CUDA_TRY(cudaGetLastError()); }
  if (r16) { convert_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(r64, r16, total); HDG_CUDA_TRY(cudaGetLastError()); }
  if (r2) { convert_kernel<float2><<<blocks, 256, 0, s>>>(r64, r2, total); HDG_CUDA_TRY(cudaGetLastError()); }
  return cudaSuccess;
}

cudaError_t launch_build_records(Context* c, int p, cudaStream_t s) {
  PLevel& L = c->plev[p];
  return write_records(c, p, L.Sdense, L.S64, L.S32, L.S16, L.S2, s);
}

// ---------------------------------------------------------------------------
// Weighted additive Schwarz blocks on element patches (Sec. 6.4.2): the
// assembled operator restricted to the element's 4 faces is S_K plus, on each
// interior face, the neighbour's diagonal block for that face. Boundary faces
// are removed (identity rows/cols, zero in the result). The stored block is
// W A_patch^-1 with W = 1/2 (every interior dof lies in two patches).
__global__ void asm_kernel(int nx, int ny, int n1, const double* __restrict__ Sd, double* __restrict__ Md,
                           int* err) {
  extern __shared__ double sm[];
  const int m = 4 * n1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  double* A = sm + (size_t)wid * (2 * m * m);
  double* X = A + m * m;
  const int nel = nx * ny;
  for (int e = blockIdx.x * wpb + wid; e < nel; e += gridDim.x * wpb) {
    const int i = e % nx, j = e / nx;
    bool bnd[4] = {i == 0, i == nx - 1, j == 0, j == ny - 1};
    int nb[4] = {e - 1, e + 1, e - nx, e + nx};
    const int opp[4] = {1, 0, 3, 2};
    const double* S = Sd + (size_t)e * m * m;
    for (int idx = lane; idx < m * m; idx += 32) {
      const int r = idx / m, cc = idx % m;
      const int fr = r / n1, fc = cc / n1;
      double v;
      if (bnd[fr] || bnd[fc]) {
        v = (r == cc) ? 1.0 : 0.0;
      } else {
        v = S[idx];
        if (fr == fc) {
          const double* Sn = Sd + (size_t)nb[fr] * m * m;
          const int o = opp[fr];
          v += Sn[(o * n1 + r % n1) * m + o * n1 + cc % n1];
        }
      }
      A[idx] = v;
    }
    __syncwarp();
    bool bad = false;
    for (int jj = 0; jj < m; ++jj) {
      const double ajj = A[jj * m + jj];
      if (!(ajj > 0.0)) bad = true;
      const double d = sqrt(fmax(ajj, 1e-300));
      __syncwarp();
      for (int r = jj + 1 + lane; r < m; r += 32) A[r * m + jj] /= d;
      if (lane == 0) A[jj * m + jj] = d;
      __syncwarp();
      for (int r = jj + 1; r < m; ++r) {
        const double lrj = A[r * m + jj];
        for (int l = jj + 1 + lane; l <= r; l += 32) A[r * m + l] -= lrj * A[l * m + jj];
      }
      __syncwarp();
    }
    if (bad && lane == 0) atomicExch(err, 2);
    // inverse: solve L L^T X = I, one column per lane
    for (int col = lane; col < m; col += 32) {
      for (int r = 0; r < m; ++r) {
        double sacc = (r == col) ? 1.0 : 0.0;
        for (int l = 0; l < r; ++l) sacc -= A[r * m + l] * X[l * m + col];
        X[r * m + col] = sacc / A[r * m + r];
      }
      for (int r = m - 1; r >= 0; --r) {
        double sacc = X[r * m + col];
        for (int l = r + 1; l < m; ++l) sacc -= A[l * m + r] * X[l * m + col];
        X[r * m + col] = sacc / A[r * m + r];
      }
    }
    __syncwarp();
    double* Mo = Md + (size_t)e * m * m;
    for (int idx = lane; idx < m * m; idx += 32) {
      const int r = idx / m, cc = idx % m;
      Mo[idx] = (bnd[r / n1] || bnd[cc / n1]) ? 0.0 : 0.5 * X[idx];
    }
    __syncwarp();
  }
}

cudaError_t launch_asm_blocks(Context* c, int p, cudaStream_t s) {
  PLevel& L = c->plev[p];
  const size_t per_warp = (size_t)2 * L.m * L.m * sizeof(double);
  int wpb = (int)((64 * 1024) / per_warp);
  if (wpb < 1) wpb = 1;
  if (wpb > 8) wpb = 8;
  const size_t smem = per_warp * wpb;
  HDG_CUDA_TRY(cudaFuncSetAttribute(asm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, c->smem_optin));
  double* Md = nullptr;
  HDG_CUDA_TRY(cudaMallocAsync((void**)&Md, (size_t)c->nel * L.m * L.m * sizeof(double), s));
  int blocks = (c->nel + wpb - 1) / wpb;
  if (blocks > c->num_sms * 16) blocks = c->num_sms * 16;
  asm_kernel<<<blocks, 32 * wpb, smem, s>>>(c->mesh.nx, c->mesh.ny, L.n1, L.Sdense, Md, c->err_flag);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = write_records(c, p, Md, L.M64, L.M32, L.M16, L.M2, s);
  if (e == cudaSuccess && L.M32 && c->red_z) {   // packed copy for the float cycles' one-vector applies
    const size_t ep = ((size_t)c->nel + 31) / 32 * 32;
    e = ctx_alloc(c, (void**)&L.Mp32, (size_t)L.m * (L.m + 1) / 2 * ep * sizeof(float));
    if (e == cudaSuccess) e = launch_sym_pack(c, p, Md, s);
  }
  cudaError_t e2 = cudaFreeAsync(Md, s);
  return e != cudaSuccess ? e : e2;
}

// ---------------------------------------------------------------------------
// Inverse diagonal of the assembled p = 0 operator (0 on boundary edges).
__global__ void p0_diag_kernel(int n_edges, const int32_t* __restrict__ edge_elem,
                               const int32_t* __restrict__ edge_face, const double* __restrict__ S0,
                               double* __restrict__ dinv64, float* __restrict__ dinv32) {
  for (int ed = blockIdx.x * blockDim.x + threadIdx.x; ed < n_edges; ed += gridDim.x * blockDim.x) {
    const int e1 = edge_elem[2 * ed], e2 = edge_elem[2 * ed + 1];
    double v = 0.0;
    if (e1 >= 0 && e2 >= 0) {
      const int f1 = edge_face[2 * ed], f2 = edge_face[2 * ed + 1];
      const double d = S0[(size_t)e1 * 16 + f1 * 4 + f1] + S0[(size_t)e2 * 16 + f2 * 4 + f2];
      v = 1.0 / d;
    }
    dinv64[ed] = v;
    if (dinv32) dinv32[ed] = (float)v;
  }
}

cudaError_t launch_p0_diag(Context* c, cudaStream_t s) {
  PLevel& L = c->plev[0];
  int blocks = (c->n_edges + 255) / 256;
  if (blocks > c->num_sms * 32) blocks = c->num_sms * 32;
  p0_diag_kernel<<<blocks, 256, 0, s>>>(c->n_edges, c->edge_elem, c->edge_face, L.Sdense, L.dinv64, L.dinv32);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Index maps of the mesh numbering (Map0..Map3 of Alg. 3).
__global__ void maps_kernel(int nx, int ny, int32_t* __restrict__ e2e, int32_t* __restrict__ edge_elem,
                            int32_t* __restrict__ edge_face) {
  const int nel = nx * ny;
  const int n_edges = (nx + 1) * ny + nx * (ny + 1);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_edges; t += gridDim.x * blockDim.x) {
    int lo = -1, hi = -1, flo = -1, fhi = -1;
    const int nv = (nx + 1) * ny;
    if (t < nv) {
      const int i = t % (nx + 1), j = t / (nx + 1);
      if (i > 0) { lo = (i - 1) + nx * j; flo = 1; }
      if (i < nx) { hi = i + nx * j; fhi = 0; }
    } else {
      const int u = t - nv, i = u % nx, j = u / nx;
      if (j > 0) { lo = i + nx * (j - 1); flo = 3; }
      if (j < ny) { hi = i + nx * j; fhi = 2; }
    }
    edge_elem[2 * t] = lo; edge_elem[2 * t + 1] = hi;
    edge_face[2 * t] = flo; edge_face[2 * t + 1] = fhi;
    if (t < nel) {
      const int i = t % nx, j = t / nx;
      e2e[4 * t + 0] = vedge(i, j, nx);
      e2e[4 * t + 1] = vedge(i + 1, j, nx);
      e2e[4 * t + 2] = hedge(i, j, nx, ny);
      e2e[4 * t + 3] = hedge(i, j + 1, nx, ny);
    }
  }
}

cudaError_t launch_maps(Context* c, cudaStream_t s) {
  const int total = c->n_edges > c->nel ? c->n_edges : c->nel;
  int blocks = (total + 255) / 256;
  if (blocks > c->num_sms * 32) blocks = c->num_sms * 32;
  maps_kernel<<<blocks, 256, 0, s>>>(c->mesh.nx, c->mesh.ny, c->e2e, c->edge_elem, c->edge_face);
  return cudaGetLastError();
}

// kappa validation: err = 3 on a non-positive or non-finite entry
__global__ void check_kappa_kernel(int nel, const double* __restrict__ kappa, int* err) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nel; e += gridDim.x * blockDim.x) {
    const double v = kappa[e];
    if (!(v > 0.0) || !isfinite(v)) atomicExch(err, 3);
  }
}

cudaError_t launch_check_kappa(Context* c, cudaStream_t s) {
  int blocks = (c->nel + 255) / 256;
  if (blocks > c->num_sms * 32) blocks = c->num_sms * 32;
  check_kappa_kernel<<<blocks, 256, 0, s>>>(c->nel, c->kappa, c->err_flag);
  return cudaGetLastError();
}

}  // namespace hdg
