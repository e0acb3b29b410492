// Element-local operations around the trace solve (Sec. 3 steps (ii) and (iv),
// Sec. 8.3 "Projection from volume to surface"), and the adjoint gradient.
// They reuse the finest-level local factors stored at setup: the Cholesky factor
// L of A_u = kappa P + tau Mb (packed lower triangle) and V = L^-1 W.
//   condensed RHS  b_K = V^T L^-1 F                       (= W^T A_u^-1 F)
//   recovery       U = L^-T (V lambda_K + L^-1 F)
//                  Q_c = kappa (M^-1 B_c^T U - M^-1 C_c lambda_K)
//   adjoint        dJ/dtheta_K = -(kappa^-1 q(lambda, f), q(psi, 0))_K
//                  dJ/df_q     = w_q |J| u(psi, 0)(x_q)
#include "hdg_internal.h"

namespace hdg {

constexpr int kMaxN = (kMaxDegree + 1) * (kMaxDegree + 1);

struct LocalArgs {
  int nel, n, m, nf;
  const double *Lfac, *Vfac, *kappa;
  const double *Vf, *wJf, *MiBt, *MiC, *M;
  const int32_t* e2e;
};

// y = L^-1 y (packed lower, row i starts at i(i+1)/2)
__device__ __forceinline__ void fwd_solve(const double* __restrict__ L, double* y, int n) {
  for (int i = 0; i < n; ++i) {
    const double* Li = L + i * (i + 1) / 2;
    double s = y[i];
    for (int l = 0; l < i; ++l) s -= Li[l] * y[l];
    y[i] = s / Li[i];
  }
}
// y = L^-T y
__device__ __forceinline__ void bwd_solve(const double* __restrict__ L, double* y, int n) {
  for (int i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int l = i + 1; l < n; ++l) s -= L[l * (l + 1) / 2 + i] * y[l];
    y[i] = s / L[i * (i + 1) / 2 + i];
  }
}

__device__ __forceinline__ void load_F(const LocalArgs& a, const double* __restrict__ fq, int e, double* F) {
  for (int I = 0; I < a.n; ++I) F[I] = 0.0;
  const double* f = fq + (size_t)e * a.nf;
  for (int q = 0; q < a.nf; ++q) {
    const double w = a.wJf[q] * f[q];
    const double* Vq = a.Vf + (size_t)q * a.n;
    for (int I = 0; I < a.n; ++I) F[I] += Vq[I] * w;
  }
}

// per-element b_K into scratch [nel][m]
__global__ void condense_elem_kernel(LocalArgs a, const double* __restrict__ fq, double* __restrict__ bK) {
  double y[kMaxN];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < a.nel; e += gridDim.x * blockDim.x) {
    load_F(a, fq, e, y);
    const double* L = a.Lfac + (size_t)e * (a.n * (a.n + 1) / 2);
    fwd_solve(L, y, a.n);
    const double* V = a.Vfac + (size_t)e * a.n * a.m;
    for (int c = 0; c < a.m; ++c) {
      double s = 0.0;
      for (int i = 0; i < a.n; ++i) s += V[i * a.m + c] * y[i];
      bK[(size_t)e * a.m + c] = s;
    }
  }
}

// b[edge] = contributions of its two elements (0 on boundary edges)
__global__ void gather_edges_kernel(int n_edges, int n1, const int32_t* __restrict__ edge_elem,
                                    const int32_t* __restrict__ edge_face, const double* __restrict__ bK,
                                    double* __restrict__ b, int nrhs, int r) {
  const int m = 4 * n1;
  const size_t total = (size_t)n_edges * n1;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int ed = (int)(t / n1), a = (int)(t % n1);
    const int e1 = edge_elem[2 * ed], e2 = edge_elem[2 * ed + 1];
    double v = 0.0;
    if (e1 >= 0 && e2 >= 0) {
      const int f1 = edge_face[2 * ed], f2 = edge_face[2 * ed + 1];
      v = bK[(size_t)e1 * m + f1 * n1 + a] + bK[(size_t)e2 * m + f2 * n1 + a];
    }
    b[t * nrhs + r] = v;
  }
}

static LocalArgs local_args(Context* c) {
  LocalArgs a{};
  a.nel = c->nel; a.n = c->ref.n; a.m = c->ref.m; a.nf = c->ref.nf;
  a.Lfac = c->Lfac; a.Vfac = c->Vfac; a.kappa = c->kappa;
  a.Vf = c->d_ref + c->off_Vf; a.wJf = c->d_ref + c->off_wJf;
  a.MiBt = c->d_ref + c->off_MiBt; a.MiC = c->d_ref + c->off_MiC; a.M = c->d_ref + c->off_M;
  a.e2e = c->e2e;
  return a;
}

static int grid_of(size_t n, int cap) {
  size_t b = (n + 127) / 128;
  if (b > (size_t)cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_condense(Context* c, const double* f_q, double* b, int nrhs, cudaStream_t s) {
  LocalArgs a = local_args(c);
  for (int r = 0; r < nrhs; ++r) {
    condense_elem_kernel<<<grid_of(c->nel, c->num_sms * 16), 128, 0, s>>>(a, f_q + (size_t)r * c->nel * a.nf,
                                                                         c->elem_scratch);
    HDG_CUDA_TRY(cudaGetLastError());
    gather_edges_kernel<<<grid_of((size_t)c->n_edges * c->ref.n1, c->num_sms * 32), 128, 0, s>>>(
        c->n_edges, c->ref.n1, c->edge_elem, c->edge_face, c->elem_scratch, b, nrhs, r);
    HDG_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

// Same as launch_condense with the per-element partial results in `scratch`
// ([nel][m] doubles, caller-provided).
cudaError_t launch_condense_into(Context* c, const double* f_q, double* b, int nrhs, double* scratch,
                                 cudaStream_t s) {
  LocalArgs a = local_args(c);
  for (int r = 0; r < nrhs; ++r) {
    condense_elem_kernel<<<grid_of(c->nel, c->num_sms * 16), 128, 0, s>>>(a, f_q + (size_t)r * c->nel * a.nf,
                                                                         scratch);
    HDG_CUDA_TRY(cudaGetLastError());
    gather_edges_kernel<<<grid_of((size_t)c->n_edges * c->ref.n1, c->num_sms * 32), 128, 0, s>>>(
        c->n_edges, c->ref.n1, c->edge_elem, c->edge_face, scratch, b, nrhs, r);
    HDG_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

// Local solution (U, Q) of element e for trace values lamK [m] and load F
// (F may be null for f = 0). U [n], Q [2n].
__device__ void local_solution(const LocalArgs& a, int e, const double* lamK, const double* F, double* U,
                               double* Q) {
  const double* L = a.Lfac + (size_t)e * (a.n * (a.n + 1) / 2);
  const double* V = a.Vfac + (size_t)e * a.n * a.m;
  double y[kMaxN];
  for (int i = 0; i < a.n; ++i) y[i] = F ? F[i] : 0.0;
  if (F) fwd_solve(L, y, a.n);
  for (int i = 0; i < a.n; ++i) {
    double s = y[i];
    for (int c = 0; c < a.m; ++c) s += V[i * a.m + c] * lamK[c];
    U[i] = s;
  }
  bwd_solve(L, U, a.n);
  const double kap = a.kappa[e];
  for (int cmp = 0; cmp < 2; ++cmp) {
    const double* MiBt = a.MiBt + (size_t)cmp * a.n * a.n;
    const double* MiC = a.MiC + (size_t)cmp * a.n * a.m;
    for (int i = 0; i < a.n; ++i) {
      double s = 0.0;
      for (int j = 0; j < a.n; ++j) s += MiBt[i * a.n + j] * U[j];
      for (int c = 0; c < a.m; ++c) s -= MiC[i * a.m + c] * lamK[c];
      Q[cmp * a.n + i] = kap * s;
    }
  }
}

__device__ __forceinline__ void gather_trace(const LocalArgs& a, const double* __restrict__ lam, int e, int nx,
                                             int ny, double* lamK) {
  const int n1 = a.m / 4;
  const int i = e % nx, j = e / nx;
  const bool bnd[4] = {i == 0, i == nx - 1, j == 0, j == ny - 1};
  for (int f = 0; f < 4; ++f) {
    const int ed = a.e2e[4 * e + f];
    for (int b = 0; b < n1; ++b) lamK[f * n1 + b] = bnd[f] ? 0.0 : lam[(size_t)ed * n1 + b];
  }
}

__global__ void recover_kernel(LocalArgs a, int nx, int ny, const double* __restrict__ lam,
                               const double* __restrict__ fq, double* __restrict__ u, double* __restrict__ q) {
  double lamK[4 * (kMaxDegree + 1)], F[kMaxN], U[kMaxN], Q[2 * kMaxN];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < a.nel; e += gridDim.x * blockDim.x) {
    gather_trace(a, lam, e, nx, ny, lamK);
    load_F(a, fq, e, F);
    local_solution(a, e, lamK, F, U, Q);
    if (u) for (int i = 0; i < a.n; ++i) u[(size_t)e * a.n + i] = U[i];
    if (q) for (int i = 0; i < 2 * a.n; ++i) q[(size_t)e * 2 * a.n + i] = Q[i];
  }
}

cudaError_t launch_recover(Context* c, const double* lam, const double* f_q, double* u, double* q,
                           cudaStream_t s) {
  LocalArgs a = local_args(c);
  recover_kernel<<<grid_of(c->nel, c->num_sms * 16), 128, 0, s>>>(a, c->mesh.nx, c->mesh.ny, lam, f_q, u, q);
  return cudaGetLastError();
}

__global__ void adjoint_kernel(LocalArgs a, int nx, int ny, const double* __restrict__ lam,
                               const double* __restrict__ psi, const double* __restrict__ fq,
                               double* __restrict__ dth, double* __restrict__ dfq) {
  double lamK[4 * (kMaxDegree + 1)], F[kMaxN], U[kMaxN], Q[2 * kMaxN], Up[kMaxN], Qp[2 * kMaxN];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < a.nel; e += gridDim.x * blockDim.x) {
    gather_trace(a, lam, e, nx, ny, lamK);
    load_F(a, fq, e, F);
    local_solution(a, e, lamK, F, U, Q);
    gather_trace(a, psi, e, nx, ny, lamK);
    local_solution(a, e, lamK, nullptr, Up, Qp);
    if (dth) {
      double s = 0.0;
      for (int cmp = 0; cmp < 2; ++cmp)
        for (int i = 0; i < a.n; ++i) {
          double mq = 0.0;
          for (int j = 0; j < a.n; ++j) mq += a.M[i * a.n + j] * Qp[cmp * a.n + j];
          s += Q[cmp * a.n + i] * mq;
        }
      dth[e] = -s / a.kappa[e];
    }
    if (dfq) {
      for (int qq = 0; qq < a.nf; ++qq) {
        double s = 0.0;
        for (int i = 0; i < a.n; ++i) s += a.Vf[(size_t)qq * a.n + i] * Up[i];
        dfq[(size_t)e * a.nf + qq] = a.wJf[qq] * s;
      }
    }
  }
}

cudaError_t launch_adjoint(Context* c, const double* f_q, const double* lam, const double* psi, double* dJ_dlogk,
                           double* dJ_df, cudaStream_t s) {
  LocalArgs a = local_args(c);
  adjoint_kernel<<<grid_of(c->nel, c->num_sms * 16), 128, 0, s>>>(a, c->mesh.nx, c->mesh.ny, lam, psi, f_q,
                                                                  dJ_dlogk, dJ_df);
  return cudaGetLastError();
}

}  // namespace hdg
