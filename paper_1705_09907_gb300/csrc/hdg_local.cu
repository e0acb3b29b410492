// Element-local operations around the trace solve (Sec. 3 steps (ii) and (iv),
// Sec. 8.3 "Projection from volume to surface"), and the adjoint gradient.
// They reuse the finest-level local operators stored at setup, A_u^-1 (A_u =
// kappa P + tau Mb) and G = A_u^-1 W (W = kappa Z + tau Eb):
//   condensed RHS  b_K = G^T F                            (= W^T A_u^-1 F)
//   recovery       U = A_u^-1 (F + W lambda_K)
//                  Q_c = kappa (M^-1 B_c^T U - M^-1 C_c lambda_K)
//   adjoint        dJ/dtheta_K = -(kappa^-1 q(lambda, f), q(psi, 0))_K  (tau fixed)
//                  dJ/dtheta_K = -psi_K^T S_K lambda_K                 (tau_K = kappa_K:
//                                S_K = kappa_K S_ref and b_K does not depend on kappa_K;
//                                from the reduced blocks, apply_reduced.cu)
//                  dJ/df_q     = w_q |J| u(psi, 0)(x_q)
#include "hdg_internal.h"

namespace hdg {


struct LocalArgs {
  int nel, n, m, nf;
  double tau;
  int tau_kappa;                 // 1: tau_K = kappa_K
  const double *Ainv, *Gfac, *kappa;
  const double *Vf, *wJf, *M;
  // transposed reference matrices (one contiguous row per column of the original)
  const double *ZT, *EbT, *MiBtT, *MiCT, *VfT;
  const int32_t* e2e;
};

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

// ---------------------------------------------------------------------------
// Warp-per-element forms of condense and recovery: one warp per element, the
// element's n <= 64 volume values held two per lane (I = lane, lane + 32), the
// 4(k+1) <= 32 trace values one per lane; the triangular solves run column by
// column with the pivot broadcast by shuffle, and rows of the element's V and L
// are read by consecutive lanes.

// value of index I (0 <= I < 64) held in (lo, hi) across the warp
template <bool H>
__device__ __forceinline__ double wget(double lo, double hi, int I) {
  return __shfl_sync(0xffffffffu, (H && I >= 32) ? hi : lo, I & 31);
}

// F = Vf^T (wJf .* f) for element e, two values per lane; the weighted source
// values are formed once (lane q holds q, q + 32, q + 64; nf <= 81) and broadcast
template <bool H>
__device__ __forceinline__ void warp_load_F(const LocalArgs& a, const double* __restrict__ fq, int e, int lane,
                                            double& F0, double& F1) {
  const int n = a.n, nf = a.nf;
  const double* f = fq + (size_t)e * nf;
  const double w0 = lane < nf ? a.wJf[lane] * f[lane] : 0.0;
  const double w1 = lane + 32 < nf ? a.wJf[lane + 32] * f[lane + 32] : 0.0;
  const double w2 = lane + 64 < nf ? a.wJf[lane + 64] * f[lane + 64] : 0.0;
  F0 = 0.0; F1 = 0.0;
  for (int q = 0; q < nf; ++q) {
    const double w = __shfl_sync(0xffffffffu, q < 32 ? w0 : (q < 64 ? w1 : w2), q & 31);
    const double* Vq = a.Vf + (size_t)q * n;
    if (lane < n) F0 += Vq[lane] * w;
    if (H && lane + 32 < n) F1 += Vq[lane + 32] * w;
  }
}

template <bool H>
__global__ void condense_warp_kernel(LocalArgs a, const double* __restrict__ fq, double* __restrict__ bK) {
  const int lane = threadIdx.x & 31;
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int n = a.n, m = a.m;
  for (int e = wg; e < a.nel; e += nw) {
    double f0, f1;
    warp_load_F<H>(a, fq, e, lane, f0, f1);
    // b_K[c] = sum_I G[I][c] F_I, lanes over c
    const double* G = a.Gfac + (size_t)e * n * m;
    double b = 0.0;
    for (int I = 0; I < n; ++I) {
      const double fi = wget<H>(f0, f1, I);
      if (lane < m) b += G[I * m + lane] * fi;
    }
    if (lane < m) bK[(size_t)e * m + lane] = b;
  }
}

static LocalArgs local_args(Context* c) {
  LocalArgs a{};
  a.nel = c->nel; a.n = c->ref.n; a.m = c->ref.m; a.nf = c->ref.nf;
  a.Ainv = c->Ainv; a.Gfac = c->Gfac; a.kappa = c->kappa;
  a.tau = c->opt.tau; a.tau_kappa = c->opt.tau_kappa;
  a.Vf = c->d_ref + c->off_Vf; a.wJf = c->d_ref + c->off_wJf; a.M = c->d_ref + c->off_M;
  a.ZT = c->d_ref + c->off_ZT; a.EbT = c->d_ref + c->off_EbT;
  a.MiBtT = c->d_ref + c->off_MiBtT; a.MiCT = c->d_ref + c->off_MiCT; a.VfT = c->d_ref + c->off_VfT;
  a.e2e = c->e2e;
  return a;
}

static int grid_of(size_t n, int cap) {
  size_t b = (n + 127) / 128;
  if (b > (size_t)cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

static int warp_grid(int nel, int num_sms) {
  // 8 warps per block, up to 16 blocks per SM
  const long b = ((long)nel + 7) / 8;
  const long cap = (long)num_sms * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

cudaError_t launch_condense(Context* c, const double* f_q, double* b, int nrhs, cudaStream_t s) {
  LocalArgs a = local_args(c);
  for (int r = 0; r < nrhs; ++r) {
    if (a.n > 32) condense_warp_kernel<true><<<warp_grid(c->nel, c->num_sms), 256, 0, s>>>(a, f_q + (size_t)r * c->nel * a.nf, c->elem_scratch);
    else condense_warp_kernel<false><<<warp_grid(c->nel, c->num_sms), 256, 0, s>>>(a, f_q + (size_t)r * c->nel * a.nf, c->elem_scratch);
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
    if (a.n > 32) condense_warp_kernel<true><<<warp_grid(c->nel, c->num_sms), 256, 0, s>>>(a, f_q + (size_t)r * c->nel * a.nf, scratch);
    else condense_warp_kernel<false><<<warp_grid(c->nel, c->num_sms), 256, 0, s>>>(a, f_q + (size_t)r * c->nel * a.nf, scratch);
    HDG_CUDA_TRY(cudaGetLastError());
    gather_edges_kernel<<<grid_of((size_t)c->n_edges * c->ref.n1, c->num_sms * 32), 128, 0, s>>>(
        c->n_edges, c->ref.n1, c->edge_elem, c->edge_face, scratch, b, nrhs, r);
    HDG_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

// trace values of element e, lane c holds dof c (0 on boundary faces)
__device__ __forceinline__ double warp_trace(const LocalArgs& a, const double* __restrict__ lam, int e, int nx,
                                             int ny, int lane) {
  const int m = a.m, n1 = m / 4;
  double lc = 0.0;
  if (lane < m) {
    const int f = lane / n1, b = lane - f * n1;
    const int i = e % nx, j = e / nx;
    const bool bnd = f == 0 ? i == 0 : f == 1 ? i == nx - 1 : f == 2 ? j == 0 : j == ny - 1;
    if (!bnd) lc = lam[(size_t)a.e2e[4 * e + f] * n1 + b];
  }
  return lc;
}

// Local solution of element e (Eq. shur0) for trace values lc (lane c) and
// load F (f0, f1 hold F, or 0): U = A_u^-1 (F + W lambda_K) with W = kappa Z +
// tau Eb; Q_c = kappa (M^-1 B_c^T U - M^-1 C_c lambda_K). U returns in (f0, f1),
// Q_c in (q[2c], q[2c+1]).
template <bool H>
__device__ __forceinline__ void warp_local_solution(const LocalArgs& a, int e, double lc, int lane, double& f0,
                                                    double& f1, double (&q)[4]) {
  const int n = a.n, m = a.m;
  const double kap = a.kappa[e], tau = a.tau_kappa ? kap : a.tau;
  double z0 = 0.0, z1 = 0.0, b0 = 0.0, b1 = 0.0;          // Z lambda, Eb lambda
  for (int c = 0; c < m; ++c) {
    const double l = __shfl_sync(0xffffffffu, lc, c);
    const double* zc = a.ZT + (size_t)c * n;
    const double* ec = a.EbT + (size_t)c * n;
    if (lane < n) { z0 += zc[lane] * l; b0 += ec[lane] * l; }
    if (H && lane + 32 < n) { z1 += zc[lane + 32] * l; b1 += ec[lane + 32] * l; }
  }
  const double s0 = f0 + kap * z0 + tau * b0, s1 = f1 + kap * z1 + tau * b1;
  // U = A_u^-1 s (symmetric: row J of A_u^-1 is column J)
  const double* Ai = a.Ainv + (size_t)e * n * n;
  f0 = 0.0; f1 = 0.0;
  for (int J = 0; J < n; ++J) {
    const double sj = wget<H>(s0, s1, J);
    const double* row = Ai + (size_t)J * n;
    if (lane < n) f0 += row[lane] * sj;
    if (H && lane + 32 < n) f1 += row[lane + 32] * sj;
  }
  for (int cmp = 0; cmp < 2; ++cmp) {
    const double* MiBtT = a.MiBtT + (size_t)cmp * n * n;
    const double* MiCT = a.MiCT + (size_t)cmp * n * m;
    double q0 = 0.0, q1 = 0.0;
    for (int jj = 0; jj < n; ++jj) {
      const double uj = wget<H>(f0, f1, jj);
      const double* col = MiBtT + (size_t)jj * n;
      if (lane < n) q0 += col[lane] * uj;
      if (H && lane + 32 < n) q1 += col[lane + 32] * uj;
    }
    for (int c = 0; c < m; ++c) {
      const double l = __shfl_sync(0xffffffffu, lc, c);
      const double* col = MiCT + (size_t)c * n;
      if (lane < n) q0 -= col[lane] * l;
      if (H && lane + 32 < n) q1 -= col[lane + 32] * l;
    }
    q[2 * cmp] = kap * q0;
    q[2 * cmp + 1] = kap * q1;
  }
}

template <bool H>
__global__ void recover_warp_kernel(LocalArgs a, int nx, int ny, const double* __restrict__ lam,
                                    const double* __restrict__ fq, double* __restrict__ u, double* __restrict__ q) {
  const int lane = threadIdx.x & 31;
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int n = a.n;
  for (int e = wg; e < a.nel; e += nw) {
    double f0, f1, Q[4];
    warp_load_F<H>(a, fq, e, lane, f0, f1);
    warp_local_solution<H>(a, e, warp_trace(a, lam, e, nx, ny, lane), lane, f0, f1, Q);
    if (u) {
      if (lane < n) u[(size_t)e * n + lane] = f0;
      if (H && lane + 32 < n) u[(size_t)e * n + lane + 32] = f1;
    }
    if (q) {
      for (int cmp = 0; cmp < 2; ++cmp) {
        double* qo = q + (size_t)e * 2 * n + (size_t)cmp * n;
        if (lane < n) qo[lane] = Q[2 * cmp];
        if (H && lane + 32 < n) qo[lane + 32] = Q[2 * cmp + 1];
      }
    }
  }
}

cudaError_t launch_recover(Context* c, const double* lam, const double* f_q, double* u, double* q,
                           cudaStream_t s) {
  LocalArgs a = local_args(c);
  if (a.n > 32) recover_warp_kernel<true><<<warp_grid(c->nel, c->num_sms), 256, 0, s>>>(a, c->mesh.nx, c->mesh.ny, lam, f_q, u, q);
  else recover_warp_kernel<false><<<warp_grid(c->nel, c->num_sms), 256, 0, s>>>(a, c->mesh.nx, c->mesh.ny, lam, f_q, u, q);
  return cudaGetLastError();
}

template <bool H>
__global__ void adjoint_warp_kernel(LocalArgs a, int nx, int ny, const double* __restrict__ lam,
                                    const double* __restrict__ psi, const double* __restrict__ fq,
                                    double* __restrict__ dth, double* __restrict__ dfq) {
  const int lane = threadIdx.x & 31;
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int n = a.n;
  for (int e = wg; e < a.nel; e += nw) {
    // (U, Q) for (lambda, f) and (Up, Qp) for (psi, 0)
    double u0, u1, Q[4];
    warp_load_F<H>(a, fq, e, lane, u0, u1);
    warp_local_solution<H>(a, e, warp_trace(a, lam, e, nx, ny, lane), lane, u0, u1, Q);
    double p0 = 0.0, p1 = 0.0, Qp[4];
    warp_local_solution<H>(a, e, warp_trace(a, psi, e, nx, ny, lane), lane, p0, p1, Qp);
    if (dth) {
      // -(kappa^-1 Q, Qp)_K = -kappa^-1 sum_c Q_c^T M Qp_c
      double part = 0.0;
      for (int cmp = 0; cmp < 2; ++cmp) {
        double m0 = 0.0, m1 = 0.0;
        for (int jj = 0; jj < n; ++jj) {     // M is symmetric: column jj = row jj
          const double qj = wget<H>(Qp[2 * cmp], Qp[2 * cmp + 1], jj);
          const double* col = a.M + (size_t)jj * n;
          if (lane < n) m0 += col[lane] * qj;
          if (H && lane + 32 < n) m1 += col[lane + 32] * qj;
        }
        part += Q[2 * cmp] * m0 + Q[2 * cmp + 1] * m1;   // zero beyond n (Q is zero there)
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == 0) dth[e] = -part / a.kappa[e];
    }
    if (dfq) {
      // dJ/df_q = w_q |J| u(psi, 0)(x_q), lanes over the quadrature points
      for (int q0 = 0; q0 < a.nf; q0 += 32) {
        const int qq = q0 + lane;
        double sacc = 0.0;
        for (int I = 0; I < n; ++I) {
          const double ui = wget<H>(p0, p1, I);
          if (qq < a.nf) sacc += a.VfT[(size_t)I * a.nf + qq] * ui;
        }
        if (qq < a.nf) dfq[(size_t)e * a.nf + qq] = a.wJf[qq] * sacc;
      }
    }
  }
}

cudaError_t launch_adjoint(Context* c, const double* f_q, const double* lam, const double* psi, double* dJ_dlogk,
                           double* dJ_df, cudaStream_t s) {
  LocalArgs a = local_args(c);
  double* dth = c->opt.tau_kappa ? nullptr : dJ_dlogk;
  if (dth || dJ_df) {
    if (a.n > 32) adjoint_warp_kernel<true><<<warp_grid(c->nel, c->num_sms), 256, 0, s>>>(a, c->mesh.nx, c->mesh.ny, lam, psi, f_q, dth, dJ_df);
    else adjoint_warp_kernel<false><<<warp_grid(c->nel, c->num_sms), 256, 0, s>>>(a, c->mesh.nx, c->mesh.ny, lam, psi, f_q, dth, dJ_df);
    HDG_CUDA_TRY(cudaGetLastError());
  }
  if (c->opt.tau_kappa && dJ_dlogk) return launch_reduced_theta(c, lam, psi, dJ_dlogk, s);
  return cudaSuccess;
}

}  // namespace hdg
