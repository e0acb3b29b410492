// Host-side reference tables: 1-D quadrature, nodal bases and the element
// matrices of the HDG local solver (Sec. 3 Eqs. static_1, static_2, shur0 and
// the basis choices of Sec. 4), computed once in FP64 and uploaded.
//
// Element-level algebra used by the device kernels. With (q, v) ranging over
// the vector volume space, u, w over the scalar one and lambda, mu over the 4
// faces' trace spaces:
//   Eq. static_1:  kappa^-1 M Q_c - B_c^T U + C_c Lambda = 0            (c = x, y)
//   Eq. static_2:  sum_c B_c Q_c + tau Mb U - tau Eb Lambda = F
// where M_ij = (phi_j, phi_i), (B_c)_ij = (phi_i, d_c phi_j),
// (C_c)_{i,(f,a)} = <mu_a, phi_i n_c>_f, Mb_ij = <phi_j, phi_i>_dK,
// (Eb)_{i,(f,a)} = <mu_a, phi_i>_f. Eliminating Q_c = kappa M^-1 (B_c^T U - C_c
// Lambda) leaves the SPD system
//   (kappa P + tau Mb) U = (kappa Z + tau Eb) Lambda + F,
//   P = sum_c B_c M^-1 B_c^T,  Z = sum_c B_c M^-1 C_c,
// and the face flux of Eq. shur1 gives the condensed block
//   S_K = kappa Y + tau diag(Ml) - W^T (kappa P + tau Mb)^-1 W,
//   W = kappa Z + tau Eb,  Y = sum_c C_c^T M^-1 C_c,  Ml = face mass (diagonal
// for the Gauss-Legendre nodal trace basis).
#include <cmath>
#include <stdexcept>

#include "hdg_internal.h"

namespace hdg {

static void legendre(int n, double x, double& pn, double& dpn) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { pn = 1.0; dpn = 0.0; return; }
  for (int m = 2; m <= n; ++m) {
    double p2 = ((2.0 * m - 1.0) * x * p1 - (m - 1.0) * p0) / m;
    p0 = p1; p1 = p2;
  }
  pn = p1;
  // P_n' by the derivative recurrence P_n' = n (x P_n - P_{n-1}) / (x^2 - 1)
  dpn = (std::fabs(x * x - 1.0) < 1e-300) ? 0.5 * n * (n + 1) * std::pow(x, n + 1)
                                          : n * (x * p1 - p0) / (x * x - 1.0);
}

void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    // Newton from the asymptotic initial guess, root i counted from +1
    double z = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(q, z, p, dp);
      double dz = p / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p, dp;
    legendre(q, z, p, dp);
    x[q - 1 - i] = z;
    w[q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

void gauss_lobatto(int q, std::vector<double>& x, std::vector<double>& w) {
  if (q < 2) throw std::invalid_argument("gauss_lobatto: q >= 2");
  const int n = q - 1;
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  x[0] = -1.0;
  x[n] = 1.0;
  for (int i = 1; i < n; ++i) {
    // interior nodes: roots of P_n'; Newton with P_n'' from Legendre's equation
    double z = -std::cos(M_PI * i / n);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(n, z, p, dp);
      double d2p = (2.0 * z * dp - n * (n + 1.0) * p) / (1.0 - z * z);
      double dz = dp / d2p;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  for (int i = 0; i <= n; ++i) {
    double p, dp;
    legendre(n, x[i], p, dp);
    w[i] = 2.0 / (n * (n + 1.0) * p * p);
  }
}

// Lagrange basis on `nodes` at point t (product form) and its derivative.
static void lagrange_eval(const std::vector<double>& nodes, double t, std::vector<double>& val,
                          std::vector<double>& der) {
  const int n = (int)nodes.size();
  val.assign(n, 0.0);
  der.assign(n, 0.0);
  if (n == 1) { val[0] = 1.0; return; }
  for (int j = 0; j < n; ++j) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) v *= (t - nodes[m]) / (nodes[j] - nodes[m]);
    val[j] = v;
    double d = 0.0;
    for (int m = 0; m < n; ++m) {
      if (m == j) continue;
      double term = 1.0 / (nodes[j] - nodes[m]);
      for (int l = 0; l < n; ++l)
        if (l != j && l != m) term *= (t - nodes[l]) / (nodes[j] - nodes[l]);
      d += term;
    }
    der[j] = d;
  }
}

void p_prolongation_1d(int p, std::vector<double>& Pp) {
  std::vector<double> xc, wc, xf, wf, v, d;
  gauss_legendre(p + 1, xc, wc);
  gauss_legendre(p + 2, xf, wf);
  Pp.assign((size_t)(p + 2) * (p + 1), 0.0);
  for (int a = 0; a < p + 2; ++a) {
    lagrange_eval(xc, xf[a], v, d);
    for (int b = 0; b < p + 1; ++b) Pp[a * (p + 1) + b] = v[b];
  }
}

// Dense SPD inverse by Cholesky (small matrices, host).
static void spd_inverse(int n, const std::vector<double>& A, std::vector<double>& Ai) {
  std::vector<double> L(A);
  for (int j = 0; j < n; ++j) {
    double s = L[j * n + j];
    for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
    if (!(s > 0.0)) throw std::runtime_error("spd_inverse: not positive definite");
    s = std::sqrt(s);
    L[j * n + j] = s;
    for (int i = j + 1; i < n; ++i) {
      double t = L[i * n + j];
      for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = t / s;
    }
  }
  Ai.assign((size_t)n * n, 0.0);
  std::vector<double> y(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) {
      double t = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) t -= L[i * n + k] * y[k];
      y[i] = t / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double t = y[i];
      for (int k = i + 1; k < n; ++k) t -= L[k * n + i] * Ai[k * n + c];
      Ai[i * n + c] = t / L[i * n + i];
    }
  }
}

void build_ref_tables(int p, double hx, double hy, RefTables& t) {
  t.p = p; t.n1 = p + 1; t.n = (p + 1) * (p + 1); t.m = 4 * (p + 1);
  t.nf = (p + 2) * (p + 2); t.hx = hx; t.hy = hy;
  const int n1 = t.n1, n = t.n, m = t.m;
  std::vector<double> vn;                      // volume nodes
  if (p == 0) vn = {0.0};
  else { std::vector<double> w; gauss_lobatto(p + 1, vn, w); }
  std::vector<double> tn, tw;                  // trace nodes
  gauss_legendre(p + 1, tn, tw);
  const int nq = p + 2;                        // exact for degree 2p+3 >= 2p
  std::vector<double> xq, wq;
  gauss_legendre(nq, xq, wq);
  // 1-D tables at the quadrature points
  std::vector<double> B1(nq * n1), D1(nq * n1), T1(nq * n1), v, d;
  for (int q = 0; q < nq; ++q) {
    lagrange_eval(vn, xq[q], v, d);
    for (int i = 0; i < n1; ++i) { B1[q * n1 + i] = v[i]; D1[q * n1 + i] = (p == 0) ? 0.0 : d[i]; }
    lagrange_eval(tn, xq[q], v, d);
    for (int a = 0; a < n1; ++a) T1[q * n1 + a] = v[a];
  }
  std::vector<double> Em(n1), Ep(n1);
  lagrange_eval(vn, -1.0, v, d); for (int i = 0; i < n1; ++i) Em[i] = v[i];
  lagrange_eval(vn, 1.0, v, d);  for (int i = 0; i < n1; ++i) Ep[i] = v[i];
  const double jac = hx * hy / 4.0, dxi = 2.0 / hx, deta = 2.0 / hy;

  // volume matrices
  std::vector<double> M(n * n, 0.0), Bx(n * n, 0.0), By(n * n, 0.0);
  for (int qy = 0; qy < nq; ++qy)
    for (int qx = 0; qx < nq; ++qx) {
      const double wgt = wq[qx] * wq[qy] * jac;
      for (int I = 0; I < n; ++I) {
        const int ix = I % n1, iy = I / n1;
        const double phiI = B1[qx * n1 + ix] * B1[qy * n1 + iy];
        for (int J = 0; J < n; ++J) {
          const int jx = J % n1, jy = J / n1;
          const double phiJ = B1[qx * n1 + jx] * B1[qy * n1 + jy];
          const double dxJ = D1[qx * n1 + jx] * dxi * B1[qy * n1 + jy];
          const double dyJ = B1[qx * n1 + jx] * D1[qy * n1 + jy] * deta;
          M[I * n + J] += wgt * phiI * phiJ;
          Bx[I * n + J] += wgt * phiI * dxJ;
          By[I * n + J] += wgt * phiI * dyJ;
        }
      }
    }
  // face matrices; face f: 0 W (xi=-1), 1 E (xi=+1), 2 S (eta=-1), 3 N (eta=+1)
  std::vector<double> Cx(n * m, 0.0), Cy(n * m, 0.0);
  t.Mb.assign(n * n, 0.0); t.Eb.assign(n * m, 0.0); t.Ml.assign(m, 0.0);
  for (int f = 0; f < 4; ++f) {
    const bool vert = (f < 2);
    const std::vector<double>& end = (f == 0 || f == 2) ? Em : Ep;
    const double len = vert ? hy : hx;
    const double nx_ = (f == 0) ? -1.0 : (f == 1) ? 1.0 : 0.0;
    const double ny_ = (f == 2) ? -1.0 : (f == 3) ? 1.0 : 0.0;
    for (int q = 0; q < nq; ++q) {
      const double wgt = wq[q] * len / 2.0;
      std::vector<double> phi(n);
      for (int I = 0; I < n; ++I) {
        const int ix = I % n1, iy = I / n1;
        phi[I] = vert ? end[ix] * B1[q * n1 + iy] : B1[q * n1 + ix] * end[iy];
      }
      for (int a = 0; a < n1; ++a) {
        const double mu = T1[q * n1 + a];
        const int col = f * n1 + a;
        for (int I = 0; I < n; ++I) {
          Cx[I * m + col] += wgt * phi[I] * mu * nx_;
          Cy[I * m + col] += wgt * phi[I] * mu * ny_;
          t.Eb[I * m + col] += wgt * phi[I] * mu;
        }
        t.Ml[col] += wgt * mu * mu;
      }
      for (int I = 0; I < n; ++I)
        for (int J = 0; J < n; ++J) t.Mb[I * n + J] += wgt * phi[I] * phi[J];
    }
  }
  std::vector<double> Mi;
  spd_inverse(n, M, Mi);
  t.M = M;
  // MiBt_c = M^-1 B_c^T, MiC_c = M^-1 C_c
  t.MiBt.assign(2 * n * n, 0.0);
  t.MiC.assign(2 * n * m, 0.0);
  for (int c = 0; c < 2; ++c) {
    const std::vector<double>& B = c ? By : Bx;
    const std::vector<double>& C = c ? Cy : Cx;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int l = 0; l < n; ++l) s += Mi[i * n + l] * B[j * n + l];
        t.MiBt[c * n * n + i * n + j] = s;
      }
    for (int i = 0; i < n; ++i)
      for (int a = 0; a < m; ++a) {
        double s = 0.0;
        for (int l = 0; l < n; ++l) s += Mi[i * n + l] * C[l * m + a];
        t.MiC[c * n * m + i * m + a] = s;
      }
  }
  t.P.assign(n * n, 0.0); t.Z.assign(n * m, 0.0); t.Y.assign(m * m, 0.0);
  for (int c = 0; c < 2; ++c) {
    const std::vector<double>& B = c ? By : Bx;
    const std::vector<double>& C = c ? Cy : Cx;
    const double* MiBt = &t.MiBt[c * n * n];
    const double* MiC = &t.MiC[c * n * m];
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int l = 0; l < n; ++l) s += B[i * n + l] * MiBt[l * n + j];
        t.P[i * n + j] += s;
      }
      for (int a = 0; a < m; ++a) {
        double s = 0.0;
        for (int l = 0; l < n; ++l) s += B[i * n + l] * MiC[l * m + a];
        t.Z[i * m + a] += s;
      }
    }
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) {
        double s = 0.0;
        for (int l = 0; l < n; ++l) s += C[l * m + a] * MiC[l * m + b];
        t.Y[a * m + b] += s;
      }
  }
  // source samples at the (p+2)^2 Gauss-Legendre points
  t.Vf.assign(t.nf * n, 0.0);
  t.wJf.assign(t.nf, 0.0);
  for (int qy = 0; qy < nq; ++qy)
    for (int qx = 0; qx < nq; ++qx) {
      const int r = qy * nq + qx;
      t.wJf[r] = wq[qx] * wq[qy] * jac;
      for (int I = 0; I < n; ++I) t.Vf[r * n + I] = B1[qx * n1 + I % n1] * B1[qy * n1 + I / n1];
    }
}

// Tables of the element-local postprocessing (Sec. 3 step (v)) for degree p
// on an hx x hy rectangle. u* lies in Q_{p+1} (Lagrange at the (p+2)^2 GLL
// tensor nodes) and solves (kappa grad u*, grad w) = -(q_h, grad w) for all w
// in Q_{p+1}, with the element mean of u_h. The Neumann matrix S (ns x ns,
// ns = (p+2)^2) is singular only on constants and the right-hand side g sums
// to zero, so fixing the first nodal value gives the SPD system S[1:,1:] and a
// solution u~; the constant shift c 1 that restores the mean follows from the
// node integrals m_i = (phi*_i, 1):
//   u* = kappa^-1 (I - 1 m^T / |K|) A g + 1 (u_h, 1) / |K|,  g = -sum_c D_c^T W V q_c
// with A = [[0, 0], [0, S[1:,1:]^-1]]. Outputs (row-major):
//   Hq [2][ns][n]  (kappa = 1 map from q_x, q_y nodal values to u*)
//   mu [n]         ((phi_j, 1) / |K|: the mean of u_h is mu . u)
//   Dn [2][ns][ns] (d/dx, d/dy of the Q_{p+1} interpolant at its own nodes)
void build_post_tables(int p, double hx, double hy, std::vector<double>& Hq, std::vector<double>& mu,
                       std::vector<double>& Dn) {
  const int n1 = p + 1, n = n1 * n1, s1 = p + 2, ns = s1 * s1;
  std::vector<double> vn, vw, sn, sw;
  if (p == 0) vn = {0.0};
  else gauss_lobatto(p + 1, vn, vw);
  gauss_lobatto(p + 2, sn, sw);
  const int nq = p + 3;                         // exact for the degree 2p+2 products
  std::vector<double> xq, wq, v, d;
  gauss_legendre(nq, xq, wq);
  std::vector<double> Bh(nq * n1), Bs(nq * s1), Ds(nq * s1);
  for (int q = 0; q < nq; ++q) {
    lagrange_eval(vn, xq[q], v, d);
    for (int i = 0; i < n1; ++i) Bh[q * n1 + i] = v[i];
    lagrange_eval(sn, xq[q], v, d);
    for (int i = 0; i < s1; ++i) { Bs[q * s1 + i] = v[i]; Ds[q * s1 + i] = d[i]; }
  }
  const double jac = hx * hy / 4.0, dxi = 2.0 / hx, deta = 2.0 / hy, area = hx * hy;
  // S, the gradient load G_c[i][j] = (d_c phi*_i, phi_j), node integrals
  std::vector<double> S(ns * ns, 0.0), G(2 * ns * n, 0.0), ms(ns, 0.0);
  mu.assign(n, 0.0);
  for (int qy = 0; qy < nq; ++qy)
    for (int qx = 0; qx < nq; ++qx) {
      const double wgt = wq[qx] * wq[qy] * jac;
      std::vector<double> gx(ns), gy(ns), ph(ns), pv(n);
      for (int I = 0; I < ns; ++I) {
        const int ix = I % s1, iy = I / s1;
        ph[I] = Bs[qx * s1 + ix] * Bs[qy * s1 + iy];
        gx[I] = Ds[qx * s1 + ix] * dxi * Bs[qy * s1 + iy];
        gy[I] = Bs[qx * s1 + ix] * Ds[qy * s1 + iy] * deta;
      }
      for (int J = 0; J < n; ++J) pv[J] = Bh[qx * n1 + J % n1] * Bh[qy * n1 + J / n1];
      for (int I = 0; I < ns; ++I) {
        ms[I] += wgt * ph[I];
        for (int K = 0; K < ns; ++K) S[I * ns + K] += wgt * (gx[I] * gx[K] + gy[I] * gy[K]);
        for (int J = 0; J < n; ++J) {
          G[I * n + J] += wgt * gx[I] * pv[J];
          G[ns * n + I * n + J] += wgt * gy[I] * pv[J];
        }
      }
      for (int J = 0; J < n; ++J) mu[J] += wgt * pv[J] / area;
    }
  // inverse of S with the first node fixed
  const int r = ns - 1;
  std::vector<double> S11((size_t)r * r), S11i;
  for (int i = 0; i < r; ++i)
    for (int k = 0; k < r; ++k) S11[(size_t)i * r + k] = S[(size_t)(i + 1) * ns + (k + 1)];
  spd_inverse(r, S11, S11i);
  Hq.assign((size_t)2 * ns * n, 0.0);
  for (int c = 0; c < 2; ++c) {
    // t = A g per unit q_j: t[0] = 0, t[1:] = -S11^-1 G_c[1:, j]
    std::vector<double> t((size_t)ns * n, 0.0);
    for (int i = 1; i < ns; ++i)
      for (int j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int k = 1; k < ns; ++k) acc += S11i[(size_t)(i - 1) * r + (k - 1)] * G[(size_t)c * ns * n + k * n + j];
        t[(size_t)i * n + j] = -acc;
      }
    for (int j = 0; j < n; ++j) {
      double mt = 0.0;
      for (int i = 0; i < ns; ++i) mt += ms[i] * t[(size_t)i * n + j];
      for (int i = 0; i < ns; ++i) Hq[(size_t)c * ns * n + i * n + j] = t[(size_t)i * n + j] - mt / area;
    }
  }
  // nodal derivative matrices of Q_{p+1} at its own nodes
  Dn.assign((size_t)2 * ns * ns, 0.0);
  std::vector<double> D1(s1 * s1), E1(s1 * s1);
  for (int a = 0; a < s1; ++a) {
    lagrange_eval(sn, sn[a], v, d);
    for (int b = 0; b < s1; ++b) { D1[a * s1 + b] = d[b]; E1[a * s1 + b] = (a == b) ? 1.0 : 0.0; }
  }
  for (int I = 0; I < ns; ++I)
    for (int K = 0; K < ns; ++K) {
      const int ix = I % s1, iy = I / s1, kx = K % s1, ky = K / s1;
      Dn[(size_t)I * ns + K] = D1[ix * s1 + kx] * dxi * E1[iy * s1 + ky];
      Dn[(size_t)ns * ns + I * ns + K] = E1[ix * s1 + kx] * D1[iy * s1 + ky] * deta;
    }
}

}  // namespace hdg
