"""Adjoint gradient of J = 1/2 |lambda - lambda_obs|^2 for the condensed HDG
system A(theta) lambda = b(theta, f), theta_K = log kappa_K; float64 CPU oracle
(test infrastructure only).

The paper has no adjoint; this is the plain definition of the derivative of the
discrete solve (the trace vector lambda is the state u of J; Euclidean norm):

    psi = A^-1 (lambda - lambda_obs)                  (A is symmetric)
    dJ/dtheta_K = psi^T (db/dtheta_K - dA/dtheta_K lambda)
    dJ/df       = (db/df)^T psi

with dA/dtheta_K = A_K^T (dS_K/dtheta_K) A_K and S_K, b_K from Eqs. shur0 and
shur1 as in oracle.hdg:
    S_K = GH L^-1 CE + tau Ml,  b_K = GH L^-1 [0; F],  GH = [G  tau H],
    CE = [C; E],  d(L^-1) = -L^-1 (dL) L^-1.
With tau fixed only the (kappa^-1 q, v) block A of L_K depends on theta_K, and
d(kappa^-1)/dtheta = -kappa^-1: dL = [[-A, 0], [0, 0]]. With tau_K = kappa_K
the tau-proportional pieces vary too (d tau/dtheta = tau): D and E of L_K and
CE, the tau H half of GH and tau Ml, so dL also has D in its (u, u) block,
dCE = [0; E], dGH = [0, tau H] and d(tau Ml) = tau Ml.
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import hdg
from . import quadrature as qd


def gradients(prob, f_q, lam_obs):
    """Return (J, lam, dJ/dtheta [nel], dJ/df_q [nel, p+2, p+2])."""
    nel, n = prob.mesh.nel, prob.ref.n
    b = prob.condense_rhs(f_q)
    A_int, idx = prob.assemble_interior()
    lu = spla.splu(A_int.tocsc())
    lam = np.zeros(prob.ndof)
    lam[idx] = lu.solve(b[idx])
    res = lam - lam_obs
    res_b = np.zeros_like(res)
    res_b[idx] = res[idx]           # J only sees interior dofs (boundary trace is fixed)
    J = 0.5 * float(res_b @ res_b)
    psi = np.zeros(prob.ndof)
    psi[idx] = lu.solve(res_b[idx])
    F = prob.load_vectors(f_q)
    # F = Vf^T (wJ f_q): the load map used by the condensed right-hand side
    xq, wq = qd.gauss_legendre(prob.p + 2)
    B1 = qd.lagrange_matrix(prob.ref.vnodes, xq)
    Vf = np.kron(B1, B1)
    wJf = np.kron(wq, wq) * prob.mesh.hx * prob.mesh.hy / 4.0
    dtheta = np.zeros(nel)
    df = np.zeros((nel, (prob.p + 2) ** 2))
    for e in range(nel):
        mt = prob.mats(e)
        L = hdg.local_system(mt)
        CE = np.vstack([mt["C"], mt["E"]])
        GH = np.hstack([mt["G"], mt["tau"] * mt["H"]])
        dL = np.zeros_like(L)
        dL[:2 * n, :2 * n] = -mt["A"]
        dCE = np.zeros_like(CE)
        dGH = np.zeros_like(GH)
        dMl = np.zeros_like(mt["Ml"])
        if prob.tau == "kappa":
            dL[2 * n:, 2 * n:] = mt["D"]
            dCE[2 * n:] = mt["E"]
            dGH[:, 2 * n:] = mt["tau"] * mt["H"]
            dMl = mt["tau"] * mt["Ml"]
        rhsF = np.zeros(3 * n)
        rhsF[2 * n:] = F[e]
        Linv_CE = np.linalg.solve(L, CE)
        Linv_F = np.linalg.solve(L, rhsF)
        GH_Linv = np.linalg.solve(L.T, GH.T).T
        dS = dGH @ Linv_CE - GH_Linv @ dL @ Linv_CE + GH_Linv @ dCE + dMl
        db = dGH @ Linv_F - GH_Linv @ dL @ Linv_F
        d = prob.dofs(e)
        dtheta[e] = psi[d] @ (db - dS @ lam[d])
        # db_K/dF = GH L^-1 [0; I]  ->  dJ/dF_K = [0 I] L^-T GH^T psi_K
        dJdF = GH_Linv[:, 2 * n:].T @ psi[d]
        df[e] = wJf * (Vf @ dJdF)
    return J, lam, dtheta, df.reshape(nel, prob.p + 2, prob.p + 2)


def objective(mesh, p, log_kappa, f_q, lam_obs, tau=1.0):
    """J(theta, f) by a fresh direct solve (for finite differences)."""
    prob = hdg.HDGProblem(mesh, p, np.exp(log_kappa), tau)
    lam = prob.solve_direct(prob.condense_rhs(f_q))
    r = lam - lam_obs
    r[np.setdiff1d(np.arange(prob.ndof), prob.interior_dofs())] = 0.0
    return 0.5 * float(r @ r)
