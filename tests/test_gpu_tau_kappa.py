"""The tau_K = kappa_K variant (hdg_options.tau_kappa = 1) against the FP64
oracle run with tau = "kappa": the condensed operator (reduced and dense
blocks), the condensed right-hand side, the solve, the recovery, the V-cycle
and the adjoint gradient, on a rectangular-element mesh with a lognormal
coefficient (ragged record segments and several reduced-apply tiles)."""
import numpy as np
import pytest
import torch

from oracle import adjoint as oadj, gmg as ogmg, hdg as ohdg, mesh as omesh
from paper_1705_09907_gb300 import inputs

pytestmark = pytest.mark.gpu


def cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("k", [0, 1, 3, 4])
def test_apply_condense_solve_recover(k):
    from paper_1705_09907_gb300 import hdg
    nx, ny = 37, 10
    m = omesh.Mesh(nx, ny, 0.0, 0.0, 1.0, 0.6)
    kap = np.exp(1.5 * inputs.gaussian_field(nx, seed=k, corr_len=0.2, ny=ny))
    prob = ohdg.HDGProblem(m, k, kap, "kappa")
    A, idx = prob.assemble_interior()
    x = inputs.random_trace(m.n_edges, k, seed=300 + k)
    ref = np.zeros(prob.ndof)
    ref[idx] = A @ x[idx]
    bound = np.zeros(prob.ndof)
    bound[idx] = abs(A) @ np.abs(x[idx])
    fq = np.random.default_rng(9 + k).normal(size=(m.nel, k + 2, k + 2))
    b_ref = prob.condense_rhs(fq)
    lam_ref = prob.solve_direct(b_ref)
    u_ref, q_ref = prob.recover(lam_ref, fq)
    for reduced in (1, 0):
        s = hdg.HDGSolver(nx, ny, k, cuda(kap), y1=0.6, tau_kappa=1, reduced=reduced)
        for prec, tol in (("fp64", 1e-12), ("fp32", 3e-6)):
            dt = torch.float64 if prec == "fp64" else torch.float32
            xd = cuda(x, dt)
            xh = host(xd)
            r2 = np.zeros(prob.ndof)
            r2[idx] = A @ xh[idx]
            b2 = np.zeros(prob.ndof)
            b2[idx] = abs(A) @ np.abs(xh[idx])
            y = host(s.apply(xd, prec=prec))
            assert np.all(np.abs(y - r2) <= tol * b2 + 1e-300), (reduced, prec)
        b = s.condense_rhs(cuda(fq))
        assert np.abs(host(b) - b_ref).max() <= 1e-12 * np.abs(b_ref).max()
        lam, info = s.solve(b, rtol=1e-13, maxit=200)
        assert info["relres"] <= 1e-13
        assert np.linalg.norm(host(lam) - lam_ref) <= 1e-9 * np.linalg.norm(lam_ref)
        u, q = s.recover(lam, cuda(fq))
        assert np.abs(host(u) - u_ref).max() <= 1e-9 * np.abs(u_ref).max()
        assert np.abs(host(q) - q_ref).max() <= 1e-9 * np.abs(q_ref).max()
        s.close()


@pytest.mark.parametrize("k,nx,ny", [(2, 24, 12), (4, 16, 16)])
def test_vcycle_vs_oracle(k, nx, ny):
    from paper_1705_09907_gb300 import hdg
    m = omesh.Mesh(nx, ny)
    kap = np.exp(inputs.gaussian_field(nx, seed=6, corr_len=0.2, ny=ny))
    G = ogmg.NestedGMG(m, k, kap, tau="kappa")
    top = G.plevels[k]
    r = np.zeros(top.ndof)
    r[top.idx] = np.random.default_rng(17).normal(size=len(top.idx))
    s = hdg.HDGSolver(nx, ny, k, cuda(kap), tau_kappa=1)
    z = host(s.vcycle(cuda(r)))
    z_ref = G.vcycle(r)
    assert np.linalg.norm(z - z_ref) <= 1e-11 * np.linalg.norm(z_ref)
    s.close()


def test_adjoint_vs_oracle():
    """dJ/dlog(kappa) = -psi_K^T S_K lambda_K (b_K does not depend on kappa when
    tau_K = kappa_K) and dJ/df = w_q |J| u(psi, 0)(x_q), against the oracle's
    general derivative of the local system."""
    from paper_1705_09907_gb300 import hdg
    nx, ny, k = 12, 10, 2
    m = omesh.Mesh(nx, ny)
    th = inputs.gaussian_field(nx, seed=2, corr_len=0.2, ny=ny)
    fq = np.random.default_rng(3).normal(size=(m.nel, k + 2, k + 2))
    lam_obs = np.random.default_rng(4).normal(size=m.n_edges * (k + 1)) * 1e-2
    J_ref, lam_ref, dth_ref, df_ref = oadj.gradients(ohdg.HDGProblem(m, k, np.exp(th), "kappa"), fq, lam_obs)
    for reduced in (1, 0):
        s = hdg.HDGSolver(nx, ny, k, cuda(np.exp(th)), tau_kappa=1, reduced=reduced)
        lam, _ = s.solve(s.condense_rhs(cuda(fq)), rtol=1e-14, maxit=200)
        J, dth, df, _ = s.adjoint_grad(cuda(fq), lam, cuda(lam_obs), rtol=1e-14, maxit=200)
        assert abs(J.item() - J_ref) <= 1e-10 * abs(J_ref)
        assert np.abs(host(dth) - dth_ref).max() <= 1e-8 * np.abs(dth_ref).max()
        assert np.abs(host(df) - df_ref).max() <= 1e-8 * np.abs(df_ref).max()
        s.close()
