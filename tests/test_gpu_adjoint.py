"""Adjoint gradient on the GPU: through torch.autograd against the FP64 oracle's
assembled adjoint and central finite differences, and at full size (512 x 512,
k = 2, lognormal log-kappa) against finite differences on 20 seeded elements."""
import numpy as np
import pytest
import torch

from oracle import adjoint as oadj, hdg as ohdg, mesh as omesh
from paper_1705_09907_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_autograd_matches_oracle_adjoint():
    from paper_1705_09907_gb300.autograd import hdg_solve
    nx = ny = 8
    k = 2
    m = omesh.Mesh(nx, ny)
    th0 = inputs.gaussian_field(nx, seed=0, corr_len=0.2)
    fq0 = np.random.default_rng(4).normal(size=(m.nel, k + 2, k + 2))
    lam_obs = np.random.default_rng(5).normal(size=m.n_edges * (k + 1)) * 1e-3
    th = torch.tensor(th0, device="cuda", requires_grad=True)
    fq = torch.tensor(fq0, device="cuda", requires_grad=True)
    lam = hdg_solve(th, fq, nx, ny, k, rtol=1e-14)
    obs = torch.as_tensor(lam_obs, device="cuda")
    # J sees interior dofs only (boundary entries of lambda are 0 by definition)
    interior = torch.as_tensor(ohdg.HDGProblem(m, k, np.ones(m.nel)).interior_dofs(), device="cuda")
    J = 0.5 * ((lam - obs)[interior] ** 2).sum()
    J.backward()
    J_ref, _, dth_ref, df_ref = oadj.gradients(ohdg.HDGProblem(m, k, np.exp(th0)), fq0, lam_obs)
    assert abs(J.item() - J_ref) <= 1e-10 * abs(J_ref)
    assert np.abs(th.grad.cpu().numpy() - dth_ref).max() <= 1e-8 * np.abs(dth_ref).max()
    assert np.abs(fq.grad.cpu().numpy() - df_ref).max() <= 1e-8 * np.abs(df_ref).max()


def test_autograd_retain_graph_and_dtypes():
    """A graph kept with retain_graph=True differentiates twice (the solver lives
    with the autograd node) with the same gradients, and the gradients come back
    in the inputs' dtypes (float32 sources give a float32 dL/df)."""
    from paper_1705_09907_gb300.autograd import hdg_solve
    nx = ny = 8
    k = 1
    th = torch.tensor(inputs.gaussian_field(nx, seed=0, corr_len=0.2), device="cuda", requires_grad=True)
    fq = torch.tensor(np.random.default_rng(4).normal(size=(nx * ny, k + 2, k + 2)), device="cuda",
                      dtype=torch.float32, requires_grad=True)
    lam = hdg_solve(th, fq, nx, ny, k, rtol=1e-13)
    J = 0.5 * (lam ** 2).sum()
    J.backward(retain_graph=True)
    g1 = (th.grad.clone(), fq.grad.clone())
    assert fq.grad.dtype == torch.float32 and th.grad.dtype == torch.float64
    th.grad = None
    fq.grad = None
    J.backward()
    assert torch.allclose(th.grad, g1[0], rtol=1e-9, atol=0) and torch.allclose(fq.grad, g1[1], rtol=1e-6, atol=0)


def test_adjoint_full_size_vs_finite_differences():
    """512 x 512, k = 2: log kappa = seeded Gaussian field (seed 0), lambda_obs =
    the solve at a second field (seed 1) plus N(0, 1e-3) noise (seed 2), f = 1;
    dJ/dlog(kappa) against central differences on 20 elements drawn with seed 5.
    Step 1e-3: the solves stop at relative residual 1e-13, so J carries ~1e-13
    relative error and a smaller step would drown the per-element derivative
    (about J / nel) in it; the O(h^2) truncation stays ~1e-6 relative."""
    from paper_1705_09907_gb300 import hdg
    N, k = 512, 2
    th = inputs.gaussian_field(N, seed=0)
    fq = torch.as_tensor(inputs.constant_f(N, k), device="cuda")
    s1 = hdg.HDGSolver(N, N, k, torch.as_tensor(np.exp(inputs.gaussian_field(N, seed=1)), device="cuda"))
    lam1, _ = s1.solve(s1.condense_rhs(fq), rtol=1e-13, maxit=400)
    lam_obs = lam1 + torch.as_tensor(inputs.observation_noise(s1.ndof, seed=2), device="cuda")
    _, el, _ = s1.maps()
    interior = ((el[:, 0] >= 0) & (el[:, 1] >= 0)).repeat_interleave(k + 1)
    s1.close()

    def J_of(theta):
        s = hdg.HDGSolver(N, N, k, torch.as_tensor(np.exp(theta), device="cuda"), mixed=0, autotune=0)
        lam, _ = s.solve(s.condense_rhs(fq), rtol=1e-13, maxit=400)
        s.close()
        d = (lam - lam_obs)[interior]
        return 0.5 * float((d * d).sum())

    s = hdg.HDGSolver(N, N, k, torch.as_tensor(np.exp(th), device="cuda"))
    lam, _ = s.solve(s.condense_rhs(fq), rtol=1e-13, maxit=400)
    Jv, dth, _, _ = s.adjoint_grad(fq, lam, lam_obs, rtol=1e-13, maxit=400)
    dth = dth.cpu().numpy()
    s.close()
    assert abs(Jv.item() - J_of(th)) <= 1e-10 * abs(Jv.item())
    elems = np.random.default_rng(5).choice(N * N, size=20, replace=False)
    h = 1e-3
    scale = np.abs(dth).max()
    for e in elems:
        tp, tm = th.copy(), th.copy()
        tp[e] += h
        tm[e] -= h
        fd = (J_of(tp) - J_of(tm)) / (2 * h)
        assert abs(fd - dth[e]) <= 1e-4 * scale + 1e-4 * abs(fd), (e, fd, dth[e])
