"""Full-size checks in the benchmark's launch configuration, on sampled outputs
the oracle computes one by one from its own element blocks:
  * 512 x 512, k = 4, lognormal kappa (seed 0), f = 1, FP64 V-cycle: the trace
    apply at 300 sampled interior edges, the condensed right-hand side there,
    and the residual of the solve there;
  * 1024 x 1024, k = 3, same generator, FP32 V-cycle (mixed): the same checks,
    and agreement with the FP64-preconditioned solve.
Residual bound per row: rtol |b|_2 (the CG stopping rule on the updated
residual) plus the rounding of a recomputed residual, which is of order
eps * (8(k+1) terms) * (|S||lambda|)_row times the drift that accumulates over
the iterations; 1e-13 (|S||lambda|)_row covers both (at 512^2 the rounding term
alone is already ~1e-10 |b|_2, growing like h^-2)."""
import numpy as np
import pytest
import torch

from oracle import hdg as ohdg, mesh as omesh
from paper_1705_09907_gb300 import inputs

pytestmark = pytest.mark.gpu


def _oracle_edge_rows(m, k, kappa, fq, edges, tau=1.0):
    """For each sampled interior edge, per adjacent element: (S_K rows of the
    edge, the element's global dofs, b_K rows of the edge)."""
    el, fc = m.edge_to_elem()
    prob = ohdg.HDGProblem(m, k, kappa, tau)
    out = []
    for e in edges:
        rows = []
        for side in (0, 1):
            K, f = el[e, side], fc[e, side]
            mt = prob.mats(K)
            S = ohdg.schur_block(mt)
            bK = ohdg.rhs_block(mt, ohdg.load_vector(prob.ref, mt, fq[K]))
            sl = slice(f * (k + 1), (f + 1) * (k + 1))
            rows.append((S[sl], prob.dofs(K), bK[sl]))
        out.append(rows)
    return out, prob


@pytest.mark.parametrize("N,k,inner", [(512, 4, "fp64"), (1024, 3, "fp32")])
def test_fullsize_apply_condense_solve_sampled(N, k, inner):
    from paper_1705_09907_gb300 import hdg
    m = omesh.Mesh(N, N)
    kappa = inputs.lognormal_kappa(N, 0)
    fq = inputs.constant_f(N, k)
    edges = np.random.default_rng(N + k).choice(m.interior_edges(), size=300, replace=False)
    rows, prob = _oracle_edge_rows(m, k, kappa, fq, edges)
    boundary = np.setdiff1d(np.arange(prob.ndof), prob.interior_dofs())
    n1 = k + 1
    s = hdg.HDGSolver(N, N, k, torch.as_tensor(kappa, device="cuda"))
    # apply: boundary entries of x are nonzero and must be ignored
    x = inputs.random_trace(m.n_edges, k, seed=7)
    y = s.apply(torch.as_tensor(x, device="cuda")).cpu().numpy()
    xm = x.copy()
    xm[boundary] = 0.0
    for e, rr in zip(edges, rows):
        ref = sum(S @ xm[d] for S, d, _ in rr)
        scale = sum(np.abs(S) @ np.abs(xm[d]) for S, d, _ in rr)
        assert np.all(np.abs(y[e * n1:(e + 1) * n1] - ref) <= 1e-12 * scale)
    # condensed right-hand side
    b = s.condense_rhs(torch.as_tensor(fq, device="cuda"))
    b_h = b.cpu().numpy()
    bmax, b2 = np.abs(b_h).max(), np.linalg.norm(b_h)
    for e, rr in zip(edges, rows):
        assert np.abs(b_h[e * n1:(e + 1) * n1] - sum(bk for _, _, bk in rr)).max() <= 1e-12 * bmax
    # solve: residual of the GPU lambda in the oracle's operator at the sampled rows
    rtol = 1e-10
    lam, info = s.solve(b, rtol=rtol, maxit=400, inner=inner)
    assert info["relres"] <= rtol
    lam_h = lam.cpu().numpy()
    assert np.all(lam_h[boundary] == 0.0)
    for e, rr in zip(edges, rows):
        res = sum(bk for _, _, bk in rr) - sum(S @ lam_h[d] for S, d, _ in rr)
        absl = sum(np.abs(S) @ np.abs(lam_h[d]) for S, d, _ in rr)
        assert np.all(np.abs(res) <= rtol * b2 + 1e-13 * absl)
    if inner != "fp64":
        lam64, _ = s.solve(b, rtol=rtol, maxit=400, inner="fp64")
        assert float(torch.linalg.norm(lam - lam64) / torch.linalg.norm(lam64)) <= 1e-7
    s.close()


def test_fullsize_batched_solve_sampled():
    """256 x 256, k = 5, kappa = 1, 64 Fourier right-hand sides (seed 3): the
    batched solve with the FP32 V-cycle reaches 1e-10 on every column; at 300
    sampled interior edges the residual of columns 0, 31 and 63 in the oracle's
    operator meets the same per-row bound as above, and column 0 agrees with its
    own plain FP64 solve."""
    from paper_1705_09907_gb300 import hdg
    N, k, nb = 256, 5, 64
    m = omesh.Mesh(N, N)
    kappa = np.ones(m.nel)
    F = inputs.fourier_rhs(N, k, nb, seed=3)
    edges = np.random.default_rng(5).choice(m.interior_edges(), size=300, replace=False)
    cols = (0, 31, 63)
    n1 = k + 1
    s = hdg.HDGSolver(N, N, k, torch.as_tensor(kappa, device="cuda"))
    B = s.condense_rhs(torch.as_tensor(F, device="cuda"))
    rtol = 1e-10
    lam, info = s.solve(B, rtol=rtol, maxit=400, inner="fp32")
    assert info["relres"] <= rtol
    L = lam.cpu().numpy()
    Bh = B.cpu().numpy()
    for j in cols:
        rows, _ = _oracle_edge_rows(m, k, kappa, F[j], edges)
        b2 = np.linalg.norm(Bh[:, j])
        for e, rr in zip(edges, rows):
            b_ref = sum(bk for _, _, bk in rr)
            assert np.abs(Bh[e * n1:(e + 1) * n1, j] - b_ref).max() <= 1e-12 * np.abs(Bh[:, j]).max()
            res = b_ref - sum(S @ L[d, j] for S, d, _ in rr)
            absl = sum(np.abs(S) @ np.abs(L[d, j]) for S, d, _ in rr)
            assert np.all(np.abs(res) <= rtol * b2 + 1e-13 * absl)
    lam0, _ = s.solve(B[:, 0].contiguous(), rtol=rtol, maxit=400, inner="fp64")
    assert float(torch.linalg.norm(lam[:, 0] - lam0) / torch.linalg.norm(lam0)) <= 1e-7
    s.close()


def test_fullsize_uneven_instances_sampled():
    """12 uneven meshes (N in {64, 128, 256, 512}, k in {2, 3, 4}, seed 4),
    kappa = 1, set up in one hdg_setup_batch call and applied in one
    hdg_apply_multi launch as the benchmark does: every instance agrees with its
    own single apply, and at 40 sampled interior edges per instance with the
    oracle's element blocks (FP64 bound of an 8(k+1)-term sum)."""
    from paper_1705_09907_gb300 import hdg
    mix = inputs.instance_mix(12, seed=4)
    sols = hdg.setup_batch([(N, N, k, torch.ones(N * N, dtype=torch.float64, device="cuda")) for N, k in mix],
                           mixed=0)
    xs = [torch.as_tensor(inputs.random_trace(s.n_edges, s.k, seed=60 + q), device="cuda")
          for q, s in enumerate(sols)]
    ys = hdg.apply_multi(sols, xs)
    for q, ((N, k), s, x, y) in enumerate(zip(mix, sols, xs, ys)):
        y1 = s.apply(x)
        yh, y1h = y.cpu().numpy(), y1.cpu().numpy()
        m = omesh.Mesh(N, N)
        edges = np.random.default_rng(100 + q).choice(m.interior_edges(), size=40, replace=False)
        rows, prob = _oracle_edge_rows(m, k, np.ones(m.nel), inputs.constant_f(N, k), edges)
        xm = x.cpu().numpy()
        xm[np.setdiff1d(np.arange(prob.ndof), prob.interior_dofs())] = 0.0
        n1 = k + 1
        for e, rr in zip(edges, rows):
            ref = sum(S @ xm[d] for S, d, _ in rr)
            scale = sum(np.abs(S) @ np.abs(xm[d]) for S, d, _ in rr)
            assert np.all(np.abs(yh[e * n1:(e + 1) * n1] - ref) <= 1e-12 * scale), (q, N, k, e)
            assert np.all(np.abs(yh[e * n1:(e + 1) * n1] - y1h[e * n1:(e + 1) * n1]) <= 2e-12 * scale)
    for s in sols:
        s.close()


def test_fullsize_tau_kappa_sampled():
    """512 x 512, k = 4, lognormal kappa (seed 0), f = 1 with tau_K = kappa_K:
    the reduced apply, the condensed right-hand side and the solve's residual at
    300 sampled interior edges against the oracle's element blocks (tau = kappa),
    as in the tau = 1 check above."""
    from paper_1705_09907_gb300 import hdg
    N, k = 512, 4
    m = omesh.Mesh(N, N)
    kappa = inputs.lognormal_kappa(N, 0)
    fq = inputs.constant_f(N, k)
    edges = np.random.default_rng(77).choice(m.interior_edges(), size=300, replace=False)
    rows, prob = _oracle_edge_rows(m, k, kappa, fq, edges, tau="kappa")
    boundary = np.setdiff1d(np.arange(prob.ndof), prob.interior_dofs())
    n1 = k + 1
    s = hdg.HDGSolver(N, N, k, torch.as_tensor(kappa, device="cuda"), tau_kappa=1)
    x = inputs.random_trace(m.n_edges, k, seed=8)
    y = s.apply(torch.as_tensor(x, device="cuda")).cpu().numpy()
    xm = x.copy()
    xm[boundary] = 0.0
    for e, rr in zip(edges, rows):
        ref = sum(S @ xm[d] for S, d, _ in rr)
        scale = sum(np.abs(S) @ np.abs(xm[d]) for S, d, _ in rr)
        assert np.all(np.abs(y[e * n1:(e + 1) * n1] - ref) <= 1e-12 * scale)
    b = s.condense_rhs(torch.as_tensor(fq, device="cuda"))
    b_h = b.cpu().numpy()
    bmax, b2 = np.abs(b_h).max(), np.linalg.norm(b_h)
    for e, rr in zip(edges, rows):
        assert np.abs(b_h[e * n1:(e + 1) * n1] - sum(bk for _, _, bk in rr)).max() <= 1e-12 * bmax
    rtol = 1e-10
    lam, info = s.solve(b, rtol=rtol, maxit=400)
    assert info["relres"] <= rtol
    lam_h = lam.cpu().numpy()
    for e, rr in zip(edges, rows):
        res = sum(bk for _, _, bk in rr) - sum(S @ lam_h[d] for S, d, _ in rr)
        absl = sum(np.abs(S) @ np.abs(lam_h[d]) for S, d, _ in rr)
        assert np.all(np.abs(res) <= rtol * b2 + 1e-13 * absl)
    s.close()
