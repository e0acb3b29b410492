"""Degenerate and extreme inputs through the C ABI, against the FP64 oracle:
a zero source (the solution is exactly zero and CG stops before iterating), the
smallest mesh (2 x 2: one interior vertex on the only Q1 level), the highest
degree (k = 7), skinny and odd meshes (a single Q1 level, coarse solve on the
mesh itself), a coefficient contrast of 1e8 across a checkerboard, and a batch
whose columns repeat one right-hand side."""
import numpy as np
import pytest
import torch

from oracle import gmg as ogmg, hdg as ohdg, mesh as omesh
from paper_1705_09907_gb300 import inputs

pytestmark = pytest.mark.gpu


def cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("inner", ["fp64", "fp32"])
def test_zero_source_gives_zero_trace(inner):
    from paper_1705_09907_gb300 import hdg
    n, k = 12, 2
    s = hdg.HDGSolver(n, n, k, cuda(np.ones(n * n)))
    b = s.condense_rhs(cuda(np.zeros((n * n, k + 2, k + 2))))
    assert float(b.abs().max()) == 0.0
    lam, info = s.solve(b, rtol=1e-10, inner=inner)
    assert info["iterations"] == 0 and info["relres"] == 0.0
    assert float(lam.abs().max()) == 0.0
    u, q = s.recover(lam, cuda(np.zeros((n * n, k + 2, k + 2))))
    assert float(u.abs().max()) == 0.0 and float(q.abs().max()) == 0.0
    s.close()


@pytest.mark.parametrize("nx,ny,k", [(2, 2, 1), (2, 2, 7), (3, 17, 2), (5, 64, 3), (9, 9, 7)])
def test_small_odd_and_high_degree_meshes(nx, ny, k):
    """Solve to 1e-13 and compare with the oracle's direct solve; the V-cycle
    against the oracle's V-cycle."""
    from paper_1705_09907_gb300 import hdg
    m = omesh.Mesh(nx, ny)
    kap = np.exp(inputs.gaussian_field(nx, seed=3, corr_len=0.4, ny=ny))
    prob = ohdg.HDGProblem(m, k, kap)
    fq = np.random.default_rng(nx * 100 + ny).normal(size=(m.nel, k + 2, k + 2))
    lam_ref = prob.solve_direct(prob.condense_rhs(fq))
    s = hdg.HDGSolver(nx, ny, k, cuda(kap))
    lam, info = s.solve(s.condense_rhs(cuda(fq)), rtol=1e-13, maxit=300)
    assert info["relres"] <= 1e-13
    assert np.linalg.norm(host(lam) - lam_ref) <= 1e-9 * np.linalg.norm(lam_ref)
    G = ogmg.NestedGMG(m, k, kap)
    top = G.plevels[k]
    r = np.zeros(top.ndof)
    r[top.idx] = np.random.default_rng(7).normal(size=len(top.idx))
    z = host(s.vcycle(cuda(r)))
    z_ref = G.vcycle(r)
    assert np.linalg.norm(z - z_ref) <= 1e-11 * np.linalg.norm(z_ref)
    s.close()


@pytest.mark.parametrize("inner", ["fp64", "fp32", "bf16"])
def test_high_contrast_checkerboard(inner):
    """kappa alternates 1e-4 / 1e4 between 4 x 4 blocks of elements on 32 x 32,
    k = 2: every precision reaches 1e-10 and agrees with the oracle's direct solve
    to the accuracy the condition number allows."""
    from paper_1705_09907_gb300 import hdg
    n, k = 32, 2
    I, J = np.meshgrid(np.arange(n), np.arange(n))
    kap = np.where(((I // 4) + (J // 4)) % 2 == 0, 1e-4, 1e4).ravel().astype(np.float64)
    m = omesh.Mesh(n, n)
    prob = ohdg.HDGProblem(m, k, kap)
    fq = inputs.constant_f(n, k)
    lam_ref = prob.solve_direct(prob.condense_rhs(fq))
    s = hdg.HDGSolver(n, n, k, cuda(kap))
    lam, info = s.solve(s.condense_rhs(cuda(fq)), rtol=1e-10, maxit=500, inner=inner)
    assert info["relres"] <= 1e-10
    err = np.linalg.norm(host(lam) - lam_ref) / np.linalg.norm(lam_ref)
    assert err <= 1e-5
    s.close()


def test_repeated_columns_match_single_solve():
    """A batch of 33 identical columns: every column equals the single-vector
    solve of that right-hand side to rounding (the column kernels sum in another
    order), and all columns are bitwise equal to each other."""
    from paper_1705_09907_gb300 import hdg
    n, k, nb = 24, 3, 33
    s = hdg.HDGSolver(n, n, k, cuda(np.exp(inputs.gaussian_field(n, seed=9, corr_len=0.2))))
    b = s.condense_rhs(cuda(inputs.fourier_rhs(n, k, 1, seed=2)[0]))
    B = b[:, None].repeat(1, nb).contiguous()
    L, info = s.solve(B, rtol=1e-12, maxit=200)
    lam, info1 = s.solve(b, rtol=1e-12, maxit=200)
    assert abs(info["iterations"] - info1["iterations"]) <= 1
    Lh = host(L)
    assert all(np.array_equal(Lh[:, 0], Lh[:, j]) for j in range(1, nb))
    assert np.linalg.norm(Lh[:, 0] - host(lam)) <= 1e-10 * np.linalg.norm(host(lam))
    s.close()
