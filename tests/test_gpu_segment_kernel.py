"""The one-CTA-per-segment apply kernel (forced with autotune = 2 / 3 / 4:
8 / 4 / 2 warps) against the FP64 oracle's assembled operator and against the ring
kernel (autotune = 0), for every degree, all four precisions and ragged
segments; then the residual form y = c - A x inside a V-cycle, and a solve.
reduced = 0 throughout, so the condensed blocks also go through these kernels."""
import numpy as np
import pytest
import torch

from oracle import gmg as ogmg, hdg as ohdg, mesh as omesh
from paper_1705_09907_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "f32x2": 1e-12, "fp32": 3e-6, "bf16": 1.2e-2}


def cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("mode", [2, 3, 4])
@pytest.mark.parametrize("prec", ["fp64", "f32x2", "fp32", "bf16"])
@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("nx,ny", [(37, 6), (16, 3)])
def test_segment_apply_vs_assembled(prec, k, nx, ny, mode):
    from paper_1705_09907_gb300 import hdg
    m = omesh.Mesh(nx, ny, 0.0, 0.0, 1.0, 0.7)
    kap = np.exp(inputs.gaussian_field(nx, seed=k, corr_len=0.3, ny=ny))
    prob = ohdg.HDGProblem(m, k, kap)
    A, idx = prob.assemble_interior()
    dt = torch.float64 if prec in ("fp64", "f32x2") else torch.float32
    xd = cuda(inputs.random_trace(m.n_edges, k, seed=70 + k), dt)
    x = host(xd)
    seg = hdg.HDGSolver(nx, ny, k, cuda(kap), y1=0.7, autotune=mode, reduced=0)
    ring = hdg.HDGSolver(nx, ny, k, cuda(kap), y1=0.7, autotune=0, reduced=0)
    y = host(seg.apply(xd, prec=prec))
    ref = np.zeros(prob.ndof)
    ref[idx] = A @ x[idx]
    bound = np.zeros(prob.ndof)
    bound[idx] = abs(A) @ np.abs(x[idx])
    tol = TOL[prec]
    assert np.all(np.abs(y - ref) <= tol * bound + 1e-300)
    assert np.all(y[np.setdiff1d(np.arange(prob.ndof), idx)] == 0.0)
    y_ring = host(ring.apply(xd, prec=prec))
    assert np.all(np.abs(y - y_ring) <= 2 * tol * bound + 1e-300)
    seg.close()
    ring.close()


@pytest.mark.parametrize("mode", [2, 3, 4])
@pytest.mark.parametrize("k", [1, 3, 4])
def test_segment_vcycle_and_solve(k, mode):
    """V-cycle (residual-form applies y = c - A x and Schwarz blocks) against the
    oracle's V-cycle, and a solve to 1e-12 against the oracle's direct solve."""
    from paper_1705_09907_gb300 import hdg
    nx, ny = 24, 16
    m = omesh.Mesh(nx, ny)
    kap = np.exp(inputs.gaussian_field(nx, seed=5, corr_len=0.2, ny=ny))
    G = ogmg.NestedGMG(m, k, kap)
    top = G.plevels[k]
    r = np.zeros(top.ndof)
    r[top.idx] = np.random.default_rng(21).normal(size=len(top.idx))
    s = hdg.HDGSolver(nx, ny, k, cuda(kap), autotune=mode, reduced=0)
    for prec, tol in (("fp64", 1e-11), ("f32x2", 1e-10)):
        z = host(s.vcycle(cuda(r), prec=prec))
        z_ref = G.vcycle(r)
        assert np.linalg.norm(z - z_ref) <= tol * np.linalg.norm(z_ref)
    prob = ohdg.HDGProblem(m, k, kap)
    fq = np.random.default_rng(22).normal(size=(m.nel, k + 2, k + 2))
    b_ref = prob.condense_rhs(fq)
    lam_ref = prob.solve_direct(b_ref)
    lam, info = s.solve(s.condense_rhs(cuda(fq)), rtol=1e-12, maxit=100)
    assert info["relres"] <= 1e-12
    assert np.linalg.norm(host(lam) - lam_ref) <= 1e-9 * np.linalg.norm(lam_ref)
    s.close()
