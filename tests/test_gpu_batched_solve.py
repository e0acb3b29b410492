"""Many right-hand sides at once (vectors [ndof][nrhs], right-hand side fastest):
the column-batched trace apply against the FP64 oracle's assembled operator, the
batched V-cycle against the oracle's V-cycle column by column, and the batched
CG against the oracle's direct solve. Meshes have ragged record segments and
column counts that are not multiples of 32."""
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
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("reduced", [1, 0])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("f32x2", 1e-12), ("fp32", 3e-6), ("bf16", 1.2e-2)])
@pytest.mark.parametrize("k,nb", [(0, 2), (1, 33), (3, 64), (2, 128), (5, 7), (7, 3)])
def test_column_apply_vs_assembled(prec, tol, k, nb, reduced):
    """FP64 / F32X2: rounding of an 8(k+1)-term sum (~48 bits for F32X2); FP32 and
    BF16 blocks: entry rounding 2^-24 / 2^-9 with FP32 accumulation. Bound
    relative to |A||x| per entry; boundary rows of x are nonzero and ignored.
    reduced = 1: the reduced-block column kernels; 0: the dense column kernel."""
    from paper_1705_09907_gb300 import hdg
    nx, ny = 37, 6
    m = omesh.Mesh(nx, ny)
    kap = np.exp(inputs.gaussian_field(nx, seed=k, corr_len=0.3, ny=ny))
    prob = ohdg.HDGProblem(m, k, kap)
    A, idx = prob.assemble_interior()
    X = inputs.random_trace(m.n_edges, k, seed=40 + k, nrhs=nb)
    dt = torch.float64 if prec in ("fp64", "f32x2") else torch.float32
    Xd = cuda(X, dt)
    Xh = host(Xd)
    s = hdg.HDGSolver(nx, ny, k, cuda(kap), reduced=reduced)
    Y = host(s.apply(Xd, prec=prec))
    ref = np.zeros_like(Xh)
    ref[idx] = A @ Xh[idx]
    bound = np.zeros_like(Xh)
    bound[idx] = abs(A) @ np.abs(Xh[idx])
    assert np.all(np.abs(Y - ref) <= tol * bound + 1e-300)
    bnd = np.setdiff1d(np.arange(prob.ndof), idx)
    assert np.all(Y[bnd] == 0.0)
    # the column kernel and the single-vector kernel agree column by column
    for j in (0, nb - 1):
        yj = host(s.apply(Xd[:, j].contiguous(), prec=prec))
        assert np.all(np.abs(Y[:, j] - yj) <= 2 * tol * bound[:, j] + 1e-300)
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "f32x2", "fp32"])
@pytest.mark.parametrize("k,nx,ny,nb", [(3, 24, 12, 5), (1, 16, 16, 40), (0, 8, 8, 3), (2, 37, 10, 2)])
def test_batched_vcycle_vs_oracle(prec, k, nx, ny, nb):
    from paper_1705_09907_gb300 import hdg
    m = omesh.Mesh(nx, ny)
    kap = np.exp(inputs.gaussian_field(nx, seed=2, corr_len=0.2, ny=ny))
    G = ogmg.NestedGMG(m, k, kap)
    top = G.plevels[k]
    rng = np.random.default_rng(13)
    R = np.zeros((top.ndof, nb))
    R[top.idx] = rng.normal(size=(len(top.idx), nb))
    dt = torch.float64 if prec in ("fp64", "f32x2") else torch.float32
    s = hdg.HDGSolver(nx, ny, k, cuda(kap))
    Z = host(s.vcycle(cuda(R, dt), prec=prec))
    tol = {"fp64": 1e-11, "f32x2": 1e-10, "fp32": 1e-4}[prec]
    for j in range(nb):
        z_ref = G.vcycle(R[:, j])
        assert np.linalg.norm(Z[:, j] - z_ref) <= tol * np.linalg.norm(z_ref)
    # a second call replays the captured batched cycle: same result
    Z2 = host(s.vcycle(cuda(R, dt), prec=prec))
    assert np.array_equal(Z, Z2)
    s.close()


@pytest.mark.parametrize("inner", ["fp64", "fp32", "f32x2", "bf16"])
def test_batched_solve_vs_oracle(inner):
    """6 Fourier right-hand sides plus one zero column on 32 x 32, k = 3,
    lognormal kappa: every column reaches relative residual 1e-10 and matches the
    oracle's direct solve (the zero column stays exactly 0); the batch takes as
    many iterations as the slowest single solve, within 2."""
    from paper_1705_09907_gb300 import hdg
    nx = ny = 32
    k = 3
    nb = 7
    m = omesh.Mesh(nx, ny)
    kap = np.exp(inputs.gaussian_field(nx, seed=0, corr_len=0.05))
    prob = ohdg.HDGProblem(m, k, kap)
    F = np.concatenate([inputs.fourier_rhs(nx, k, nb - 1, seed=3), np.zeros((1, m.nel, k + 2, k + 2))])
    s = hdg.HDGSolver(nx, ny, k, cuda(kap))
    B = s.condense_rhs(cuda(F))
    assert tuple(B.shape) == (prob.ndof, nb)
    rtol = 1e-10
    lam, info = s.solve(B, rtol=rtol, maxit=200, inner=inner)
    assert info["relres"] <= rtol
    L = host(lam)
    Bh = host(B)
    assert np.all(L[:, nb - 1] == 0.0)
    its_single = []
    for j in range(nb - 1):
        lam_ref = prob.solve_direct(Bh[:, j])
        err = np.linalg.norm(L[:, j] - lam_ref) / np.linalg.norm(lam_ref)
        assert err <= 1e-7       # residual 1e-10 times the condition number of this mesh
        _, inf1 = s.solve(B[:, j].contiguous(), rtol=rtol, maxit=200, inner=inner)
        its_single.append(inf1["iterations"])
    assert info["iterations"] <= max(its_single) + 2
    s.close()


def test_batched_solve_reuses_and_replaces_work():
    """Two batch sizes in turn on one context (work vectors replaced), then the
    first again: results identical to the first call."""
    from paper_1705_09907_gb300 import hdg
    nx = ny = 16
    k = 2
    m = omesh.Mesh(nx, ny)
    s = hdg.HDGSolver(nx, ny, k, cuda(np.ones(m.nel)))
    F = inputs.fourier_rhs(nx, k, 4, seed=8)
    B4 = s.condense_rhs(cuda(F))
    B2 = B4[:, :2].contiguous()
    l4a, _ = s.solve(B4, rtol=1e-10)
    l2, _ = s.solve(B2, rtol=1e-10)
    l4b, _ = s.solve(B4, rtol=1e-10)
    assert torch.equal(l4a, l4b)
    assert torch.allclose(l2, l4a[:, :2], rtol=0, atol=1e-8 * float(l4a.abs().max()))
    s.close()
