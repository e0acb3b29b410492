"""The symmetry-reduced condensed-block apply: the two-launch form
(reduced = 1) and the tile form (reduced = 2) give bitwise-identical
results, both equal the FP64 oracle's assembled operator, on meshes with
ragged tiles in both directions (tiles are 32 elements wide and 8 high) and on
single-tile meshes; then V-cycles (residual form y = c - A x on every p-level)
of the two forms agree bitwise and match the oracle's V-cycle."""
import numpy as np
import pytest
import torch

from oracle import gmg as ogmg, hdg as ohdg, mesh as omesh
from paper_1705_09907_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "f32x2": 1e-12, "fp32": 3e-6, "bf16": 3e-6}


def cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("nx,ny", [(70, 19), (33, 9), (31, 8), (2, 2), (5, 40)])
def test_tile_and_two_launch_forms_vs_assembled(k, nx, ny):
    from paper_1705_09907_gb300 import hdg
    m = omesh.Mesh(nx, ny, 0.0, 0.0, 1.0, 0.7)
    kap = np.exp(inputs.gaussian_field(nx, seed=k, corr_len=0.3, ny=ny))
    prob = ohdg.HDGProblem(m, k, kap)
    A, idx = prob.assemble_interior()
    two = hdg.HDGSolver(nx, ny, k, cuda(kap), y1=0.7, reduced=1)
    tile = hdg.HDGSolver(nx, ny, k, cuda(kap), y1=0.7, reduced=2)
    one_tile = nx <= 32 and ny <= 8
    assert tile.info["apply_kernels"] == (1 if one_tile else 2)
    assert two.info["apply_kernels"] == 2
    bnd = np.setdiff1d(np.arange(prob.ndof), idx)
    for prec in ("fp64", "f32x2", "fp32", "bf16"):
        dt = torch.float64 if prec in ("fp64", "f32x2") else torch.float32
        xd = cuda(inputs.random_trace(m.n_edges, k, seed=200 + k), dt)
        x = host(xd)
        y1 = tile.apply(xd, prec=prec)
        y2 = two.apply(xd, prec=prec)
        assert torch.equal(y1, y2), prec
        y = host(y1)
        ref = np.zeros(prob.ndof)
        ref[idx] = A @ x[idx]
        bound = np.zeros(prob.ndof)
        bound[idx] = abs(A) @ np.abs(x[idx])
        assert np.all(np.abs(y - ref) <= TOL[prec] * bound + 1e-300), prec
        assert np.all(y[bnd] == 0.0)
    tile.close()
    two.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k,nx,ny", [(4, 40, 20), (2, 66, 18), (7, 12, 12)])
def test_vcycle_forms_agree_and_match_oracle(prec, k, nx, ny):
    from paper_1705_09907_gb300 import hdg
    m = omesh.Mesh(nx, ny)
    kap = np.exp(inputs.gaussian_field(nx, seed=4, corr_len=0.2, ny=ny))
    G = ogmg.NestedGMG(m, k, kap)
    top = G.plevels[k]
    r = np.zeros(top.ndof)
    r[top.idx] = np.random.default_rng(31).normal(size=len(top.idx))
    z_ref = G.vcycle(r)
    dt = torch.float64 if prec == "fp64" else torch.float32
    zs = []
    for red in (1, 2):
        # autotune = 3: both contexts apply the Schwarz blocks with the same
        # kernel (the autotuner could pick differently ordered sums)
        s = hdg.HDGSolver(nx, ny, k, cuda(kap), reduced=red, autotune=3)
        zs.append(s.vcycle(cuda(r, dt), prec=prec))
        s.close()
    assert torch.equal(zs[0], zs[1])
    z = host(zs[0])
    tol = 1e-11 if prec == "fp64" else 1e-4
    assert np.linalg.norm(z - z_ref) <= tol * np.linalg.norm(z_ref)


@pytest.mark.parametrize("prec", ["fp64", "f32x2"])
@pytest.mark.parametrize("k,nb", [(0, 3), (2, 33), (4, 64), (7, 5)])
def test_column_kernels_equal_single_vector_applies(prec, k, nb):
    """The reduced column kernels (nb right-hand sides, right-hand side
    fastest; used for double vectors) do per column exactly the arithmetic of
    the one-vector reduced apply: every column is bitwise equal to its own
    single apply."""
    from paper_1705_09907_gb300 import hdg
    nx, ny = 45, 11
    m = omesh.Mesh(nx, ny)
    kap = np.exp(inputs.gaussian_field(nx, seed=k, corr_len=0.3, ny=ny))
    dt = torch.float64
    s = hdg.HDGSolver(nx, ny, k, cuda(kap))
    X = cuda(inputs.random_trace(m.n_edges, k, seed=400 + k, nrhs=nb), dt)
    Y = s.apply(X, prec=prec)
    for j in range(nb):
        assert torch.equal(Y[:, j], s.apply(X[:, j].contiguous(), prec=prec)), j
    s.close()
