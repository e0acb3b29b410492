"""GPU parity: every library call against the FP64 CPU oracle on the same seeded
inputs, through the C ABI (ctypes binding). Sizes span several 16-element
segments with a ragged tail, several p- and h-levels, and k = 0..5."""
import numpy as np
import pytest
import torch

from oracle import adjoint as oadj, gmg as ogmg, hdg as ohdg, mesh as omesh
from paper_1705_09907_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_1705_09907_gb300 import hdg
    return hdg


def cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def abs_bound(prob, x):
    """|A| |x| (entrywise), the scale for the apply's rounding-error bound."""
    A, idx = prob.assemble_interior()
    y = np.zeros(prob.ndof)
    y[idx] = abs(A) @ np.abs(x[idx])
    return y


@pytest.mark.parametrize("nx,ny", [(5, 4), (37, 6)])
def test_maps_exact(H, nx, ny):
    m = omesh.Mesh(nx, ny)
    kap = np.ones(m.nel)
    s = H.HDGSolver(nx, ny, 1, cuda(kap))
    e2e, el, fc = (host(t) for t in s.maps())
    oel, ofc = m.edge_to_elem()
    assert np.array_equal(e2e, m.elem_to_edge())
    assert np.array_equal(el, oel) and np.array_equal(fc, ofc)
    s.close()


@pytest.mark.parametrize("reduced", [1, 0])
@pytest.mark.parametrize("prec", ["fp64", "f32x2"])
@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("nx,ny", [(2, 2), (37, 6), (16, 3)])
def test_apply_fp64_vs_assembled(H, k, nx, ny, prec, reduced):
    """reduced = 1: the symmetry-reduced element blocks (two launches); 0: the
    dense owner records. Rectangular elements (hy = 0.7 hx)."""
    m = omesh.Mesh(nx, ny, 0.0, 0.0, 1.0, 0.7)
    kap = np.exp(inputs.gaussian_field(nx, seed=k, corr_len=0.3, ny=ny))
    prob = ohdg.HDGProblem(m, k, kap)
    x = inputs.random_trace(m.n_edges, k, seed=100 + k)    # boundary entries nonzero: must be ignored
    y_ref = prob.apply_assembled(x)
    s = H.HDGSolver(nx, ny, k, cuda(kap), y1=0.7, reduced=reduced)
    y = host(s.apply(cuda(x), prec=prec))
    bound = abs_bound(prob, x)
    # FP64 rounding of a 8(k+1)-term sum plus the two codes' different S_K
    # rounding (the reduced form adds the roundings of F x and F^T u, sums of
    # at most 4 terms each); F32X2 keeps ~48 bits per product and sum (error
    # ~40 * 2^-48)
    assert np.all(np.abs(y - y_ref) <= 1e-12 * bound + 1e-300)
    bnd = np.setdiff1d(np.arange(prob.ndof), prob.interior_dofs())
    assert np.all(y[bnd] == 0.0)
    s.close()


@pytest.mark.parametrize("reduced", [1, 0])
@pytest.mark.parametrize("prec,tol", [("fp32", 3e-6), ("bf16", 1.2e-2)])
@pytest.mark.parametrize("k", [0, 1, 3, 4, 7])
def test_apply_low_precision(H, prec, tol, k, reduced):
    """FP32 blocks: entry rounding 2^-24 plus float accumulation; BF16 blocks:
    entry rounding 2^-9 relative, float accumulation. Bound relative to |A||x|.
    With reduced blocks both float precisions apply the FP32 reduced blocks."""
    nx, ny = 37, 5
    m = omesh.Mesh(nx, ny)
    kap = np.exp(inputs.gaussian_field(nx, seed=7, corr_len=0.3, ny=ny))
    prob = ohdg.HDGProblem(m, k, kap)
    x = inputs.random_trace(m.n_edges, k, seed=3)
    xf = x.astype(np.float32)
    y_ref = prob.apply_assembled(xf.astype(np.float64))
    s = H.HDGSolver(nx, ny, k, cuda(kap), reduced=reduced)
    y = host(s.apply(cuda(xf, torch.float32), prec=prec)).astype(np.float64)
    bound = abs_bound(prob, xf.astype(np.float64))
    assert np.all(np.abs(y - y_ref) <= tol * bound + 1e-30)
    s.close()


def test_apply_multiple_rhs(H):
    nx, ny, k = 21, 7, 2
    m = omesh.Mesh(nx, ny)
    kap = np.exp(inputs.gaussian_field(nx, seed=1, corr_len=0.3, ny=ny))
    X = inputs.random_trace(m.n_edges, k, seed=9, nrhs=5)
    prob = ohdg.HDGProblem(m, k, kap)
    A, idx = prob.assemble_interior()
    s = H.HDGSolver(nx, ny, k, cuda(kap))
    Y = host(s.apply(cuda(X)))
    for r in range(5):
        ref = np.zeros(prob.ndof)
        ref[idx] = A @ X[idx, r]
        assert np.abs(Y[:, r] - ref).max() <= 1e-12 * np.abs(ref).max()
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "f32x2"])
@pytest.mark.parametrize("k,nx,ny", [(1, 16, 16), (3, 24, 12), (4, 32, 16), (0, 8, 8), (2, 37, 10)])
def test_vcycle_fp64_vs_oracle(H, k, nx, ny, prec):
    m = omesh.Mesh(nx, ny)
    kap = np.exp(inputs.gaussian_field(nx, seed=2, corr_len=0.2, ny=ny))
    G = ogmg.NestedGMG(m, k, kap)
    rng = np.random.default_rng(11)
    top = G.plevels[k]
    r = np.zeros(top.ndof)
    r[top.idx] = rng.normal(size=len(top.idx))
    z_ref = G.vcycle(r)
    s = H.HDGSolver(nx, ny, k, cuda(kap))
    assert s.info["n_hlevels"] == len(G.hA) - 1
    z = host(s.vcycle(cuda(r), prec=prec))
    assert np.linalg.norm(z - z_ref) <= (1e-11 if prec == "fp64" else 1e-10) * np.linalg.norm(z_ref)
    # graph replay gives the same result again
    z2 = host(s.vcycle(cuda(r), prec=prec))
    assert np.array_equal(z, z2)
    s.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("bf16", 5e-2)])
def test_vcycle_low_precision(H, prec, tol):
    nx, ny, k = 32, 16, 3
    m = omesh.Mesh(nx, ny)
    kap = np.exp(inputs.gaussian_field(nx, seed=2, corr_len=0.2, ny=ny))
    G = ogmg.NestedGMG(m, k, kap)
    top = G.plevels[k]
    r = np.zeros(top.ndof)
    r[top.idx] = np.random.default_rng(12).normal(size=len(top.idx))
    z_ref = G.vcycle(r)
    s = H.HDGSolver(nx, ny, k, cuda(kap))
    z = host(s.vcycle(cuda(r, torch.float32), prec=prec)).astype(np.float64)
    assert np.linalg.norm(z - z_ref) <= tol * np.linalg.norm(z_ref)
    s.close()


@pytest.mark.parametrize("k,nx,ny", [(1, 16, 16), (2, 24, 12), (4, 16, 8)])
def test_condense_solve_recover_vs_oracle(H, k, nx, ny):
    m = omesh.Mesh(nx, ny)
    kap = np.exp(inputs.gaussian_field(nx, seed=4, corr_len=0.2, ny=ny))
    fq = inputs.fourier_rhs(nx, k, 1, seed=5)[0] if nx == ny else \
        np.random.default_rng(6).normal(size=(m.nel, k + 2, k + 2))
    prob = ohdg.HDGProblem(m, k, kap)
    b_ref = prob.condense_rhs(fq)
    lam_ref = prob.solve_direct(b_ref)
    u_ref, q_ref = prob.recover(lam_ref, fq)
    s = H.HDGSolver(nx, ny, k, cuda(kap))
    b = s.condense_rhs(cuda(fq))
    assert np.abs(host(b) - b_ref).max() <= 1e-12 * np.abs(b_ref).max()
    lam, info = s.solve(b, rtol=1e-14, maxit=100)
    assert info["relres"] <= 1e-14
    lam_h = host(lam)
    assert np.linalg.norm(lam_h - lam_ref) <= 1e-10 * np.linalg.norm(lam_ref)
    u, q = s.recover(lam, cuda(fq))
    assert np.abs(host(u) - u_ref).max() <= 1e-10 * np.abs(u_ref).max()
    assert np.abs(host(q) - q_ref).max() <= 1e-10 * np.abs(q_ref).max()
    s.close()


@pytest.mark.parametrize("inner", ["fp32", "bf16", "f32x2"])
def test_mixed_precision_solve(H, inner):
    nx = ny = 32
    k = 3
    m = omesh.Mesh(nx, ny)
    kap = np.exp(inputs.gaussian_field(nx, seed=0, corr_len=0.05))
    prob = ohdg.HDGProblem(m, k, kap)
    fq = inputs.constant_f(nx, k)
    lam_ref = prob.solve_direct(prob.condense_rhs(fq))
    s = H.HDGSolver(nx, ny, k, cuda(kap))
    b = s.condense_rhs(cuda(fq))
    _, info64 = s.solve(b, rtol=1e-10, maxit=200, inner="fp64")
    lam, info = s.solve(b, rtol=1e-10, maxit=200, inner=inner)
    assert info["relres"] <= 1e-10
    err = np.linalg.norm(host(lam) - lam_ref) / np.linalg.norm(lam_ref)
    assert err <= 1e-7      # residual 1e-10 times the condition number of this mesh
    # the low-precision V-cycle is nearly as good a preconditioner as the FP64 one
    assert info["iterations"] <= info64["iterations"] + (2 if inner != "bf16" else 6)
    s.close()


def test_adjoint_vs_oracle(H):
    nx = ny = 8
    k = 2
    m = omesh.Mesh(nx, ny)
    th = inputs.gaussian_field(nx, seed=0, corr_len=0.2)
    fq = inputs.constant_f(nx, k)
    rng = np.random.default_rng(2)
    lam_obs = rng.normal(size=m.n_edges * (k + 1)) * 1e-3
    J_ref, lam_ref, dth_ref, df_ref = oadj.gradients(ohdg.HDGProblem(m, k, np.exp(th)), fq, lam_obs)
    s = H.HDGSolver(nx, ny, k, cuda(np.exp(th)))
    lam, _ = s.solve(s.condense_rhs(cuda(fq)), rtol=1e-14)
    J, dth, df, psi = s.adjoint_grad(cuda(fq), lam, cuda(lam_obs), rtol=1e-14)
    assert abs(host(J)[0] - J_ref) <= 1e-10 * abs(J_ref)
    assert np.abs(host(dth) - dth_ref).max() <= 1e-8 * np.abs(dth_ref).max()
    assert np.abs(host(df) - df_ref).max() <= 1e-8 * np.abs(df_ref).max()
    s.close()


def test_invalid_arguments(H):
    with pytest.raises(H.HDGError) as e:
        H.HDGSolver(16, 16, 1, cuda(-np.ones(256)))
    assert e.value.status == H.HDG_ERR_INVALID_ARG
    with pytest.raises(H.HDGError):
        H.HDGSolver(1, 16, 1, cuda(np.ones(16)))
    with pytest.raises(H.HDGError):
        H.HDGSolver(4, 4, 9, cuda(np.ones(16)))
    s = H.HDGSolver(4, 4, 1, cuda(np.ones(16)), mixed=0)
    x = torch.zeros(s.ndof, dtype=torch.float32, device="cuda")
    with pytest.raises(H.HDGError) as e:
        s.apply(x, prec="fp32")
    assert e.value.status == H.HDG_ERR_UNSUPPORTED
    s.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("bf16", 5e-2)])
@pytest.mark.parametrize("k,nx,ny", [(5, 12, 10), (6, 9, 8), (7, 8, 6)])
def test_vcycle_low_precision_high_degree(H, prec, tol, k, nx, ny):
    """Float V-cycles at the high degrees (the packed Schwarz blocks of 24..32
    face dofs, the double-float finest correction) against the oracle's FP64
    V-cycle; and the mixed-precision CG reaches the direct solution."""
    m = omesh.Mesh(nx, ny)
    kap = np.exp(inputs.gaussian_field(nx, seed=3, corr_len=0.3, ny=ny))
    G = ogmg.NestedGMG(m, k, kap)
    top = G.plevels[k]
    r = np.zeros(top.ndof)
    r[top.idx] = np.random.default_rng(14).normal(size=len(top.idx))
    z_ref = G.vcycle(r)
    s = H.HDGSolver(nx, ny, k, cuda(kap))
    z = host(s.vcycle(cuda(r, torch.float32), prec=prec)).astype(np.float64)
    assert np.linalg.norm(z - z_ref) <= tol * np.linalg.norm(z_ref)
    prob = G.plevels[k].prob
    fq = np.random.default_rng(15).normal(size=(m.nel, k + 2, k + 2))
    lam_ref = prob.solve_direct(prob.condense_rhs(fq))
    lam, info = s.solve(s.condense_rhs(cuda(fq)), rtol=1e-12, maxit=200, inner=prec)
    assert info["relres"] <= 1e-12
    assert np.linalg.norm(host(lam) - lam_ref) <= 1e-9 * np.linalg.norm(lam_ref)
    s.close()
