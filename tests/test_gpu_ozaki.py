"""FP64 shared-block apply on the tensor cores by exact slice splitting
(hdg_apply_shared_fp64) against the FP64 oracle's assembled operator: every
column within the FP64 rounding of |A||x| (normwise per column, 1e-13), for
k = 1..7, uneven meshes, columns whose scales differ by up to 10^6, two calls in
a row (the slice scratch is reused), and against the CUDA-core FP64 column
apply of the same context."""
import numpy as np
import pytest
import torch

from oracle import hdg as ohdg, mesh as omesh

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k,nx,ny,nrhs", [(1, 9, 7, 64), (3, 21, 10, 64), (4, 16, 16, 128), (5, 13, 11, 64),
                                          (7, 6, 5, 64)])
def test_ozaki_fp64_vs_oracle(k, nx, ny, nrhs):
    from paper_1705_09907_gb300 import hdg
    kappa = 2.3
    m = omesh.Mesh(nx, ny)
    prob = ohdg.HDGProblem(m, k, np.full(m.nel, kappa))
    A, idx = prob.assemble_interior()
    s = hdg.HDGSolver(nx, ny, k, torch.full((m.nel,), kappa, dtype=torch.float64, device="cuda"))
    rng = np.random.default_rng(10 + k)
    for call in range(2):
        X = rng.standard_normal((prob.ndof, nrhs)) * 10.0 ** rng.uniform(-3, 3, size=nrhs)
        Y = s.apply_shared_fp64(torch.as_tensor(X, device="cuda")).cpu().numpy()
        ref = np.zeros_like(X)
        ref[idx] = A @ X[idx]
        bound = np.zeros_like(X)
        bound[idx] = abs(A) @ np.abs(X[idx])
        err = np.linalg.norm(Y - ref, axis=0) / np.linalg.norm(bound, axis=0)
        assert err.max() < 1e-13, err.max()
        bnd = np.setdiff1d(np.arange(prob.ndof), idx)
        assert np.all(Y[bnd] == 0.0)
        # the CUDA-core FP64 column apply of the same operator
        Yc = s.apply(torch.as_tensor(X, device="cuda")).cpu().numpy()
        assert (np.linalg.norm(Y - Yc, axis=0) / np.linalg.norm(bound, axis=0)).max() < 1e-13
    s.close()


def test_ozaki_fp64_requires_uniform_kappa():
    from paper_1705_09907_gb300 import hdg
    kap = torch.ones(64, dtype=torch.float64, device="cuda")
    kap[3] = 2.0
    s = hdg.HDGSolver(8, 8, 2, kap)
    X = torch.zeros((s.ndof, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(hdg.HDGError) as e:
        s.apply_shared_fp64(X)
    assert e.value.status == hdg.HDG_ERR_UNSUPPORTED
    s.close()


@pytest.mark.parametrize("inner", ["fp64", "fp32"])
def test_batched_solve_with_tensor_core_outer_apply(inner):
    """hdg_solve with 64 right-hand sides and a uniform coefficient applies the
    outer operator of the batched CG with hdg_apply_shared_fp64 (tensor_apply =
    1, the default): the solutions match the oracle's direct solves and the
    CUDA-core path (tensor_apply = 0) column by column."""
    from paper_1705_09907_gb300 import hdg, inputs
    nx, ny, k, nb = 24, 16, 3, 64
    m = omesh.Mesh(nx, ny)
    prob = ohdg.HDGProblem(m, k, np.ones(m.nel))
    fq = np.random.default_rng(5).normal(size=(nb, m.nel, k + 2, k + 2))
    kap = torch.ones(m.nel, dtype=torch.float64, device="cuda")
    s1 = hdg.HDGSolver(nx, ny, k, kap)
    s0 = hdg.HDGSolver(nx, ny, k, kap, tensor_apply=0)
    B = s1.condense_rhs(torch.as_tensor(fq, device="cuda"))
    L1, i1 = s1.solve(B, rtol=1e-12, maxit=300, inner=inner)
    L0, i0 = s0.solve(B, rtol=1e-12, maxit=300, inner=inner)
    assert abs(i1["iterations"] - i0["iterations"]) <= 1
    L1h, L0h = L1.cpu().numpy(), L0.cpu().numpy()
    for j in (0, 17, 63):
        ref = prob.solve_direct(prob.condense_rhs(fq[j]))
        nr = np.linalg.norm(ref)
        assert np.linalg.norm(L1h[:, j] - ref) <= 1e-10 * nr
        assert np.linalg.norm(L1h[:, j] - L0h[:, j]) <= 1e-10 * nr
    s1.close()
    s0.close()
