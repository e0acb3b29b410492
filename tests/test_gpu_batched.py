"""Tensor-core batched apply (uniform coefficient, shared element block) against
the FP64 oracle's assembled operator applied to the same BF16-rounded inputs.
BF16 blocks carry a relative rounding of 2^-9 per entry and the products are
accumulated in FP32, so the bound is 8e-3 * (|A| |x|) per entry."""
import numpy as np
import pytest
import torch

from oracle import hdg as ohdg, mesh as omesh

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k,nx,ny,nrhs", [(5, 37, 12, 64), (1, 16, 16, 128), (2, 20, 7, 64), (3, 33, 9, 64)])
def test_shared_batched_apply_vs_oracle(k, nx, ny, nrhs):
    from paper_1705_09907_gb300 import hdg
    kappa = 1.7
    m = omesh.Mesh(nx, ny)
    prob = ohdg.HDGProblem(m, k, np.full(m.nel, kappa))
    A, idx = prob.assemble_interior()
    rng = np.random.default_rng(k)
    X = torch.as_tensor(rng.standard_normal((prob.ndof, nrhs)), dtype=torch.bfloat16, device="cuda")
    Xh = X.float().cpu().numpy().astype(np.float64)
    s = hdg.HDGSolver(nx, ny, k, torch.full((m.nel,), kappa, dtype=torch.float64, device="cuda"))
    Y = s.apply_shared_batched(X)
    torch.cuda.synchronize()
    Y = Y.cpu().numpy().astype(np.float64)
    ref = np.zeros_like(Xh)
    ref[idx] = A @ Xh[idx]
    bound = np.zeros_like(Xh)
    bound[idx] = abs(A) @ np.abs(Xh[idx])
    assert np.all(np.abs(Y - ref) <= 8e-3 * bound + 1e-30)
    bnd = np.setdiff1d(np.arange(prob.ndof), idx)
    assert np.all(Y[bnd] == 0.0)
    s.close()


def test_shared_batched_requires_uniform_kappa():
    from paper_1705_09907_gb300 import hdg
    kap = torch.ones(64, dtype=torch.float64, device="cuda")
    kap[5] = 2.0
    s = hdg.HDGSolver(8, 8, 1, kap)
    X = torch.zeros((s.ndof, 64), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(hdg.HDGError) as e:
        s.apply_shared_batched(X)
    assert e.value.status == hdg.HDG_ERR_UNSUPPORTED
    s.close()


@pytest.mark.parametrize("k,nx,ny", [(4, 24, 10), (2, 13, 9)])
def test_shared_batched_tau_kappa_vs_oracle(k, nx, ny):
    """tau_K = kappa_K with a lognormal kappa: every S_K = kappa_K S_ref, one
    shared block with each element's part scaled by its kappa, against the
    oracle's assembled operator of that discretisation on the same BF16 inputs."""
    from paper_1705_09907_gb300 import hdg, inputs
    m = omesh.Mesh(nx, ny)
    kap = np.exp(inputs.gaussian_field(nx, seed=k, corr_len=0.2, ny=ny))
    prob = ohdg.HDGProblem(m, k, kap, tau="kappa")
    A, idx = prob.assemble_interior()
    rng = np.random.default_rng(30 + k)
    X = torch.as_tensor(rng.standard_normal((prob.ndof, 64)), dtype=torch.bfloat16, device="cuda")
    Xh = X.float().cpu().numpy().astype(np.float64)
    s = hdg.HDGSolver(nx, ny, k, torch.as_tensor(kap, device="cuda"), tau_kappa=1)
    Y = s.apply_shared_batched(X)
    torch.cuda.synchronize()
    Y = Y.cpu().numpy().astype(np.float64)
    ref = np.zeros_like(Xh)
    ref[idx] = A @ Xh[idx]
    bound = np.zeros_like(Xh)
    bound[idx] = abs(A) @ np.abs(Xh[idx])
    assert np.all(np.abs(Y - ref) <= 8e-3 * bound + 1e-30)
    bnd = np.setdiff1d(np.arange(prob.ndof), idx)
    assert np.all(Y[bnd] == 0.0)
    s.close()
