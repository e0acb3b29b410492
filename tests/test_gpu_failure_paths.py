"""Error paths of the library, exercised without faulting the GPU: an
iteration limit (NOT_CONVERGED), non-finite coefficients (INVALID_ARG), a
memory cap (OOM, at set-up and for the batched work of many right-hand sides)
and a bounded device wait that gives up (TIMEOUT, through the wait_probe
option: a barrier that nothing completes), each followed by a call on the same
or a fresh context that still gives the oracle's answer."""
import numpy as np
import pytest
import torch

from oracle import hdg as ohdg, mesh as omesh
from paper_1705_09907_gb300 import inputs

pytestmark = pytest.mark.gpu


def _problem(N=16, k=2, seed=0):
    kap = np.exp(inputs.gaussian_field(N, seed=seed, corr_len=0.2))
    fq = inputs.constant_f(N, k)
    prob = ohdg.HDGProblem(omesh.Mesh(N, N), k, kap)
    lam_ref = prob.solve_direct(prob.condense_rhs(fq))
    return kap, fq, lam_ref


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_not_converged_then_converges():
    from paper_1705_09907_gb300 import hdg
    N, k = 16, 2
    kap, fq, lam_ref = _problem(N, k)
    s = hdg.HDGSolver(N, N, k, torch.as_tensor(kap, device="cuda"))
    b = s.condense_rhs(torch.as_tensor(fq, device="cuda"))
    lam, info = s.solve(b, rtol=1e-12, maxit=2, raise_on_error=False)
    assert info["status"] == hdg.HDG_ERR_NOT_CONVERGED and info["iterations"] == 2
    assert info["relres"] > 1e-12
    lam, info = s.solve(b, rtol=1e-13, maxit=200)
    assert _rel(lam.cpu().numpy(), lam_ref) < 1e-10
    s.close()


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf"), 0.0, -1.0])
def test_non_finite_or_non_positive_kappa_rejected(bad):
    from paper_1705_09907_gb300 import hdg
    N, k = 8, 1
    kap = torch.ones(N * N, dtype=torch.float64, device="cuda")
    kap[13] = bad
    with pytest.raises(hdg.HDGError) as ei:
        hdg.HDGSolver(N, N, k, kap)
    assert ei.value.status == hdg.HDG_ERR_INVALID_ARG
    # the device is still usable: a valid problem sets up and solves
    kap[13] = 1.0
    s = hdg.HDGSolver(N, N, k, kap)
    lam, info = s.solve(s.condense_rhs(torch.as_tensor(inputs.constant_f(N, k), device="cuda")), rtol=1e-10)
    assert info["status"] == hdg.HDG_OK
    s.close()


def test_memory_cap_gives_oom_at_setup():
    from paper_1705_09907_gb300 import hdg
    N, k = 64, 3
    kap = torch.ones(N * N, dtype=torch.float64, device="cuda")
    with pytest.raises(hdg.HDGError) as ei:
        hdg.HDGSolver(N, N, k, kap, max_device_bytes=1 << 20)
    assert ei.value.status == hdg.HDG_ERR_OOM
    s = hdg.HDGSolver(N, N, k, kap)          # no cap: fine
    assert s.info["device_bytes"] > (1 << 20)
    s.close()


def test_memory_cap_gives_oom_for_batched_work_only():
    """A cap that holds the set-up data but not the batched work of 16
    right-hand sides: the batched solve reports OOM, the single solve on the
    same context still matches the oracle."""
    from paper_1705_09907_gb300 import hdg
    N, k = 16, 2
    kap, fq, lam_ref = _problem(N, k)
    probe = hdg.HDGSolver(N, N, k, torch.as_tensor(kap, device="cuda"))
    need = probe.info["device_bytes"]
    probe.close()
    s = hdg.HDGSolver(N, N, k, torch.as_tensor(kap, device="cuda"), max_device_bytes=need + 4096)
    b = s.condense_rhs(torch.as_tensor(fq, device="cuda"))
    B = b[:, None].repeat(1, 16).contiguous()
    _, info = s.solve(B, rtol=1e-10, raise_on_error=False)
    assert info["status"] == hdg.HDG_ERR_OOM
    lam, info = s.solve(b, rtol=1e-13)
    assert _rel(lam.cpu().numpy(), lam_ref) < 1e-10
    s.close()


def test_bounded_wait_gives_up_then_context_recovers():
    """wait_probe = 1 with the one-CTA-per-segment apply (autotune = 3): the
    first such launch after set-up gives up its first wait (~1 s bound) on a
    barrier nothing completes, drains its own block copy and exits; the solve
    reports TIMEOUT. The next solve on the same context runs normally and
    matches the oracle."""
    from paper_1705_09907_gb300 import hdg
    N, k = 16, 2
    kap, fq, lam_ref = _problem(N, k)
    s = hdg.HDGSolver(N, N, k, torch.as_tensor(kap, device="cuda"), autotune=3, wait_probe=1)
    b = s.condense_rhs(torch.as_tensor(fq, device="cuda"))
    _, info = s.solve(b, rtol=1e-10, maxit=50, raise_on_error=False)
    assert info["status"] == hdg.HDG_ERR_TIMEOUT
    lam, info = s.solve(b, rtol=1e-13, maxit=200)
    assert info["status"] == hdg.HDG_OK
    assert _rel(lam.cpu().numpy(), lam_ref) < 1e-10
    s.close()
