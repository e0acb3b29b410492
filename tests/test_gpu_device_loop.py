"""The device-resident CG loop (one conditional WHILE node of a CUDA graph,
use_graphs = 1) against the host-driven loop (use_graphs = 0): the same
iterates bit for bit, the same iteration counts, residual histories and
status codes, for every inner precision, both smoothers and a full multigrid
start; the graph is reused across calls with other tolerances and limits."""
import numpy as np
import pytest
import torch

from paper_1705_09907_gb300 import hdg, inputs

pytestmark = pytest.mark.gpu


def _solvers(nx, k, **kw):
    # a fixed kernel choice (autotune = 0): timing-based choices could differ
    # between the two contexts and change the order of floating-point sums
    kap = torch.as_tensor(np.exp(inputs.gaussian_field(nx, seed=5, corr_len=0.2)), device="cuda")
    return (hdg.HDGSolver(nx, nx, k, kap, autotune=0, **kw),
            hdg.HDGSolver(nx, nx, k, kap, autotune=0, use_graphs=0, **kw))


def _rhs(s, nx, k):
    return s.condense_rhs(torch.as_tensor(inputs.constant_f(nx, k), device="cuda"))


@pytest.mark.parametrize("inner", ["fp64", "fp32", "bf16", "f32x2"])
@pytest.mark.parametrize("opts", [{}, {"smoother": 1}, {"fmg_start": 2}])
def test_device_loop_equals_host_loop(inner, opts):
    nx, k = 64, 3
    a, b = _solvers(nx, k, **opts)
    rhs = _rhs(a, nx, k)
    la, ia = a.solve(rhs, rtol=1e-10, inner=inner)
    lb, ib = b.solve(rhs, rtol=1e-10, inner=inner)
    assert ia["iterations"] == ib["iterations"] and ia["iterations"] > 3
    assert ia["relres"] == ib["relres"] <= 1e-10
    assert ia["history"] == ib["history"] and len(ia["history"]) == ia["iterations"] + 1
    assert torch.equal(la, lb)
    a.close()
    b.close()


def test_device_loop_graph_reused_across_tolerances_and_limits():
    nx, k = 32, 2
    a, b = _solvers(nx, k)
    rhs = _rhs(a, nx, k)
    for rtol, maxit in ((1e-4, 200), (1e-10, 200), (1e-12, 3), (1e-6, 200)):
        la, ia = a.solve(rhs, rtol=rtol, maxit=maxit, raise_on_error=False)
        lb, ib = b.solve(rhs, rtol=rtol, maxit=maxit, raise_on_error=False)
        assert ia["status"] == ib["status"], (rtol, maxit)
        assert ia["iterations"] == ib["iterations"], (rtol, maxit)
        assert torch.equal(la, lb)
        if maxit == 3:
            assert ia["status"] == hdg.HDG_ERR_NOT_CONVERGED and ia["iterations"] == 3
        else:
            assert ia["status"] == hdg.HDG_OK and ia["relres"] <= rtol
    a.close()
    b.close()


def test_device_loop_zero_rhs_and_small_mesh():
    # the 16 x 16, k = 1 mesh (the smallest workload) and b = 0
    a, b = _solvers(16, 1)
    rhs = _rhs(a, 16, 1)
    la, ia = a.solve(rhs, rtol=1e-10)
    lb, ib = b.solve(rhs, rtol=1e-10)
    assert ia["iterations"] == ib["iterations"] and torch.equal(la, lb)
    z, iz = a.solve(torch.zeros_like(rhs), rtol=1e-10)
    assert iz["iterations"] == 0 and torch.count_nonzero(z) == 0
    a.close()
    b.close()
