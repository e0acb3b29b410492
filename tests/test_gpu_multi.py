"""One launch (per pass) over several uneven meshes (hdg_apply_multi) against
each mesh's own apply and, for one instance, the FP64 oracle: dense owner
records (reduced = 0) and reduced blocks (reduced = 1)."""
import numpy as np
import pytest
import torch

from oracle import hdg as ohdg, mesh as omesh
from paper_1705_09907_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [(16, 16, 2), (37, 10, 3), (24, 24, 4), (8, 40, 2), (20, 12, 0), (33, 5, 5)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_multi_instance_apply(prec):
    from paper_1705_09907_gb300 import hdg
    solvers, xs = [], []
    dt = torch.float64 if prec == "fp64" else torch.float32
    for q, (nx, ny, k) in enumerate(CASES):
        kap = np.exp(inputs.gaussian_field(nx, seed=q, corr_len=0.3, ny=ny))
        # autotune = 3, reduced = 0: the single apply runs the 4-warp segment
        # kernel, whose per-segment arithmetic the multi-instance launch shares
        s = hdg.HDGSolver(nx, ny, k, torch.as_tensor(kap, device="cuda"), autotune=3, reduced=0)
        solvers.append(s)
        xs.append(torch.as_tensor(inputs.random_trace(s.n_edges, k, seed=50 + q), dtype=dt, device="cuda"))
    ys = hdg.apply_multi(solvers, xs, prec=prec)
    for s, x, y in zip(solvers, xs, ys):
        y1 = s.apply(x, prec=prec)
        torch.cuda.synchronize()
        # the same kernel arithmetic per segment: results agree to the last bits
        assert torch.allclose(y, y1, rtol=0, atol=1e-12 * float(y1.abs().max()))
    # one instance against the oracle
    nx, ny, k = CASES[1]
    m = omesh.Mesh(nx, ny)
    prob = ohdg.HDGProblem(m, k, np.exp(inputs.gaussian_field(nx, seed=1, corr_len=0.3, ny=ny)))
    xh = xs[1].double().cpu().numpy()
    ref = prob.apply_assembled(xh)
    A, idx = prob.assemble_interior()
    bound = np.zeros_like(ref)
    bound[idx] = abs(A) @ np.abs(xh[idx])
    tol = 1e-12 if prec == "fp64" else 3e-6
    assert np.all(np.abs(ys[1].double().cpu().numpy() - ref) <= tol * bound + 1e-30)
    for s in solvers:
        s.close()


def test_multi_instance_rejects_bad_input():
    from paper_1705_09907_gb300 import hdg
    s = hdg.HDGSolver(8, 8, 6, torch.ones(64, dtype=torch.float64, device="cuda"))   # degree 6 > 5
    x = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(hdg.HDGError) as e:
        hdg.apply_multi([s], [x])
    assert e.value.status == hdg.HDG_ERR_INVALID_ARG
    s.close()


def test_setup_batch_and_multi_apply():
    """hdg_setup_batch builds the uneven instances in one call; their multi apply
    equals the instances' own applies, and a bad instance fails the whole call."""
    from paper_1705_09907_gb300 import hdg
    problems = []
    for q, (nx, ny, k) in enumerate([(16, 16, 2), (24, 24, 4), (32, 32, 3)]):
        kap = np.exp(inputs.gaussian_field(nx, seed=q, corr_len=0.3, ny=ny))
        problems.append((nx, ny, k, torch.as_tensor(kap, device="cuda")))
    sols = hdg.setup_batch(problems, autotune=3, reduced=0)
    xs = [torch.as_tensor(inputs.random_trace(s.n_edges, s.k, seed=80 + q), device="cuda") for q, s in enumerate(sols)]
    ys = hdg.apply_multi(sols, xs)
    for s, x, y in zip(sols, xs, ys):
        y1 = s.apply(x)
        torch.cuda.synchronize()
        assert torch.allclose(y, y1, rtol=0, atol=1e-12 * float(y1.abs().max()))
    for s in sols:
        s.close()
    bad = list(problems)
    bad[1] = (24, 24, 4, -torch.ones(24 * 24, dtype=torch.float64, device="cuda"))
    with pytest.raises(hdg.HDGError) as e:
        hdg.setup_batch(bad)
    assert e.value.status == hdg.HDG_ERR_INVALID_ARG


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_multi_instance_reduced_blocks(prec):
    """Contexts with reduced blocks: the batch runs the element and face passes
    of the reduced apply once each for all instances; every instance's result
    is bitwise equal to its own apply (the same per-element arithmetic) and
    one instance matches the oracle."""
    from paper_1705_09907_gb300 import hdg
    dt = torch.float64 if prec == "fp64" else torch.float32
    probs = [(nx, ny, k, torch.as_tensor(np.exp(inputs.gaussian_field(nx, seed=q, corr_len=0.3, ny=ny)),
                                         device="cuda")) for q, (nx, ny, k) in enumerate(CASES)]
    sols = hdg.setup_batch(probs, reduced=1)
    xs = [torch.as_tensor(inputs.random_trace(s.n_edges, s.k, seed=80 + q), dtype=dt, device="cuda")
          for q, s in enumerate(sols)]
    ys = hdg.apply_multi(sols, xs, prec=prec)
    for s, x, y in zip(sols, xs, ys):
        assert torch.equal(y, s.apply(x, prec=prec))
    nx, ny, k = CASES[2]
    m = omesh.Mesh(nx, ny)
    prob = ohdg.HDGProblem(m, k, probs[2][3].cpu().numpy())
    xh = xs[2].double().cpu().numpy()
    ref = prob.apply_assembled(xh)
    A, idx = prob.assemble_interior()
    bound = np.zeros_like(ref)
    bound[idx] = abs(A) @ np.abs(xh[idx])
    tol = 1e-12 if prec == "fp64" else 3e-6
    assert np.all(np.abs(ys[2].double().cpu().numpy() - ref) <= tol * bound + 1e-30)
    for s in sols:
        s.close()
