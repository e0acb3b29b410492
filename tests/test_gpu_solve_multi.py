"""hdg_solve_multi: uneven problems (sizes, degrees, coefficients) solved
together, each on its own stream. Each instance's solution is bitwise the one
its own hdg_solve gives, converges to the tolerance, and matches the oracle's
direct solve; the instance mix of the benchmark (N in 64..512, k in 2..4) runs
at full size."""
import numpy as np
import pytest
import torch

from oracle import hdg as ohdg, mesh as omesh
from paper_1705_09907_gb300 import inputs

pytestmark = pytest.mark.gpu


def _problems(spec, seed0):
    out = []
    for q, (N, k) in enumerate(spec):
        kap = np.exp(inputs.gaussian_field(N, seed=seed0 + q, corr_len=0.2))
        fq = np.random.default_rng(seed0 + 50 + q).normal(size=(N * N, k + 2, k + 2))
        out.append((N, k, kap, fq))
    return out


@pytest.mark.parametrize("inner", ["fp64", "fp32"])
def test_solve_multi_equals_own_solves_and_oracle(inner):
    from paper_1705_09907_gb300 import hdg
    probs = _problems([(16, 1), (32, 2), (24, 3), (40, 4), (8, 2)], 20)
    sols = hdg.setup_batch([(N, N, k, torch.as_tensor(kap, device="cuda")) for N, k, kap, _ in probs])
    bs = [s.condense_rhs(torch.as_tensor(fq, device="cuda")) for s, (_, _, _, fq) in zip(sols, probs)]
    lams, infos = hdg.solve_multi(sols, bs, rtol=1e-12, maxit=300, inner=inner)
    torch.cuda.synchronize()
    for q, (s, b, (N, k, kap, fq)) in enumerate(zip(sols, bs, probs)):
        own, inf = s.solve(b, rtol=1e-12, maxit=300, inner=inner)
        assert torch.equal(own, lams[q])
        assert infos[q]["status"] == hdg.HDG_OK and infos[q]["iterations"] == inf["iterations"]
        assert infos[q]["relres"] <= 1e-12
        prob = ohdg.HDGProblem(omesh.Mesh(N, N), k, kap)
        ref = prob.solve_direct(prob.condense_rhs(fq))
        assert np.linalg.norm(lams[q].cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)
    for s in sols:
        s.close()


def test_solve_multi_benchmark_mix_full_size():
    from paper_1705_09907_gb300 import hdg
    mix = inputs.instance_mix(12, seed=4)
    sols = hdg.setup_batch([(N, N, k, torch.ones(N * N, dtype=torch.float64, device="cuda")) for N, k in mix],
                           mixed=0)
    bs = [s.condense_rhs(torch.as_tensor(inputs.fourier_rhs(N, k, 1, seed=40 + q)[0], device="cuda"))
          for q, (s, (N, k)) in enumerate(zip(sols, mix))]
    lams, infos = hdg.solve_multi(sols, bs, rtol=1e-10, maxit=300)
    for q, s in enumerate(sols):
        own, inf = s.solve(bs[q], rtol=1e-10, maxit=300)
        assert torch.equal(own, lams[q]) and infos[q]["relres"] <= 1e-10
        s.close()


def test_solve_multi_rejects_bad_arguments():
    from paper_1705_09907_gb300 import hdg
    s = hdg.HDGSolver(8, 8, 1, torch.ones(64, dtype=torch.float64, device="cuda"), mixed=0)
    b = s.condense_rhs(torch.ones((64, 3, 3), dtype=torch.float64, device="cuda"))
    with pytest.raises(hdg.HDGError) as e:       # the same context twice
        hdg.solve_multi([s, s], [b, b.clone()])
    assert e.value.status == hdg.HDG_ERR_INVALID_ARG
    with pytest.raises(hdg.HDGError) as e:       # FP32 cycles without mixed blocks
        hdg.solve_multi([s], [b], inner="fp32")
    assert e.value.status == hdg.HDG_ERR_UNSUPPORTED
    s.close()


def test_solve_multi_one_graph_statuses_and_zero_rhs():
    """The one-graph path: a zero right-hand side stops its loop before the first
    pass (status OK, no iterations, lambda = 0); a small maxit leaves an
    instance NOT_CONVERGED with exactly maxit iterations; the others converge as
    in their own solves; a context without graphs sends the call down the
    per-thread path with the same results."""
    from paper_1705_09907_gb300 import hdg
    probs = _problems([(16, 2), (32, 3), (24, 1)], 60)
    sols = hdg.setup_batch([(N, N, k, torch.as_tensor(kap, device="cuda")) for N, k, kap, _ in probs])
    bs = [s.condense_rhs(torch.as_tensor(fq, device="cuda")) for s, (_, _, _, fq) in zip(sols, probs)]
    bs[2] = torch.zeros_like(bs[2])
    lams, infos = hdg.solve_multi(sols, bs, rtol=1e-10, maxit=300, raise_on_error=False)
    assert infos[2]["status"] == hdg.HDG_OK and infos[2]["iterations"] == 0
    assert torch.count_nonzero(lams[2]) == 0
    for q in (0, 1):
        own, inf = sols[q].solve(bs[q], rtol=1e-10, maxit=300)
        assert torch.equal(own, lams[q]) and infos[q]["iterations"] == inf["iterations"]
    lams3, infos3 = hdg.solve_multi(sols[:2], bs[:2], rtol=1e-12, maxit=3, raise_on_error=False)
    assert all(i["status"] == hdg.HDG_ERR_NOT_CONVERGED and i["iterations"] == 3 for i in infos3)
    for s in sols:
        s.close()
    # a context with use_graphs = 0 among them: the per-thread path
    N, k, kap, fq = probs[1]
    a = hdg.HDGSolver(N, N, k, torch.as_tensor(kap, device="cuda"), autotune=0)
    c = hdg.HDGSolver(N, N, k, torch.as_tensor(kap, device="cuda"), autotune=0, use_graphs=0)
    b = a.condense_rhs(torch.as_tensor(fq, device="cuda"))
    lm, im = hdg.solve_multi([a, c], [b, b.clone()], rtol=1e-10, maxit=300)
    assert im[0]["iterations"] == im[1]["iterations"] and im[0]["status"] == hdg.HDG_OK
    assert torch.equal(lm[0], lm[1])
    a.close()
    c.close()
