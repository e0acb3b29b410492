"""Full multigrid (Sec. 7; hdg_fmg and hdg_options.fmg_start) on the GPU: one
FMG cycle against the oracle's NestedGMG.fmg element by element, the
discretisation-level accuracy on the manufactured problem, and CG started from
FMG against the direct solution."""
import numpy as np
import pytest
import torch

from oracle import gmg as ogmg, hdg as ohdg, mesh as omesh
from paper_1705_09907_gb300 import inputs

pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float64, device="cuda").contiguous()


@pytest.mark.parametrize("k,smoother,cycles", [(2, 0, 1), (3, 0, 2), (3, 1, 1), (4, 1, 2)])
def test_fmg_vs_oracle(k, smoother, cycles):
    from paper_1705_09907_gb300 import hdg
    N = 16
    m = omesh.Mesh(N, N)
    kap = np.exp(inputs.gaussian_field(N, seed=7, corr_len=0.2))
    G = ogmg.NestedGMG(m, k, kap, smoother="fsai" if smoother else "asm")
    fq = np.random.default_rng(3).normal(size=(m.nel, k + 2, k + 2))
    b = G.plevels[k].prob.condense_rhs(fq)
    x_ref = G.fmg(b, cycles=cycles)
    s = hdg.HDGSolver(N, N, k, cuda(kap), smoother=smoother)
    x = s.fmg(cuda(b), cycles=cycles).cpu().numpy()
    s.close()
    assert np.linalg.norm(x - x_ref) <= 1e-11 * np.linalg.norm(x_ref)


@pytest.mark.parametrize("k", [2, 3, 4])
def test_fmg_reaches_discretisation_error(k):
    """u = sin(pi x) sin(pi y), K = 1, 32 x 32: after one FMG cycle with three
    V-cycles per level the L2 error of the recovered u is within 10% of the
    discretisation error (that of the exact discrete solution); with one
    V-cycle per level it is far above it (measured 40-36000x), which is why the
    number of cycles per level is a parameter."""
    from paper_1705_09907_gb300 import hdg
    N = 32
    m = omesh.Mesh(N, N)
    fq = inputs.manufactured_poisson_f(N, k)
    prob = ohdg.HDGProblem(m, k, np.ones(m.nel))
    ue = lambda x, y: np.sin(np.pi * x) * np.sin(np.pi * y)
    qe = lambda x, y: (-np.pi * np.cos(np.pi * x) * np.sin(np.pi * y), -np.pi * np.sin(np.pi * x) * np.cos(np.pi * y))
    lam_h = prob.solve_direct(prob.condense_rhs(fq))
    u_h, q_h = prob.recover(lam_h, fq)
    e_disc = ohdg.l2_errors(prob, u_h, q_h, ue, qe)[0]
    s = hdg.HDGSolver(N, N, k, torch.ones(N * N, dtype=torch.float64, device="cuda"))
    fd = cuda(fq)
    b = s.condense_rhs(fd)
    lam3 = s.fmg(b, cycles=3)
    u3, q3 = s.recover(lam3, fd)
    e3 = ohdg.l2_errors(prob, u3.cpu().numpy(), q3.cpu().numpy().reshape(m.nel, 2, -1), ue, qe)[0]
    s.close()
    assert e3 <= 1.1 * e_disc, (e3, e_disc)


def test_cg_from_fmg_start():
    from paper_1705_09907_gb300 import hdg
    nx, ny, k = 24, 16, 3
    m = omesh.Mesh(nx, ny)
    kap = np.exp(inputs.gaussian_field(nx, seed=2, corr_len=0.2, ny=ny))
    fq = np.random.default_rng(1).normal(size=(m.nel, k + 2, k + 2))
    prob = ohdg.HDGProblem(m, k, kap)
    ref = prob.solve_direct(prob.condense_rhs(fq))
    s0 = hdg.HDGSolver(nx, ny, k, cuda(kap))
    s2 = hdg.HDGSolver(nx, ny, k, cuda(kap), fmg_start=2)
    b = s0.condense_rhs(cuda(fq))
    l0, i0 = s0.solve(b, rtol=1e-12, maxit=300)
    l2, i2 = s2.solve(b, rtol=1e-12, maxit=300)
    for lam in (l0, l2):
        assert np.linalg.norm(lam.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)
    assert i2["iterations"] < i0["iterations"]
    s0.close()
    s2.close()
