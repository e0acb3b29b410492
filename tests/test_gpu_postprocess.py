"""Element-local postprocessing on the GPU (hdg_postprocess): u* and q* against
the oracle on the same (u_h, q_h) inputs, for k = 0..7 on rectangles with a
lognormal coefficient, and the whole GPU pipeline (condense, solve, recover,
postprocess) against the paper's Table 1 u* and q* columns."""
import os

import numpy as np
import pytest
import torch

from oracle import hdg as ohdg, mesh as omesh, quadrature as oqd
from paper_1705_09907_gb300 import inputs

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("k", list(range(8)))
def test_postprocess_vs_oracle(k):
    from paper_1705_09907_gb300 import hdg
    nx, ny = 7, 5
    m = omesh.Mesh(nx, ny, 0.0, 0.0, 1.0, 0.6)
    kap = np.exp(inputs.gaussian_field(nx, seed=k, corr_len=0.3, ny=ny))
    s = hdg.HDGSolver(nx, ny, k, torch.as_tensor(kap, device="cuda"), x1=1.0, y1=0.6, mixed=0)
    rng = np.random.default_rng(100 + k)
    n = (k + 1) ** 2
    u = rng.normal(size=(m.nel, n))
    q = rng.normal(size=(m.nel, 2, n))
    us_g, qs_g = s.postprocess(torch.as_tensor(u, device="cuda"), torch.as_tensor(q, device="cuda"))
    torch.cuda.synchronize()
    prob = ohdg.HDGProblem(m, k, kap)
    us_o = ohdg.postprocess(prob, u, q)
    xs = oqd.volume_nodes(k + 1)
    D1 = oqd.lagrange_derivative_matrix(xs, xs)
    I1 = np.eye(k + 2)
    Dx = np.kron(I1, D1) * (2 / m.hx)
    Dy = np.kron(D1, I1) * (2 / m.hy)
    qs_o = np.stack([-(kap[:, None]) * (us_o @ Dx.T), -(kap[:, None]) * (us_o @ Dy.T)], axis=1)
    us_g, qs_g = us_g.cpu().numpy(), qs_g.cpu().numpy()
    # FP64 local solves of size (k+2)^2 on both sides: 1e-11 of the data scale
    scale_u = np.abs(us_o).max()
    scale_q = np.abs(qs_o).max()
    assert np.abs(us_g - us_o).max() <= 1e-11 * scale_u
    assert np.abs(qs_g - qs_o).max() <= 1e-11 * scale_q
    s.close()


def _tab1_post():
    rows = {}
    with open(os.path.join(HERE, "golden", "tab1_postprocessed_errors.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                p, N, a, b = line.split()
                rows[(int(p), int(N))] = (float(a), float(b))
    return rows


@pytest.mark.parametrize("k", [3, 4])
def test_pipeline_reproduces_table1_postprocessed(k):
    """K = 1, u = x(x-1)y(y-1)exp(-x^2-y^2): GPU condense + solve (rtol 1e-13) +
    recover + postprocess; the u* and q* errors by the (k+2)-point GL rule (flux
    per component) within 2% of Table 1 at N = 8 and 16 (the library samples f
    at (k+2)^2 points where the table used k+1: a < 0.5% difference there)."""
    from paper_1705_09907_gb300 import hdg
    tab = _tab1_post()
    for N in (8, 16):
        s = hdg.HDGSolver(N, N, k, torch.ones(N * N, dtype=torch.float64, device="cuda"))
        fq = torch.as_tensor(inputs.bump_f(N, k), device="cuda")
        lam, _ = s.solve(s.condense_rhs(fq), rtol=1e-13, maxit=200)
        u, q = s.recover(lam, fq)
        us, qs = s.postprocess(u, q)
        us, qs = us.cpu().numpy(), qs.cpu().numpy()
        s.close()
        xs = oqd.volume_nodes(k + 1)
        xq, wq = np.polynomial.legendre.leggauss(k + 2)
        B = oqd.lagrange_matrix(xs, xq)
        V = np.kron(B, B)
        h = 1.0 / N
        w = np.kron(wq, wq) * h * h / 4
        eu = ex = 0.0
        for e in range(N * N):
            i, j = e % N, e // N
            X, Y = np.meshgrid(i * h + h * (xq + 1) / 2, j * h + h * (xq + 1) / 2)
            ue, (qxe, _), _ = inputs.bump_solution(X.ravel(), Y.ravel())
            eu += np.sum(w * (V @ us[e] - ue) ** 2)
            ex += np.sum(w * (V @ qs[e, 0] - qxe) ** 2)
        tu, tq = tab[(k, N)]
        assert abs(np.sqrt(eu) / tu - 1) < 0.02, (k, N, np.sqrt(eu), tu)
        assert abs(np.sqrt(ex) / tq - 1) < 0.02, (k, N, np.sqrt(ex), tq)
