"""Pins for the oracle's element-local postprocessing (Sec. 3 step (v), Sec. 5):
the paper's Table 1 columns for u_h^* and q_h^* to the printed digits,
reproduction of Q_p potentials, the mean condition, and the p+2 rate."""
import os

import numpy as np
import pytest

from oracle import hdg, mesh as omesh, quadrature as qd

HERE = os.path.dirname(os.path.abspath(__file__))


def _load():
    rows = {}
    with open(os.path.join(HERE, "golden", "tab1_postprocessed_errors.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                p, N, a, b = line.split()
                rows[(int(p), int(N))] = (float(a), float(b))
    return rows


def _exact():
    sy = pytest.importorskip("sympy")
    x, y = sy.symbols("x y")
    u = x * (x - 1) * y * (y - 1) * sy.exp(-x ** 2 - y ** 2)
    f = -(sy.diff(u, x, 2) + sy.diff(u, y, 2))
    lam = lambda e: sy.lambdify((x, y), e, "numpy")
    qx, qy = lam(-sy.diff(u, x)), lam(-sy.diff(u, y))
    return lam(f), lam(u), (lambda a, b: (qx(a, b), qy(a, b)))


def _solve_table1(p, N, fl):
    m = omesh.Mesh(N, N)
    X, Y = hdg.f_quadrature_points(m, p, npts=p + 1)
    prob = hdg.HDGProblem(m, p, np.ones(m.nel))
    fq = fl(X, Y)
    uu, qq = prob.recover(prob.solve_direct(prob.condense_rhs(fq)), fq)
    return prob, uu, qq


@pytest.mark.parametrize("p", [3, 4, 5, 6])
def test_table1_postprocessed_columns_reproduced(p):
    """Table 1, |u_h^* - u| and |q_h^* - q|, K = 1 model Poisson problem (the
    reading of the u_h, q_h columns), u^* in Q_{p+1} from the local Neumann
    problem, q^* = -grad u^*, errors by the (p+2)-point GL rule, flux error per
    component: within 1% of every printed entry above 1e-12."""
    fl, ul, qe = _exact()
    tab = _load()
    for N in (2, 4, 8, 16):
        if p == 6 and N == 16:
            continue
        prob, uu, qq = _solve_table1(p, N, fl)
        us = hdg.postprocess(prob, uu, qq)
        eu, ex, ey = hdg.postprocessed_errors(prob, us, ul, qe, components=True)
        tu, tq = tab[(p, N)]
        if tu > 1e-12:
            assert abs(eu / tu - 1) < 0.01, (p, N, eu, tu)
        if tq > 1e-12:
            assert abs(ex / tq - 1) < 0.01, (p, N, ex, tq)


def test_postprocess_reproduces_qp_potentials_and_means():
    """For u_h = v and q_h = -kappa grad v with v in Q_p (so q_h is in Q_p too),
    u^* = v exactly (at the (p+2)^2 GLL nodes); for any (u_h, q_h) the element
    mean of u^* is that of u_h."""
    rng = np.random.default_rng(3)
    for p in (1, 2, 4):
        m = omesh.Mesh(3, 2, 0.0, 0.0, 0.9, 0.5)
        kap = rng.uniform(0.5, 2.0, m.nel)
        prob = hdg.HDGProblem(m, p, kap)
        xv = qd.volume_nodes(p)
        xs = qd.volume_nodes(p + 1)
        Dv = qd.lagrange_derivative_matrix(xv, xv)
        Iv = np.eye(p + 1)
        Es = qd.lagrange_matrix(xv, xs)          # Q_p nodal -> values at the Q_{p+1} nodes
        u = rng.normal(size=(m.nel, (p + 1) ** 2))
        q = np.zeros((m.nel, 2, (p + 1) ** 2))
        for e in range(m.nel):
            q[e, 0] = -kap[e] * (np.kron(Iv, Dv) * (2 / m.hx)) @ u[e]
            q[e, 1] = -kap[e] * (np.kron(Dv, Iv) * (2 / m.hy)) @ u[e]
        us = hdg.postprocess(prob, u, q)
        for e in range(m.nel):
            assert np.abs(us[e] - np.kron(Es, Es) @ u[e]).max() < 1e-12 * np.abs(u[e]).max()
        # means, for unrelated u_h and q_h
        q2 = rng.normal(size=q.shape)
        us2 = hdg.postprocess(prob, u, q2)
        xq, wq = qd.gauss_legendre(p + 3)
        Vs = np.kron(qd.lagrange_matrix(xs, xq), qd.lagrange_matrix(xs, xq))
        Vh = np.kron(qd.lagrange_matrix(xv, xq), qd.lagrange_matrix(xv, xq))
        w = np.kron(wq, wq)
        for e in range(m.nel):
            assert abs(w @ (Vs @ us2[e]) - w @ (Vh @ u[e])) < 1e-12 * np.abs(u[e]).max()


def test_postprocess_rate_p_plus_2():
    """u^* converges at rate p + 2 (Sec. 5), flux q^* at p + 1; K = 1, p = 2, 3."""
    fl, ul, qe = _exact()
    for p in (2, 3):
        errs = []
        for N in (4, 8, 16):
            prob, uu, qq = _solve_table1(p, N, fl)
            errs.append(hdg.postprocessed_errors(prob, hdg.postprocess(prob, uu, qq), ul, qe, nquad=p + 5))
        ru = np.log2(errs[1][0] / errs[2][0])
        rq = np.log2(errs[1][1] / errs[2][1])
        assert abs(ru - (p + 2)) < 0.25 and abs(rq - (p + 1)) < 0.25


def test_bump_solution_closed_form_matches_symbolic():
    """The numpy closed form of the Sec. 5 manufactured solution (used by the GPU
    tests, where sympy is absent) against sympy's derivatives."""
    from paper_1705_09907_gb300 import inputs
    fl, ul, qe = _exact()
    rng = np.random.default_rng(0)
    X, Y = rng.uniform(0, 1, 50), rng.uniform(0, 1, 50)
    u, (qx, qy), f = inputs.bump_solution(X, Y)
    qxs, qys = qe(X, Y)
    assert np.allclose(u, ul(X, Y), rtol=1e-13, atol=1e-16)
    assert np.allclose(qx, qxs, rtol=1e-13, atol=1e-15) and np.allclose(qy, qys, rtol=1e-13, atol=1e-15)
    assert np.allclose(f, fl(X, Y), rtol=1e-12, atol=1e-14)
