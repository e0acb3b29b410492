"""Pins for the oracle's HDG discretisation (paper Secs. 3 and 5): closed forms,
invariants, an independent energy formula for S_K, the uncondensed system, the
per-edge apply of Alg. 3, convergence rates and the paper's Table 1."""
import os

import numpy as np
import pytest

from oracle import hdg, mesh as omesh
from paper_1705_09907_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def test_numbering_maps_small():
    m = omesh.Mesh(3, 2)
    e2e = m.elem_to_edge()
    # element 4 = (1, 1): W = v(1,1) = 5, E = v(2,1) = 6, S = h(1,1) = 8 + 1 + 3 = 12, N = h(1,2) = 15
    assert list(e2e[4]) == [5, 6, 12, 15]
    el, fc = m.edge_to_elem()
    assert list(el[5]) == [3, 4] and list(fc[5]) == [1, 0]
    assert list(el[12]) == [1, 4] and list(fc[12]) == [3, 2]
    assert list(el[0]) == [-1, 0]
    assert m.n_edges == 2 * 4 + 3 * 3 == 17


@pytest.mark.parametrize("kappa,h,tau", [(1.0, 0.25, 1.0), (2.0, 0.125, 1.0), (0.3, 0.5, 2.0)])
def test_p0_closed_form(kappa, h, tau):
    """k = 0 on a square of side h: S_K = kappa [[1,-1],[-1,1]] (x) (W,E), (S,N)
    + tau h (I - 11^T/4); derived from Eqs. eq_h1-eq_h3 with constant q, u."""
    ref = hdg.RefElement(0, h, h)
    S = hdg.schur_block(hdg.element_matrices(ref, kappa, tau))
    D = np.array([[1, -1, 0, 0], [-1, 1, 0, 0], [0, 0, 1, -1], [0, 0, -1, 1]], float)
    exact = kappa * D + tau * h * (np.eye(4) - 0.25)
    assert np.abs(S - exact).max() < 1e-14
    # condensed RHS of a constant f: f h^2 / 4 to every face
    b = hdg.rhs_block(hdg.element_matrices(ref, kappa, tau), np.array([3.0 * h * h]))
    assert np.allclose(b, 3.0 * h * h / 4.0, atol=1e-15)


@pytest.mark.parametrize("p", range(0, 6))
def test_schur_invariants(p):
    rng = np.random.default_rng(p)
    for hx, hy in ((0.1, 0.1), (0.3, 0.07)):
        kappa = float(np.exp(rng.normal()))
        S = hdg.schur_block(hdg.element_matrices(hdg.RefElement(p, hx, hy), kappa))
        scale = np.abs(S).max()
        assert np.abs(S - S.T).max() < 1e-13 * scale
        # a constant trace gives u = const, q = 0: S 1 = 0
        assert np.abs(S.sum(axis=1)).max() < 1e-13 * scale
        w = np.linalg.eigvalsh(S)
        assert w.min() > -1e-13 * scale
        assert (w > 1e-10 * scale).sum() == 4 * (p + 1) - 1   # kernel = constants only


@pytest.mark.parametrize("p", range(0, 8))
def test_schur_reflection_symmetry(p):
    """A rectangle with constant kappa and tau is mapped to itself by the
    reflections about its centre lines, and the Gauss-Legendre trace nodes are
    symmetric, so S_K commutes with both reflections on the face dofs [W|E|S|N]
    (x-reflection: W <-> E, S and N reversed; y-reflection: S <-> N, W and E
    reversed). Fails if a face or node ordering, a normal sign or a tau term is
    wrong in the oracle (the square case also commutes with swapping x and y)."""
    rng = np.random.default_rng(40 + p)
    n = p + 1
    R = np.arange(n)[::-1]
    W, E, S_, N = (np.arange(f * n, (f + 1) * n) for f in range(4))
    sx = np.concatenate([E, W, S_[R], N[R]])
    sy = np.concatenate([W[R], E[R], N, S_])
    swap = np.concatenate([S_, N, W, E])
    for hx, hy in ((0.1, 0.1), (0.3, 0.07)):
        for tau in (1.0, 3.5):
            kappa = float(np.exp(2 * rng.normal()))
            S = hdg.schur_block(hdg.element_matrices(hdg.RefElement(p, hx, hy), kappa, tau))
            scale = np.abs(S).max()
            assert np.abs(S[np.ix_(sx, sx)] - S).max() < 1e-13 * scale
            assert np.abs(S[np.ix_(sy, sy)] - S).max() < 1e-13 * scale
            if hx == hy:
                assert np.abs(S[np.ix_(swap, swap)] - S).max() < 1e-13 * scale
            elif p > 0:
                assert np.abs(S[np.ix_(swap, swap)] - S).max() > 1e-3 * scale


def _character_coordinates(n):
    """Rows of the transform F on face dofs [W|E|S|N] (n nodes per face): face
    sums / differences of the W/E and S/N pairs, then node-pair sums (even
    part, with the middle node) / differences (odd part), grouped by the
    character (sigma_x, sigma_y) = (+,+), (+,-), (-,+), (-,-)."""
    h = n // 2
    I = np.eye(n)
    ev = [I[i] + I[n - 1 - i] for i in range(h)] + ([I[h]] if n % 2 else [])
    od = [I[i] - I[n - 1 - i] for i in range(h)]
    Z = np.zeros(n)
    P = lambda v: np.concatenate([v, v, Z, Z])
    M = lambda v: np.concatenate([v, -v, Z, Z])
    Pp = lambda v: np.concatenate([Z, Z, v, v])
    Mp = lambda v: np.concatenate([Z, Z, v, -v])
    return [np.array([P(v) for v in ev] + [Pp(v) for v in ev]),
            np.array([P(v) for v in od] + [Mp(v) for v in ev]),
            np.array([M(v) for v in ev] + [Pp(v) for v in od]),
            np.array([M(v) for v in od] + [Mp(v) for v in od])]


@pytest.mark.parametrize("p", range(0, 8))
def test_schur_character_blocks(p):
    """Consequence of the reflection symmetry used by the reduced storage: in
    the character coordinates t = F x the element block is block diagonal,
    F S_K F^T = diag(B0, B1, B2, B3) of sizes 2s, a+s, s+a, 2a (s = ceil(n/2),
    a = floor(n/2), n = p+1), and S_K = F^T D^-1 B D^-1 F with D = F F^T
    diagonal; the packed triangles hold sum d(d+1)/2 numbers (61 at p = 4)."""
    n = p + 1
    rng = np.random.default_rng(60 + p)
    blocks = [b for b in _character_coordinates(n) if len(b)]
    F = np.vstack(blocks)
    D = F @ F.T
    assert np.abs(D - np.diag(np.diag(D))).max() == 0.0
    sizes = [len(b) for b in _character_coordinates(n)]
    s_, a_ = (n + 1) // 2, n // 2
    assert sizes == [2 * s_, a_ + s_, s_ + a_, 2 * a_]
    packed = sum(d * (d + 1) // 2 for d in sizes)
    assert packed == {0: 5, 1: 12, 2: 25, 3: 40, 4: 61, 5: 84, 6: 113, 7: 144}[p]
    for hx, hy in ((0.1, 0.1), (0.3, 0.07)):
        S = hdg.schur_block(hdg.element_matrices(hdg.RefElement(p, hx, hy), float(np.exp(rng.normal())), 1.0))
        B = F @ S @ F.T
        off = np.cumsum([0] + [len(b) for b in blocks])
        mask = np.zeros_like(B, dtype=bool)
        for q in range(len(blocks)):
            mask[off[q]:off[q + 1], off[q]:off[q + 1]] = True
        scale = np.abs(B).max()
        assert np.abs(B[~mask]).max(initial=0.0) < 1e-13 * scale
        Dinv = np.diag(1.0 / np.diag(D))
        assert np.abs(F.T @ (Dinv @ np.where(mask, B, 0.0) @ Dinv) @ F - S).max() < 1e-13 * np.abs(S).max()


@pytest.mark.parametrize("p", range(0, 6))
def test_tau_kappa_scaling(p):
    """With tau_K = kappa_K every local equation is kappa_K times the kappa = 1,
    tau = 1 one once q is written as kappa q~ (the (kappa^-1 q, v) block becomes
    (q~, v), the flux and stabilisation terms gain a factor kappa), so
    S_K = kappa_K S_ref exactly and b_K = G^T F does not depend on kappa_K. The
    per-element problem's tau_of must follow kappa."""
    rng = np.random.default_rng(50 + p)
    for hx, hy in ((0.1, 0.1), (0.3, 0.07)):
        ref = hdg.RefElement(p, hx, hy)
        S1 = hdg.schur_block(hdg.element_matrices(ref, 1.0, 1.0))
        F = rng.normal(size=ref.n)
        b1 = hdg.rhs_block(hdg.element_matrices(ref, 1.0, 1.0), F)
        for kappa in (1e-3, 0.37, 42.0):
            mt = hdg.element_matrices(ref, kappa, kappa)
            assert np.abs(hdg.schur_block(mt) - kappa * S1).max() < 1e-12 * kappa * np.abs(S1).max()
            assert np.abs(hdg.rhs_block(mt, F) - b1).max() < 1e-12 * np.abs(b1).max()
            # tau fixed at 1 is not a scaling
            S_t1 = hdg.schur_block(hdg.element_matrices(ref, kappa, 1.0))
            assert np.abs(S_t1 - kappa * S1).max() > 1e-3 * kappa * np.abs(S1).max()
    m = omesh.Mesh(3, 2)
    kap = np.array([0.5, 2.0, 7.0, 1.0, 3.0, 0.25])
    prob = hdg.HDGProblem(m, p, kap, "kappa")
    assert [prob.tau_of(e) for e in range(m.nel)] == list(kap)
    with pytest.raises(ValueError):
        hdg.HDGProblem(m, p, kap, "other")


@pytest.mark.parametrize("p", range(0, 5))
def test_schur_energy_identity(p):
    """Independent second formula: lambda^T S mu = (kappa^-1 q_l, q_m)_K
    + tau <u_l - lambda, u_m - mu>_dK, with (q, u) from the local solver."""
    rng = np.random.default_rng(10 + p)
    ref = hdg.RefElement(p, 0.2, 0.15)
    kappa = 1.7
    mt = hdg.element_matrices(ref, kappa, tau=1.3)
    S = hdg.schur_block(mt)
    n, m = ref.n, ref.m
    F0 = np.zeros(n)
    lam, mu = rng.normal(size=m), rng.normal(size=m)
    Ql, Ul = hdg.local_solve(mt, lam, F0)
    Qm, Um = hdg.local_solve(mt, mu, F0)
    vol = Ql @ mt["A"] @ Qm                      # (kappa^-1 q_l, q_m)
    bnd = 0.0
    for f in range(4):
        phi, T, w, _ = ref.face_tables(f)
        sl = slice(f * (p + 1), (f + 1) * (p + 1))
        dl = phi @ Ul - T @ lam[sl]
        dm = phi @ Um - T @ mu[sl]
        bnd += 1.3 * np.sum(w * dl * dm)
    assert abs(lam @ S @ mu - (vol + bnd)) < 1e-12 * max(1.0, abs(vol + bnd))


@pytest.mark.parametrize("p", range(0, 4))
def test_rhs_identity(p):
    """b_K(mu) = (f, u_mu)_K (u_mu: local solution for trace mu, f = 0)."""
    rng = np.random.default_rng(20 + p)
    ref = hdg.RefElement(p, 0.25, 0.25)
    mt = hdg.element_matrices(ref, 0.6)
    F = rng.normal(size=ref.n)
    b = hdg.rhs_block(mt, F)
    for a in range(ref.m):
        e = np.zeros(ref.m)
        e[a] = 1.0
        _, U = hdg.local_solve(mt, e, np.zeros(ref.n))
        assert abs(b[a] - F @ U) < 1e-13 * np.abs(F).max()


def test_integration_by_parts_block():
    for p in range(0, 5):
        mt = hdg.element_matrices(hdg.RefElement(p, 0.2, 0.3), 1.0)
        assert np.abs(mt["B2"] - mt["B"]).max() < 1e-13


@pytest.mark.parametrize("tau", [1.0, "kappa"])
@pytest.mark.parametrize("p", [0, 1, 2, 3])
def test_condensed_equals_uncondensed(p, tau):
    rng = np.random.default_rng(30 + p)
    m = omesh.Mesh(3, 4, 0.0, 0.0, 1.5, 1.0)
    kappa = np.exp(rng.normal(size=m.nel))
    fq = rng.normal(size=(m.nel, p + 2, p + 2))
    prob = hdg.HDGProblem(m, p, kappa, tau)
    lam = prob.solve_direct(prob.condense_rhs(fq))
    u, q = prob.recover(lam, fq)
    lam2, u2, q2 = hdg.uncondensed_solve(m, p, kappa, fq, tau)
    assert np.abs(lam - lam2).max() < 1e-12 * np.abs(lam2).max()
    assert np.abs(u - u2).max() < 1e-12 * np.abs(u2).max()
    assert np.abs(q - q2).max() < 1e-12 * np.abs(q2).max()


@pytest.mark.parametrize("p", [0, 1, 3])
def test_global_spd_and_per_edge_apply(p):
    rng = np.random.default_rng(40 + p)
    m = omesh.Mesh(5, 4)
    prob = hdg.HDGProblem(m, p, np.exp(rng.normal(size=m.nel)))
    A, idx = prob.assemble_interior()
    Ad = A.toarray()
    assert np.abs(Ad - Ad.T).max() < 1e-13 * np.abs(Ad).max()
    np.linalg.cholesky(Ad)
    x = rng.normal(size=prob.ndof)
    y1 = prob.apply_assembled(x, A, idx)
    y2 = prob.apply_per_edge(x)
    assert np.abs(y1 - y2).max() < 1e-13 * np.abs(y1).max()
    bnd = np.setdiff1d(np.arange(prob.ndof), idx)
    assert np.all(y2[bnd] == 0.0)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_convergence_rate_manufactured(p):
    """O(h^{p+1}) for u = sin(pi x) sin(pi y), kappa = 1."""
    ue = lambda x, y: np.sin(np.pi * x) * np.sin(np.pi * y)
    qe = lambda x, y: (-np.pi * np.cos(np.pi * x) * np.sin(np.pi * y),
                       -np.pi * np.sin(np.pi * x) * np.cos(np.pi * y))
    eu, eq = [], []
    for N in (4, 8, 16):
        m = omesh.Mesh(N, N)
        fq = inputs.manufactured_poisson_f(N, p)
        prob = hdg.HDGProblem(m, p, np.ones(m.nel))
        lam = prob.solve_direct(prob.condense_rhs(fq))
        u, q = prob.recover(lam, fq)
        a, b = hdg.l2_errors(prob, u, q, ue, qe)
        eu.append(a)
        eq.append(b)
    ru = np.log2(eu[1] / eu[2])
    rq = np.log2(eq[1] / eq[2])
    assert abs(ru - (p + 1)) < 0.2 and abs(rq - (p + 1)) < 0.2


def _load_tab1():
    rows = []
    with open(os.path.join(HERE, "golden", "tab1_hdg_errors.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                p, N, eu, eq = line.split()
                rows.append((int(p), int(N), float(eu), float(eq)))
    return rows


def _table1_exact(K_is_one):
    sy = pytest.importorskip("sympy")
    x, y = sy.symbols("x y")
    K = sy.Integer(1) if K_is_one else sy.tanh(x + y) + 1
    u = x * (x - 1) * y * (y - 1) * sy.exp(-x ** 2 - y ** 2)
    f = -(sy.diff(K * sy.diff(u, x), x) + sy.diff(K * sy.diff(u, y), y))
    lam = lambda e: sy.lambdify((x, y), e, "numpy")
    fl, ul, Kl = lam(f), lam(u), lam(K + 0 * x)
    qxl, qyl = lam(-K * sy.diff(u, x)), lam(-K * sy.diff(u, y))
    return fl, ul, (lambda a, b: Kl(a, b) * np.ones_like(a)), (lambda a, b: (qxl(a, b), qyl(a, b)))


@pytest.mark.parametrize("p", [3, 4, 5, 6])
def test_table1_reproduced(p):
    """Sec. 5 Table 1, the |u_h - u| and |q_h - q| columns, reproduced to the
    printed three digits. Reading (DESIGN, reading 16): the table is the model
    Poisson problem of Sec. 5 (K = 1, tau = 1; the text's tanh coefficient does
    not give these constants), u = x(x-1)y(y-1)exp(-x^2-y^2), with the load and
    the error norms integrated by the (p+1)-point Gauss-Legendre rule per
    direction, and the flux error of one component (|q_x - q_hx| = |q_y - q_hy|
    by the x <-> y symmetry of u). Entries below 1e-12 sit on the table's
    rounding floor (the N = 32 rows grow again) and are skipped."""
    fl, ul, _, qe = _table1_exact(True)
    table = {(pp, N): (a, b) for pp, N, a, b in _load_tab1() if pp == p}
    for N in (2, 4, 8, 16):
        m = omesh.Mesh(N, N)
        X, Y = hdg.f_quadrature_points(m, p, npts=p + 1)
        prob = hdg.HDGProblem(m, p, np.ones(m.nel))
        fq = fl(X, Y)
        lam = prob.solve_direct(prob.condense_rhs(fq))
        uu, qq = prob.recover(lam, fq)
        eu, eqx, eqy = hdg.l2_errors(prob, uu, qq, ul, qe, nquad=p + 1, components=True)
        assert abs(eqx - eqy) <= 1e-4 * eqx
        tu, tq = table[(p, N)]
        if tu > 1e-12:
            assert abs(eu / tu - 1.0) < 0.01, (p, N, eu, tu)
        if tq > 1e-12:
            assert abs(eqx / tq - 1.0) < 0.01, (p, N, eqx, tq)


def test_table1_sensitive_to_its_reading():
    """The Table 1 match is not loose: the default (p+4)-point error rule, the
    norm of the whole flux, or the (p+2)-point load each move an entry by more
    than the 1% band (p = 3, N = 8: 1.057, 1.551, 1.002 -> checked > 1.04 etc.)."""
    p, N = 3, 8
    fl, ul, _, qe = _table1_exact(True)
    tu, tq = {(pp, n): (a, b) for pp, n, a, b in _load_tab1()}[(p, N)]
    m = omesh.Mesh(N, N)
    prob = hdg.HDGProblem(m, p, np.ones(m.nel))
    X, Y = hdg.f_quadrature_points(m, p, npts=p + 1)
    fq = fl(X, Y)
    uu, qq = prob.recover(prob.solve_direct(prob.condense_rhs(fq)), fq)
    eu, eq = hdg.l2_errors(prob, uu, qq, ul, qe)
    assert eu / tu > 1.04 and eq / tq > 1.5
    eu, eq = hdg.l2_errors(prob, uu, qq, ul, qe, nquad=p + 1)
    assert abs(eu / tu - 1) < 0.01 and eq / tq > 1.4
    # a load vector off by a factor 2 moves u_h by a factor 2
    uu2, qq2 = prob.recover(prob.solve_direct(prob.condense_rhs(2 * fq)), 2 * fq)
    eu2, _, _ = hdg.l2_errors(prob, uu2, qq2, ul, qe, nquad=p + 1, components=True)
    assert eu2 / tu > 10


@pytest.mark.parametrize("p", [3, 4])
def test_table1_text_coefficient_rates(p):
    """The coefficient named in the text of Sec. 5, K = tanh(x+y)+1 (evaluated at
    the quadrature points), gives the same p+1 rates for u_h and q_h as Table 1
    (within 0.25, N = 4 -> 8 -> 16), with larger constants."""
    fl, ul, Kl, qe = _table1_exact(False)
    table = {(pp, N): (a, b) for pp, N, a, b in _load_tab1() if pp == p}
    Ns = (4, 8, 16)
    ours = {}
    for N in Ns:
        m = omesh.Mesh(N, N)
        X, Y = hdg.f_quadrature_points(m, p)
        xc, yc = m.elem_centres()
        prob = hdg.HDGProblem(m, p, Kl(xc, yc), kappa_q_fn=Kl, nquad=p + 4)
        fq = fl(X, Y)
        uu, qq = prob.recover(prob.solve_direct(prob.condense_rhs(fq)), fq)
        ours[N] = hdg.l2_errors(prob, uu, qq, ul, qe)
    for N0, N1 in zip(Ns[:-1], Ns[1:]):
        for c in (0, 1):
            rate_t = np.log2(table[(p, N0)][c] / table[(p, N1)][c])
            rate_o = np.log2(ours[N0][c] / ours[N1][c])
            assert abs(rate_t - rate_o) < 0.25
