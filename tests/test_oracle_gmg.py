"""Pins for the oracle's nested multigrid (paper Sec. 6-7): exact transfers,
Galerkin structure, Chebyshev polynomial, symmetric V-cycle, the paper's
convergence factor, and the adjoint against finite differences."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import adjoint, gmg, hdg, quadrature as qd, mesh as omesh
from paper_1705_09907_gb300 import inputs


@pytest.mark.parametrize("p", range(0, 6))
def test_p_prolongation_is_embedding(p):
    """Eq. eq_mg_pro: a degree-p edge function is reproduced exactly at degree p+1."""
    P = gmg.p_prolongation_1d(p)
    xc, xf = qd.trace_nodes(p), qd.trace_nodes(p + 1)
    for deg in range(p + 1):
        assert np.abs(P @ xc ** deg - xf ** deg).max() < 1e-14
    # L2 adjointness (Eq. eq_mg_res): with diagonal GL masses, (R v, u_H) = (v, P u_H)
    wc, wf = qd.gauss_legendre(p + 1)[1], qd.gauss_legendre(p + 2)[1]
    Rl2 = np.diag(1 / wc) @ P.T @ np.diag(wf)
    # R maps a fine function to its coarse L2 projection: identity on the coarse space
    assert np.abs(Rl2 @ P - np.eye(p + 1)).max() < 1e-13


def test_q1_to_p0_edge_means():
    m = omesh.Mesh(4, 3)
    PJ = gmg.q1_to_p0(m)
    # v(x, y) = x (1 - x) y (1 - y) sampled at interior vertices; edges between
    # vertices a, b get (v_a + v_b)/2; boundary vertices are 0
    xs, ys = np.arange(m.nx + 1) / m.nx, np.arange(m.ny + 1) / m.ny
    V = np.outer(ys * (1 - ys), xs * (1 - xs))          # [j, i]
    v_int = V[1:-1, 1:-1].ravel()
    lam = PJ @ v_int
    for j in range(m.ny):
        for i in range(m.nx + 1):
            assert abs(lam[m.vedge(i, j)] - 0.5 * (V[j, i] + V[j + 1, i])) < 1e-15
    for j in range(m.ny + 1):
        for i in range(m.nx):
            assert abs(lam[m.hedge(i, j)] - 0.5 * (V[j, i] + V[j, i + 1])) < 1e-15


def test_q1_prolongation_reproduces_bilinears():
    P = gmg.q1_prolongation(4, 2)
    f = lambda x, y: (x * (1 - x)) * (y * (1 - y))   # piecewise-bilinear interpolant check below
    # a coarse bilinear-per-cell function: its fine interpolant at fine vertices
    xc, yc = np.arange(5) / 4, np.arange(3) / 2
    Vc = np.outer(yc * (1 - yc), xc * (1 - xc))
    xf, yf = np.arange(9) / 8, np.arange(5) / 4
    vf = P @ Vc[1:-1, 1:-1].ravel()
    for jf in range(1, 4):
        for i_f in range(1, 8):
            # bilinear interpolation of the coarse nodal values
            X, Y = xf[i_f] * 4, yf[jf] * 2
            i0, j0 = min(int(X), 3), min(int(Y), 1)
            sx, sy = X - i0, Y - j0
            ref = ((1 - sx) * (1 - sy) * Vc[j0, i0] + sx * (1 - sy) * Vc[j0, i0 + 1]
                   + (1 - sx) * sy * Vc[j0 + 1, i0] + sx * sy * Vc[j0 + 1, i0 + 1])
            assert abs(vf[(i_f - 1) + 7 * (jf - 1)] - ref) < 1e-15


def test_q1_stiffness_closed_form():
    """Bilinear element stiffness on hx x hy: (hy/hx) Kx + (hx/hy) Ky with the
    textbook 1/6 patterns; a 2x2 mesh has one interior vertex with A = sum of the
    four elements' corner diagonals = 4 * (2/6)(hy/hx + hx/hy) * kappa."""
    m = omesh.Mesh(2, 2, 0, 0, 1.0, 0.5)
    kap = np.array([1.0, 2.0, 3.0, 4.0])
    A = gmg.q1_stiffness(m, kap).toarray()
    hx, hy = 0.5, 0.25
    assert abs(A[0, 0] - kap.sum() * (2 / 6) * (hy / hx + hx / hy)) < 1e-14


@pytest.mark.parametrize("nx,ny,Lx,Ly", [(6, 6, 1.0, 1.0), (5, 4, 1.0, 0.5)])
def test_q1_stiffness_full_stencil(nx, ny, Lx, Ly):
    """Every entry of the Q1 stiffness (kappa grad u, grad v) against the closed
    form of the bilinear element on hx x hy (a = hy/hx, b = hx/hy): per element,
    its own vertex (a + b)/3, the vertex across an x-edge (b - 2a)/6, across a
    y-edge (a - 2b)/6, the opposite corner -(a + b)/6; on squares with kappa = 1
    this is the 9-point stencil (8, -1 x 8)/3 with zero sums on rows away from
    the boundary."""
    m = omesh.Mesh(nx, ny, 0, 0, Lx, Ly)
    rng = np.random.default_rng(11)
    kap = rng.uniform(0.5, 3.0, m.nel)
    A = gmg.q1_stiffness(m, kap).toarray()
    a, b = m.hy / m.hx, m.hx / m.hy
    own, xn, yn, cor = (a + b) / 3, (b - 2 * a) / 6, (a - 2 * b) / 6, -(a + b) / 6
    vid = lambda i, j: (i - 1) + (nx - 1) * (j - 1)
    ref = np.zeros_like(A)
    for j in range(1, ny):
        for i in range(1, nx):
            r = vid(i, j)
            for ei in (i - 1, i):
                for ej in (j - 1, j):
                    k = kap[ei + nx * ej]
                    ref[r, r] += own * k
                    # the element's other vertices: across its x-edge, y-edge, corner
                    xi = i - 1 if ei == i - 1 else i + 1
                    yj = j - 1 if ej == j - 1 else j + 1
                    for (ii, jj, v) in ((xi, j, xn), (i, yj, yn), (xi, yj, cor)):
                        if 1 <= ii < nx and 1 <= jj < ny:
                            ref[r, vid(ii, jj)] += v * k
    assert np.abs(A - ref).max() < 1e-13 * np.abs(ref).max()
    if nx == ny and Lx == Ly:
        A1 = gmg.q1_stiffness(m, np.ones(m.nel)).toarray()
        r = vid(3, 3)
        row = A1[r].reshape(ny - 1, nx - 1)
        assert np.allclose(row[1:4, 1:4], np.array([[-1, -1, -1], [-1, 8, -1], [-1, -1, -1]]) / 3, atol=1e-14)
        for j in range(2, ny - 1):
            for i in range(2, nx - 1):
                assert abs(A1[vid(i, j)].sum()) < 1e-14


def test_chebyshev_is_scaled_chebyshev_polynomial():
    """On a diagonal matrix the degree-2 step maps e0 -> T2((theta - l)/delta) /
    T2(theta/delta) e0 at every eigenvalue l (Jacobi scaling trivial)."""
    import scipy.sparse as sp
    lam = np.linspace(0.05, 2.0, 9)
    A = sp.diags(lam).tocsr()
    lmax = 2.0
    a, b = 0.1 * lmax, 1.1 * lmax
    theta, delta = (a + b) / 2, (b - a) / 2
    T2 = lambda t: 2 * t * t - 1
    e0 = np.ones(9)
    x = gmg.chebyshev(A, np.ones(9), lmax, np.zeros(9), e0)   # f = 0: x is the error
    assert np.allclose(x, T2((theta - lam) / delta) / T2(theta / delta) * e0, atol=1e-14)


def test_power_iteration_estimate():
    m = omesh.Mesh(8, 8)
    A = gmg.q1_stiffness(m, np.ones(m.nel))
    lam = gmg.lambda_max_jacobi(A)
    d = A.diagonal()
    import scipy.sparse as sp
    Ds = sp.diags(1 / np.sqrt(d))
    true = spla.eigsh(Ds @ A @ Ds, k=1, which="LA")[0][0]
    assert 0.9 * true < lam <= true * (1 + 1e-12)


def _gmg(N, k, seed=0, kappa=None):
    m = omesh.Mesh(N, N)
    kap = np.ones(m.nel) if kappa is None else kappa
    G = gmg.NestedGMG(m, k, kap)
    rng = np.random.default_rng(seed)
    top = G.plevels[k]
    b = np.zeros(top.ndof)
    b[top.idx] = rng.normal(size=len(top.idx))
    return G, b


def test_galerkin_levels_symmetric_and_element_local():
    G, _ = _gmg(6, 3)
    for p, lev in G.plevels.items():
        A = lev.A
        assert abs(A - A.T).max() < 1e-12 * abs(A).max()
    # coarse Galerkin operator = sum over elements of P_K^T S_K P_K
    fine = G.plevels[3]
    S = fine.prob.S()
    Pk = np.kron(np.eye(4), gmg.p_prolongation_1d(2))
    coarse_prob = hdg.HDGProblem(G.mesh, 2, np.ones(G.mesh.nel))
    A2, _ = coarse_prob.assemble_interior(S=np.array([Pk.T @ s @ Pk for s in S]))
    assert abs(A2 - G.plevels[2].A).max() < 1e-12 * abs(A2).max()


def test_vcycle_symmetric_positive():
    G, _ = _gmg(8, 2)
    rng = np.random.default_rng(5)
    top = G.plevels[2]
    r = np.zeros(top.ndof)
    s = np.zeros(top.ndof)
    r[top.idx] = rng.normal(size=len(top.idx))
    s[top.idx] = rng.normal(size=len(top.idx))
    Vr, Vs = G.vcycle(r), G.vcycle(s)
    assert abs(s @ Vr - r @ Vs) < 1e-11 * abs(s @ Vr)
    assert r @ Vr > 0


@pytest.mark.parametrize("k,bound", [(2, 0.32), (3, 0.22), (4, 0.22), (5, 0.22)])
def test_convergence_factor_paper(k, bound):
    """Sec. 7: with the V(2,2) cycle as a stationary solver on a 32 x 32 mesh the
    paper's convergence factor is below 0.22 for p = 2..8 (FSAI smoother). With
    the element-patch Schwarz smoother this holds from k = 3 up; k = 2 gives
    about 0.29 (recorded bound 0.32)."""
    G, b = _gmg(32, k, seed=k)
    _, hist = G.stationary(b, 9)
    assert gmg.convergence_factor(hist) < bound


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(n, n))
    return B @ B.T + n * np.eye(n)


def test_fsai_full_pattern_is_exact_inverse():
    """With every lower-triangular entry allowed, the factorized approximate
    inverse is exact: G = L^-1 for A = L L^T, so G^T G = A^-1."""
    A = _spd(12, 1)
    G = gmg.fsai_factor(A, np.tril(np.ones((12, 12)))).toarray()
    assert np.abs(G.T @ G - np.linalg.inv(A)).max() < 1e-12 * np.abs(np.linalg.inv(A)).max()
    assert np.abs(np.triu(G, 1)).max() == 0.0


def test_fsai_diagonal_pattern_is_jacobi():
    A = _spd(9, 2)
    G = gmg.fsai_factor(A, np.eye(9)).toarray()
    assert np.allclose(G, np.diag(1.0 / np.sqrt(np.diag(A))), rtol=1e-14, atol=0)


def test_fsai_rows_optimal_and_normalised():
    """For a banded pattern: G A G^T has a unit diagonal, and each row's
    Frobenius-optimality condition holds, (G A)[i, j] = 0 for the allowed
    j != i (the residual of row i is orthogonal to its pattern)."""
    n = 15
    A = _spd(n, 3)
    pat = np.tril(np.triu(np.ones((n, n)), -3))
    G = gmg.fsai_factor(A, pat).toarray()
    assert np.abs(np.diag(G @ A @ G.T) - 1.0).max() < 1e-12
    GA = G @ A
    for i in range(n):
        for j in range(max(0, i - 3), i):
            assert abs(GA[i, j]) < 1e-12 * np.abs(GA[i]).max()
    assert np.all(G[pat == 0] == 0.0)


def test_fsai_vcycle_symmetric_positive():
    m = omesh.Mesh(8, 8)
    G = gmg.NestedGMG(m, 2, np.exp(np.random.default_rng(4).normal(size=m.nel)), smoother="fsai")
    rng = np.random.default_rng(5)
    top = G.plevels[2]
    r = np.zeros(top.ndof)
    s = np.zeros(top.ndof)
    r[top.idx] = rng.normal(size=len(top.idx))
    s[top.idx] = rng.normal(size=len(top.idx))
    Vr, Vs = G.vcycle(r), G.vcycle(s)
    assert abs(s @ Vr - r @ Vs) < 1e-11 * abs(s @ Vr)
    assert r @ Vr > 0


@pytest.mark.parametrize("k", [2, 3, 4])
def test_fsai_convergence_factor_paper(k):
    """Sec. 7 with the paper's smoother: V(2,2) with FSAI of operator complexity
    one (pattern of A) as a stationary solver on 32 x 32, K = 1: every factor
    is below the paper's 0.22 (it reports 0.13-0.15 for even p); measured here
    0.157 / 0.112 / 0.109 for p = 2 / 3 / 4 with Galerkin coarse p-operators."""
    m = omesh.Mesh(32, 32)
    G = gmg.NestedGMG(m, k, np.ones(m.nel), smoother="fsai")
    top = G.plevels[k]
    b = np.zeros(top.ndof)
    b[top.idx] = np.random.default_rng(0).normal(size=len(top.idx))
    _, hist = G.stationary(b, 9)
    assert gmg.convergence_factor(hist) < 0.22


def test_rediscretized_coarse_ops_diverge_at_k1():
    """Documents the reading on coarse p-operators: the literal rediscretised
    p = 0 level (tau = 1) makes the k = 1 V-cycle diverge on a 16 x 16 mesh."""
    m = omesh.Mesh(16, 16)
    G = gmg.NestedGMG(m, 1, np.ones(m.nel), coarse_op="rediscretize")
    top = G.plevels[1]
    b = np.zeros(top.ndof)
    b[top.idx] = np.random.default_rng(0).normal(size=len(top.idx))
    _, hist = G.stationary(b, 8)
    assert gmg.convergence_factor(hist) > 1.0


def test_pcg_matches_direct_solve():
    m = omesh.Mesh(16, 16)
    k = 2
    kappa = inputs.lognormal_kappa(16, seed=0, corr_len=0.2)
    G = gmg.NestedGMG(m, k, kappa)
    fq = inputs.constant_f(16, k)
    prob = hdg.HDGProblem(m, k, kappa)
    b = prob.condense_rhs(fq)
    lam_d = prob.solve_direct(b)
    lam_c, it, hist = G.pcg(b, rtol=1e-12)
    assert hist[-1] <= 1e-12 and it < 30
    assert np.linalg.norm(lam_c - lam_d) <= 1e-10 * np.linalg.norm(lam_d)


def test_coarse_direct_solve():
    G, _ = _gmg(8, 1)
    import scipy.linalg as sla
    Ac = G.hA[-1].toarray()
    r = np.arange(1.0, Ac.shape[0] + 1)
    x = sla.cho_solve(G.coarse, r)
    assert np.abs(Ac @ x - r).max() < 1e-13 * np.abs(r).max()


@pytest.mark.parametrize("tau", [1.0, "kappa"])
def test_adjoint_vs_finite_differences(tau):
    rng = np.random.default_rng(7)
    m = omesh.Mesh(4, 4)
    p = 2
    th = rng.normal(size=m.nel)
    fq = rng.normal(size=(m.nel, p + 2, p + 2))
    lam_obs = rng.normal(size=m.n_edges * (p + 1))
    prob = hdg.HDGProblem(m, p, np.exp(th), tau)
    J, lam, dth, df = adjoint.gradients(prob, fq, lam_obs)
    h = 1e-6
    for e in (0, 6, 15):
        tp, tm = th.copy(), th.copy()
        tp[e] += h
        tm[e] -= h
        fd = (adjoint.objective(m, p, tp, fq, lam_obs, tau) - adjoint.objective(m, p, tm, fq, lam_obs, tau)) / (2 * h)
        assert abs(fd - dth[e]) <= 1e-5 * max(abs(fd), 1e-3)
    for (e, a, b) in ((3, 1, 2), (9, 0, 3)):
        fp, fm = fq.copy(), fq.copy()
        fp[e, a, b] += h
        fm[e, a, b] -= h
        fd = (adjoint.objective(m, p, th, fp, lam_obs, tau) - adjoint.objective(m, p, th, fm, lam_obs, tau)) / (2 * h)
        assert abs(fd - df[e, a, b]) <= 1e-5 * max(abs(fd), 1e-3)
    if tau == "kappa":
        # S_K = kappa_K S_ref and b_K does not depend on kappa_K, so
        # dJ/dtheta_K = -psi_K^T S_K lambda_K (psi = A^-1 (lambda - lambda_obs))
        A, idx = prob.assemble_interior()
        r = np.zeros(prob.ndof)
        r[idx] = (lam - lam_obs)[idx]
        psi = np.zeros(prob.ndof)
        psi[idx] = np.linalg.solve(A.toarray(), r[idx])
        for e in range(m.nel):
            d = prob.dofs(e)
            closed = -psi[d] @ hdg.schur_block(prob.mats(e)) @ lam[d]
            assert abs(closed - dth[e]) <= 1e-10 * np.abs(dth).max()


def test_lognormal_field_statistics():
    """Generator check: unit variance and squared-exponential correlation."""
    n = 128
    g = np.stack([inputs.gaussian_field(n, seed=s, corr_len=0.05) for s in range(40)])
    assert abs(g.var() - 1.0) < 0.1
    G = g.reshape(40, n, n)
    lag = 6                                   # r = 6 / 128
    c = np.mean(G[:, :, :-lag] * G[:, :, lag:])
    assert abs(c - np.exp(-(lag / n) ** 2 / (2 * 0.05 ** 2))) < 0.08


def test_fmg_converges_to_direct_solve_and_is_linear():
    """Full multigrid (Sec. 7): with many V-cycles per level it reaches the
    direct solution; it is linear in b; one FMG pass leaves a smaller residual
    than one V-cycle from zero (it starts every level from the interpolated
    coarser solution)."""
    m = omesh.Mesh(16, 16)
    kap = np.exp(np.random.default_rng(2).normal(size=m.nel))
    G = gmg.NestedGMG(m, 3, kap)
    top = G.plevels[3]
    rng = np.random.default_rng(5)
    b1 = np.zeros(top.ndof)
    b2 = np.zeros(top.ndof)
    b1[top.idx] = rng.normal(size=len(top.idx))
    b2[top.idx] = rng.normal(size=len(top.idx))
    x_ref = np.zeros(top.ndof)
    x_ref[top.idx] = spla.spsolve(top.A.tocsc(), b1[top.idx])
    x40 = G.fmg(b1, cycles=40)
    assert np.linalg.norm(x40 - x_ref) <= 1e-10 * np.linalg.norm(x_ref)
    lin = G.fmg(2.5 * b1 + b2) - (2.5 * G.fmg(b1) + G.fmg(b2))
    assert np.linalg.norm(lin) <= 1e-12 * np.linalg.norm(G.fmg(b1))
    r_fmg = np.linalg.norm(b1 - G.apply(G.fmg(b1)))
    r_v = np.linalg.norm(b1 - G.apply(G.vcycle(b1)))
    assert r_fmg < r_v
