"""1-D Gauss-Legendre (GL) and Gauss-Legendre-Lobatto (GLL) rules and barycentric
Lagrange evaluation, float64 (paper Sec. 4, "Basis functions").

Test infrastructure only (see the package docstring).

Readings of the paper taken here:
  * The printed explicit barycentric weights in Sec. 4 pair GLL nodes with GL
    weights and are garbled; the second (true) barycentric form is invariant to a
    common scaling of the weights, so the weights are computed from their
    definition W_j = 1 / prod_{m != j} (x_j - x_m) (the O(N^2) set-up the paper
    mentions).
  * Volume basis: Lagrange at the p+1 GLL nodes for p >= 1, tensorised with the
    lexicographic index I = i + j (p+1) of Sec. 4; for p = 0 (where GLL is
    undefined) the single basis function is the constant 1.
  * Trace basis (not stated in the paper; its node figure shows GL surface
    nodes): Lagrange at the p+1 GL nodes of each edge; p = 0 is the midpoint.
"""
import numpy as np


def legendre_and_derivative(n, x):
    """P_n(x) and P_n'(x) by the three-term recurrence (Bonnet)."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for m in range(2, n + 1):
        p0, p1 = p1, ((2 * m - 1) * x * p1 - (m - 1) * p0) / m
    # derivative from (1 - x^2) P_n' = n (P_{n-1} - x P_n), valid off +-1
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = n * (p0 - x * p1) / (1.0 - x * x)
    at_end = np.abs(np.abs(x) - 1.0) < 1e-300
    if np.any(at_end):
        dp = np.where(at_end, np.sign(x) ** (n + 1) * n * (n + 1) / 2.0, dp)
    return p1, dp


def gauss_legendre(q):
    """q-point Gauss-Legendre nodes (ascending) and weights on [-1, 1].

    Golub-Welsch: the nodes are the eigenvalues of the symmetric tridiagonal
    Jacobi matrix of the Legendre recurrence, b_m = m / sqrt(4 m^2 - 1); then two
    Newton steps on P_q polish them, and w = 2 / ((1 - x^2) P_q'(x)^2).
    Exact for polynomials of degree 2q - 1.
    """
    if q < 1:
        raise ValueError("q >= 1")
    m = np.arange(1, q, dtype=np.float64)
    b = m / np.sqrt(4.0 * m * m - 1.0)
    J = np.diag(b, 1) + np.diag(b, -1)
    x = np.sort(np.linalg.eigvalsh(J))
    for _ in range(2):
        p, dp = legendre_and_derivative(q, x)
        x = x - p / dp
    _, dp = legendre_and_derivative(q, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    return x, w


def gauss_lobatto(n_pts):
    """n_pts-point Gauss-Legendre-Lobatto nodes (ascending, including +-1) and
    weights on [-1, 1]; n_pts >= 2. Interior nodes are the roots of P_n', n =
    n_pts - 1, found by Newton on (1 - x^2) P_n'(x) from the Chebyshev-Lobatto
    points; w = 2 / (n (n + 1) P_n(x)^2). Exact for degree 2 n_pts - 3."""
    if n_pts < 2:
        raise ValueError("GLL needs at least 2 points")
    n = n_pts - 1
    x = -np.cos(np.pi * np.arange(n_pts) / n)
    for _ in range(100):
        p, dp = legendre_and_derivative(n, x)
        # f = (1-x^2) P_n' ; f' = -n(n+1) P_n (Legendre ODE)
        f = (1.0 - x * x) * dp
        fp = -n * (n + 1) * p
        step = np.zeros_like(x)
        step[1:-1] = f[1:-1] / fp[1:-1]
        x = x - step
        if np.max(np.abs(step)) < 1e-16:
            break
    x[0], x[-1] = -1.0, 1.0
    p, _ = legendre_and_derivative(n, x)
    w = 2.0 / (n * (n + 1) * p * p)
    return x, w


def barycentric_weights(nodes):
    """W_j = 1 / prod_{m != j} (x_j - x_m)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    n = len(nodes)
    W = np.ones(n)
    for j in range(n):
        for m in range(n):
            if m != j:
                W[j] /= nodes[j] - nodes[m]
    return W


def lagrange_matrix(nodes, x):
    """L[i, j] = ell_j(x_i): the Lagrange basis on `nodes` evaluated at points x,
    by the second barycentric form (Sec. 4). A point that coincides with a node
    gets the exact Kronecker row."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    if n == 1:
        return np.ones((len(x), 1))
    W = barycentric_weights(nodes)
    L = np.zeros((len(x), n))
    for i, xi in enumerate(x):
        d = xi - nodes
        hit = np.nonzero(d == 0.0)[0]
        if len(hit):
            L[i, hit[0]] = 1.0
            continue
        t = W / d
        L[i] = t / t.sum()
    return L


def differentiation_matrix(nodes):
    """D[i, j] = ell_j'(x_i) at the nodes themselves (barycentric form)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    n = len(nodes)
    if n == 1:
        return np.zeros((1, 1))
    W = barycentric_weights(nodes)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (W[j] / W[i]) / (nodes[i] - nodes[j])
        D[i, i] = -D[i].sum()
    return D


def lagrange_derivative_matrix(nodes, x):
    """L'[i, j] = ell_j'(x_i). ell_j' has degree p - 1, so it equals the
    interpolant of its nodal values D[:, j]: L' = L(x) D."""
    return lagrange_matrix(nodes, x) @ differentiation_matrix(nodes)


def volume_nodes(p):
    """1-D nodes of the degree-p volume basis: GLL for p >= 1, [0] for p = 0."""
    if p == 0:
        return np.array([0.0])
    return gauss_lobatto(p + 1)[0]


def trace_nodes(p):
    """Nodes of the degree-p trace basis on an edge: the p + 1 GL points."""
    return gauss_legendre(p + 1)[0]
