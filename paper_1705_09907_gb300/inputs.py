"""Seeded synthetic inputs for the HDG trace solver workloads.

These generators produce coefficient fields, source samples and observation
noise. They contain none of the discretisation's arithmetic and are shared by
the GPU tests, the benchmark and the CPU oracle checks, so both sides see the
same inputs. Source samples are taken at Gauss-Legendre points computed with
numpy's own `leggauss` (a library routine, independent of both solvers).

Workloads (uniform N x N quads on the unit square, element e = i + N j):
  * manufactured Poisson: kappa = 1, f = 2 pi^2 sin(pi x) sin(pi y)
  * lognormal diffusion: kappa = exp(g), g a zero-mean Gaussian field with
    variance sigma^2 and squared-exponential covariance exp(-r^2 / (2 l^2)) on
    the element centres, l = 0.05; f = 1
  * batched Fourier right-hand sides: f_j = sum_{m1,m2=1..4} c_jm sin(pi m1 x)
    sin(pi m2 y), c_jm ~ N(0, 1) / (m1^2 + m2^2)
  * uneven instance mix: N_i in {64, 128, 256, 512}, k_i in {2, 3, 4}
"""
import numpy as np


def gl_points_1d(q):
    """q Gauss-Legendre points on [-1, 1] (numpy.polynomial.legendre.leggauss)."""
    x, _ = np.polynomial.legendre.leggauss(q)
    return x


def element_sample_points(n, k, x0=0.0, y0=0.0, x1=1.0, y1=1.0, ny=None):
    """Coordinates of the (k+2) x (k+2) GL sample points of every element of an
    n x ny mesh: X, Y of shape [nel, k+2, k+2], index [e, jy, ix]."""
    ny = n if ny is None else ny
    hx, hy = (x1 - x0) / n, (y1 - y0) / ny
    g = (gl_points_1d(k + 2) + 1.0) / 2.0
    i = np.arange(n)
    j = np.arange(ny)
    # [ny, n, q] coordinates
    xs = x0 + (i[:, None] + g[None, :]) * hx            # [n, q]
    ys = y0 + (j[:, None] + g[None, :]) * hy            # [ny, q]
    X = np.broadcast_to(xs[None, :, None, :], (ny, n, k + 2, k + 2))
    Y = np.broadcast_to(ys[:, None, :, None], (ny, n, k + 2, k + 2))
    return X.reshape(n * ny, k + 2, k + 2).copy(), Y.reshape(n * ny, k + 2, k + 2).copy()


def manufactured_poisson_f(n, k):
    """f = 2 pi^2 sin(pi x) sin(pi y) at the sample points (u = sin pi x sin pi y)."""
    X, Y = element_sample_points(n, k)
    return 2.0 * np.pi ** 2 * np.sin(np.pi * X) * np.sin(np.pi * Y)


def constant_f(n, k, value=1.0, ny=None):
    ny = n if ny is None else ny
    return np.full((n * ny, k + 2, k + 2), float(value))


def gaussian_field(n, seed, corr_len=0.05, variance=1.0, ny=None):
    """Zero-mean Gaussian field on the element centres of an n x ny unit-square
    mesh with covariance variance * exp(-r^2 / (2 corr_len^2)).

    The covariance is separable, C = C_x (x) C_y, so the sample is
    G = (V_y L_y^1/2) Z (V_x L_x^1/2)^T with 1-D eigendecompositions (negative
    eigenvalues from round-off clipped to 0) and Z ~ N(0, 1) drawn by numpy's
    PCG64 generator with the given seed. Returns g flattened as e = i + n j."""
    ny = n if ny is None else ny

    def factor(m):
        c = (np.arange(m) + 0.5) / m
        C = np.exp(-(c[:, None] - c[None, :]) ** 2 / (2.0 * corr_len ** 2))
        w, V = np.linalg.eigh(C)
        return V * np.sqrt(np.clip(w, 0.0, None))[None, :]

    Ax = factor(n)
    Ay = Ax if ny == n else factor(ny)
    Z = np.random.default_rng(seed).standard_normal((ny, n))
    G = np.sqrt(variance) * (Ay @ Z @ Ax.T)
    return G.reshape(-1)


def lognormal_kappa(n, seed, corr_len=0.05, variance=1.0):
    return np.exp(gaussian_field(n, seed, corr_len, variance))


def fourier_rhs(n, k, nrhs, seed, modes=4):
    """nrhs source fields f_j sampled at the element GL points: [nrhs, nel, k+2, k+2]."""
    rng = np.random.default_rng(seed)
    m = np.arange(1, modes + 1)
    decay = 1.0 / (m[:, None] ** 2 + m[None, :] ** 2)
    c = rng.standard_normal((nrhs, modes, modes)) * decay[None]
    X, Y = element_sample_points(n, k)
    sx = np.sin(np.pi * m[:, None, None, None] * X[None])     # [modes, nel, q, q]
    sy = np.sin(np.pi * m[:, None, None, None] * Y[None])
    return np.einsum("jab,anqr,bnqr->jnqr", c, sx, sy)


def instance_mix(count=12, seed=4, sizes=(64, 128, 256, 512), degrees=(2, 3, 4)):
    """Uneven list of (N, k) instances drawn with replacement."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=count, replace=True)
    ks = rng.choice(np.asarray(degrees), size=count, replace=True)
    return [(int(a), int(b)) for a, b in zip(ns, ks)]


def random_trace(n_edges, k, seed, nrhs=None):
    """Standard normal trace vector(s) [n_edges * (k+1)] or [n_edges * (k+1), nrhs]."""
    rng = np.random.default_rng(seed)
    shape = (n_edges * (k + 1),) if nrhs is None else (n_edges * (k + 1), nrhs)
    return rng.standard_normal(shape)


def observation_noise(size, seed, std=1e-3):
    return np.random.default_rng(seed).normal(0.0, std, size=size)


def _bump_1d(t):
    """a(t) = t (t - 1) exp(-t^2) and its first two derivatives."""
    e = np.exp(-t * t)
    return ((t * t - t) * e, (-2 * t ** 3 + 2 * t * t + 2 * t - 1) * e,
            (4 * t ** 4 - 4 * t ** 3 - 10 * t * t + 6 * t + 2) * e)


def bump_solution(X, Y):
    """The manufactured solution of the paper's Sec. 5 experiment,
    u = x (x - 1) y (y - 1) exp(-x^2 - y^2) = a(x) a(y), its flux q = -grad u
    (K = 1) and f = -laplace u, at the points X, Y (any shape)."""
    ax, dax, ddax = _bump_1d(np.asarray(X, dtype=np.float64))
    ay, day, dday = _bump_1d(np.asarray(Y, dtype=np.float64))
    return ax * ay, (-dax * ay, -ax * day), -(ddax * ay + ax * dday)


def bump_f(n, k):
    """f of bump_solution at the (k+2) x (k+2) GL sample points of an n x n mesh."""
    X, Y = element_sample_points(n, k)
    return bump_solution(X, Y)[2]
