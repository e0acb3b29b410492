"""Nested p/h geometric multigrid for the condensed HDG trace system, float64
CPU oracle (test infrastructure only).

Paper passages followed (Sec. 6, "Multigrid algorithm"):
  * nested strategy: p-multigrid on the fixed mesh with full arithmetic
    coarsening p, p-1, ..., 0; at p = 0 an h-multigrid on continuous Q1 spaces;
    a direct solve on the coarsest mesh.
  * Eq. eq_mg_pro: p-prolongation is the natural embedding of degree-p edge
    functions into degree p+1 (per edge, a dense (p+2) x (p+1) matrix in the
    nodal trace basis).
  * Eq. eq_mg_res: restriction is the adjoint of prolongation; on residual
    (dual) vectors in coefficient space that is R = P^T.
  * Eq. eq_h_mg_pro: P_J maps continuous Q1 (zero on the boundary) on the finest
    mesh into the p = 0 trace space by L2 projection of its skeleton trace; for a
    function linear along an edge that is the mean of the two end values.
    Between Q1 meshes P is the identity embedding (bilinear interpolation).
  * Eq. eq_h_mg_res: R = P^T on the h-levels. Coarse h-operators are Galerkin
    triple products A_{l-1} = R A_l P (subspace inheritance) for the range the
    paper gives, 1 <= l <= J-1; that range leaves out A_{J-1}, the Q1 operator on
    the finest mesh. Reading: A_{J-1} is the conforming Q1 stiffness matrix of
    (kappa grad u, grad v) on the finest mesh (2-point Gauss rule per direction,
    exact for bilinears), as in the HDG h-multigrid the paper follows.
  * Coarse p-operators. The paper rediscretises the p-levels (subspace
    non-inheritance). With tau = 1 the rediscretised degree-(p-1) operator is up
    to ~30x weaker than the Galerkin one P^T A_p P on some modes (measured by
    their generalized eigenvalues), and the V-cycle then diverges at k = 1.
    Reading: coarse p-operators are Galerkin, A_{p-1} = P^T A_p P, which is
    again a sum of element blocks P_K^T S_K P_K because P acts per edge.
    coarse_op="rediscretize" keeps the paper's literal choice for comparison.
  * Sec. 6.4.1: FSAI smoother x += G^T G (f - A x) (the SPAI step with the
    factorized inverse for a symmetric operator), G from fsai_factor. Readings:
    the paper's "operator complexity of unity" is G on the lower-triangular
    pattern of A (applying G^T G then costs about one product with A); its more
    aggressive variant (complexity ~2.5) is the pattern of A^2; no damping, as
    in the printed update.
  * Sec. 6.4.2: weighted additive Schwarz smoother x += W M (f - A x),
    M = sum_e R_e^T A_e^-1 R_e, dense local blocks applied unassembled.
    Reading: the patch is one element (its 4 faces); A_e is the assembled
    operator restricted to those faces' interior dofs; W = diag(1 / number of
    patches sharing the dof) = 1/2.
  * Alg. 1 (hMG) and Alg. 2 (pMG) V-cycles with nu1 = nu2 = 2; Chebyshev
    smoothing on the h-levels (including the p = 0 level). Reading: each smoothing
    step is a Jacobi-preconditioned Chebyshev iteration of degree 2 on
    [0.1, 1.1] * lambda_max(D^-1 A), lambda_max from 10 power iterations started
    from the integer pattern s_i = ((7919 i) mod 1009) / 1009 - 1/2.
  * Sec. 7: the convergence factor rho_k = |r_k| / |r_{k-1}| of the fine residual
    with multigrid used as a stationary solver.
"""
import numpy as np
import scipy.sparse as sp
import scipy.linalg as sla

from . import quadrature as qd
from .hdg import HDGProblem


def p_prolongation_1d(p):
    """Per-edge embedding of degree-p trace functions into degree p+1:
    P[a', a] = mu_a^{(p)}(x_{a'}^{(p+1)}), the degree-p nodal basis at the
    degree-(p+1) GL nodes (Eq. eq_mg_pro)."""
    return qd.lagrange_matrix(qd.trace_nodes(p), qd.trace_nodes(p + 1))


def p_prolongation(n_edges, p):
    """Block-diagonal P over all edges: coarse dofs (degree p) -> fine (p+1)."""
    return sp.kron(sp.identity(n_edges), sp.csr_matrix(p_prolongation_1d(p))).tocsr()


def q1_to_p0(mesh):
    """P_J of Eq. eq_h_mg_pro: interior vertices of the Q1 space on the finest
    mesh -> p = 0 trace dofs (one per edge): edge value = mean of the two end
    vertex values (boundary vertices are 0)."""
    nx, ny = mesh.nx, mesh.ny
    nvi = (nx - 1) * (ny - 1)

    def vid(i, j):
        if i <= 0 or j <= 0 or i >= nx or j >= ny:
            return -1
        return (i - 1) + (nx - 1) * (j - 1)

    rows, cols, vals = [], [], []
    for j in range(ny):                 # vertical edges (i, j)-(i, j+1)
        for i in range(nx + 1):
            ed = mesh.vedge(i, j)
            for v in (vid(i, j), vid(i, j + 1)):
                if v >= 0:
                    rows.append(ed); cols.append(v); vals.append(0.5)
    for j in range(ny + 1):             # horizontal edges (i, j)-(i+1, j)
        for i in range(nx):
            ed = mesh.hedge(i, j)
            for v in (vid(i, j), vid(i + 1, j)):
                if v >= 0:
                    rows.append(ed); cols.append(v); vals.append(0.5)
    return sp.csr_matrix((vals, (rows, cols)), shape=(mesh.n_edges, nvi))


def q1_prolongation(nxc, nyc):
    """Bilinear interpolation of interior-vertex Q1 functions from an nxc x nyc
    mesh to the 2nxc x 2nyc mesh (the identity embedding M_{l-1} in M_l)."""
    nxf, nyf = 2 * nxc, 2 * nyc

    def cid(i, j):
        if i <= 0 or j <= 0 or i >= nxc or j >= nyc:
            return -1
        return (i - 1) + (nxc - 1) * (j - 1)

    rows, cols, vals = [], [], []
    for jf in range(1, nyf):
        for i_f in range(1, nxf):
            r = (i_f - 1) + (nxf - 1) * (jf - 1)
            xs = [(i_f // 2, 1.0)] if i_f % 2 == 0 else [(i_f // 2, 0.5), (i_f // 2 + 1, 0.5)]
            ys = [(jf // 2, 1.0)] if jf % 2 == 0 else [(jf // 2, 0.5), (jf // 2 + 1, 0.5)]
            for (ic, wx) in xs:
                for (jc, wy) in ys:
                    c = cid(ic, jc)
                    if c >= 0:
                        rows.append(r); cols.append(c); vals.append(wx * wy)
    return sp.csr_matrix((vals, (rows, cols)), shape=((nxf - 1) * (nyf - 1), (nxc - 1) * (nyc - 1)))


def interior_trace_dofs(mesh, p):
    ie = mesh.interior_edges()
    return (ie[:, None] * (p + 1) + np.arange(p + 1)).ravel()


def q1_stiffness(mesh, kappa):
    """Conforming Q1 stiffness of (kappa grad u, grad v) over interior vertices
    (u = 0 on the boundary), per-element constant kappa, by the 2 x 2 Gauss rule
    on each rectangle (exact for products of bilinear gradients)."""
    nx, ny, hx, hy = mesh.nx, mesh.ny, mesh.hx, mesh.hy
    gp, gw = qd.gauss_legendre(2)
    s_pts = (gp + 1) / 2            # on [0, 1]
    s_w = gw / 2

    def vid(i, j):
        if i <= 0 or j <= 0 or i >= nx or j >= ny:
            return -1
        return (i - 1) + (nx - 1) * (j - 1)

    # bilinear basis on [0,1]^2 with vertices (0,0), (1,0), (0,1), (1,1)
    corners = [(0, 0), (1, 0), (0, 1), (1, 1)]
    Ke = np.zeros((4, 4))
    for a_, (s_q, ws) in enumerate(zip(s_pts, s_w)):
        for b_, (t_q, wt) in enumerate(zip(s_pts, s_w)):
            grads = []
            for (cx, cy) in corners:
                fx = s_q if cx else 1 - s_q
                fy = t_q if cy else 1 - t_q
                dfx = (1 if cx else -1) / hx
                dfy = (1 if cy else -1) / hy
                grads.append((dfx * fy, fx * dfy))
            for a in range(4):
                for b in range(4):
                    Ke[a, b] += ws * wt * hx * hy * (grads[a][0] * grads[b][0] + grads[a][1] * grads[b][1])
    rows, cols, vals = [], [], []
    for j in range(ny):
        for i in range(nx):
            vs = [vid(i, j), vid(i + 1, j), vid(i, j + 1), vid(i + 1, j + 1)]
            kap = kappa[i + nx * j]
            for a in range(4):
                for b in range(4):
                    if vs[a] >= 0 and vs[b] >= 0:
                        rows.append(vs[a]); cols.append(vs[b]); vals.append(kap * Ke[a, b])
    n = (nx - 1) * (ny - 1)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def power_start(n):
    i = np.arange(n, dtype=np.int64)
    return ((7919 * i) % 1009) / 1009.0 - 0.5


def lambda_max_jacobi(A, iters=10):
    """Power iteration on D^-1 A from the fixed integer pattern."""
    d = A.diagonal()
    x = power_start(A.shape[0])
    x = x / np.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        y = (A @ x) / d
        lam = np.linalg.norm(y)
        x = y / lam
    return lam


def chebyshev(A, dinv, lmax, f, x, degree=2, lo=0.1, hi=1.1):
    """One Jacobi-preconditioned Chebyshev smoothing step of the given degree on
    [lo, hi] * lmax (the classical three-term Chebyshev iteration)."""
    a, b = lo * lmax, hi * lmax
    theta = 0.5 * (b + a)
    delta = 0.5 * (b - a)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = f - A @ x
    d = dinv * r / theta
    x = x + d
    for _ in range(1, degree):
        r = r - A @ d
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (dinv * r)
        rho = rho_new
        x = x + d
    return x


def fsai_factor(A, pattern):
    """Factorized sparse approximate inverse of an SPD matrix (Sec. 6.4.1): the
    lower-triangular G with the given sparsity (a sparse matrix whose lower
    triangle, diagonal included, is the allowed pattern) that minimises
    |I - G L|_F, L the Cholesky factor of A, normalised so that G A G^T has a
    unit diagonal; M = G^T G approximates A^-1. Row i is independent of the
    others: with J the allowed columns of row i (all <= i),
    A[J, J] g = e_i, then G[i, J] = g / sqrt(g_i)."""
    A = sp.csr_matrix(A)
    P = sp.tril(sp.csr_matrix(pattern), format="csr")
    n = A.shape[0]
    rows, cols, vals = [], [], []
    Ad = A.tolil()
    for i in range(n):
        J = P.indices[P.indptr[i]:P.indptr[i + 1]]
        J = np.unique(np.append(J, i))
        AJ = Ad[J][:, J].toarray()
        rhs = (J == i).astype(np.float64)
        g = np.linalg.solve(AJ, rhs)
        g = g / np.sqrt(g[J == i][0])
        rows.extend([i] * len(J))
        cols.extend(J.tolist())
        vals.extend(g.tolist())
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


class PLevel:
    """One p-level on the fixed mesh: interior-dof matrix and its smoother
    (weighted ASM blocks, or FSAI)."""

    def __init__(self, mesh, p, kappa, tau=1.0, A=None, smoother="asm", fsai_pattern="A"):
        self.p = p
        self.prob = HDGProblem(mesh, p, kappa, tau)
        if A is None:
            self.A, self.idx = self.prob.assemble_interior()
        else:
            self.A, self.idx = A, self.prob.interior_dofs()
        self.ndof = self.prob.ndof
        nint = len(self.idx)
        gmap = -np.ones(self.ndof, dtype=np.int64)
        gmap[self.idx] = np.arange(nint)
        self.gmap = gmap
        # element patches: interior dofs of the element's 4 faces
        Ad = self.A.tocsr()
        self.patches = []
        count = np.zeros(nint)
        for e in range(mesh.nel):
            loc = gmap[self.prob.dofs(e)]
            loc = loc[loc >= 0]
            if len(loc) == 0:
                continue
            Ae = Ad[loc][:, loc].toarray()
            self.patches.append((loc, np.linalg.inv(Ae)))
            count[loc] += 1
        self.weight = 1.0 / count
        self.smoother = smoother
        if smoother == "fsai":
            # pattern of A (operator complexity one: applying G^T G costs about
            # one product with A) or of A^2 (a wider, stronger approximate inverse)
            pat = self.A if fsai_pattern == "A" else (self.A @ self.A)
            self.G = fsai_factor(self.A, pat)
        elif smoother != "asm":
            raise ValueError(smoother)

    def fsai(self, r):
        """z = G^T G r."""
        return self.G.T @ (self.G @ r)

    def asm(self, r):
        """z = W M r, M = sum_e R_e^T A_e^-1 R_e."""
        z = np.zeros_like(r)
        for loc, Ainv in self.patches:
            z[loc] += Ainv @ r[loc]
        return self.weight * z

    def smooth(self, f, x, nu):
        M = self.fsai if self.smoother == "fsai" else self.asm
        for _ in range(nu):
            x = x + M(f - self.A @ x)
        return x


class HLevel:
    """An h-level operator (p = 0 HDG or Q1 Galerkin) with Chebyshev data."""

    def __init__(self, A):
        self.A = A.tocsr()
        self.dinv = 1.0 / self.A.diagonal()
        self.lmax = lambda_max_jacobi(self.A)

    def smooth(self, f, x, nu):
        for _ in range(nu):
            x = chebyshev(self.A, self.dinv, self.lmax, f, x)
        return x


class NestedGMG:
    """Alg. 2 (p-levels k..1) over Alg. 1 (p = 0 and the Q1 levels).

    Interior-dof vectors at the finest p-level are used throughout; the public
    vcycle() takes and returns vectors on ALL trace dofs (boundary entries 0)."""

    def __init__(self, mesh, k, kappa, tau=1.0, nu1=2, nu2=2, coarse_n=2,
                 coarse_op="galerkin", smoother="asm", fsai_pattern="A"):
        self.mesh, self.k, self.nu1, self.nu2 = mesh, k, nu1, nu2
        kappa = np.asarray(kappa, dtype=np.float64).reshape(mesh.nel)
        sm = dict(smoother=smoother, fsai_pattern=fsai_pattern)
        if coarse_op == "rediscretize":
            self.plevels = {p: PLevel(mesh, p, kappa, tau, **sm) for p in range(k, -1, -1)}
        elif coarse_op == "galerkin":
            self.plevels = {k: PLevel(mesh, k, kappa, tau, **sm)}
        else:
            raise ValueError(coarse_op)
        # p-transfers between interior-dof vectors; Galerkin coarse p-operators
        self.Pp = {}
        for p in range(k - 1, -1, -1):
            fine = self.plevels[p + 1]
            P = p_prolongation(mesh.n_edges, p)
            ic = interior_trace_dofs(mesh, p)
            self.Pp[p + 1] = P[fine.idx][:, ic].tocsr()
            if coarse_op == "galerkin":
                Ac = (self.Pp[p + 1].T @ fine.A @ self.Pp[p + 1]).tocsr()
                self.plevels[p] = PLevel(mesh, p, kappa, tau, A=Ac, **sm)
        # h-levels: index 0 = p = 0 HDG (interior edges), then Q1 finest..coarsest
        A0 = self.plevels[0].A
        PJ = q1_to_p0(mesh)[self.plevels[0].idx]
        self.hP = [PJ.tocsr()]
        self.hA = [A0]
        nx, ny = mesh.nx, mesh.ny
        Aq = q1_stiffness(mesh, kappa)
        self.hA.append(Aq)
        self.hsizes = [(nx, ny)]
        while nx % 2 == 0 and ny % 2 == 0 and nx // 2 >= coarse_n and ny // 2 >= coarse_n \
                and nx > coarse_n:
            P = q1_prolongation(nx // 2, ny // 2)
            nx, ny = nx // 2, ny // 2
            Aq = (P.T @ Aq @ P).tocsr()
            self.hP.append(P)
            self.hA.append(Aq)
            self.hsizes.append((nx, ny))
        self.hlev = [HLevel(A) for A in self.hA[:-1]]
        Ac = self.hA[-1].toarray()
        self.coarse = sla.cho_factor(Ac) if Ac.shape[0] > 0 else None

    # Alg. 1
    def hmg(self, l, r):
        if l == len(self.hA) - 1:
            return sla.cho_solve(self.coarse, r) if self.coarse is not None else np.zeros_like(r)
        lev = self.hlev[l]
        v = lev.smooth(r, np.zeros_like(r), self.nu1)
        rc = self.hP[l].T @ (r - lev.A @ v)
        vc = self.hmg(l + 1, rc)
        v = v + self.hP[l] @ vc
        return lev.smooth(r, v, self.nu2)

    # Alg. 2
    def pmg(self, p, r):
        if p == 0:
            return self.hmg(0, r)
        lev = self.plevels[p]
        v = lev.smooth(r, np.zeros_like(r), self.nu1)
        rc = self.Pp[p].T @ (r - lev.A @ v)
        vc = self.pmg(p - 1, rc)
        v = v + self.Pp[p] @ vc
        return lev.smooth(r, v, self.nu2)

    def fmg(self, b_full, cycles=1):
        """Full multigrid (Sec. 7): the right-hand side restricted to every level
        (R = P^T), a direct solve on the coarsest mesh, then level by level
        upwards: the coarser solution interpolated (P) as the start, improved
        by `cycles` V-cycles of that level's own hierarchy (Alg. 1 on the h-levels,
        Alg. 2 on the p-levels) applied to its residual. Returns the finest
        p-level solution on ALL trace dofs (boundary entries 0)."""
        top = self.plevels[self.k]
        bp = {self.k: np.asarray(b_full)[top.idx]}
        for p in range(self.k, 0, -1):
            bp[p - 1] = self.Pp[p].T @ bp[p]
        bh = [bp[0]]                       # h-level 0 is the p = 0 level
        for l in range(len(self.hA) - 1):
            bh.append(self.hP[l].T @ bh[l])
        L = len(self.hA) - 1
        x = sla.cho_solve(self.coarse, bh[L]) if self.coarse is not None else np.zeros_like(bh[L])
        for l in range(L - 1, -1, -1):
            x = self.hP[l] @ x
            for _ in range(cycles):
                x = x + self.hmg(l, bh[l] - self.hA[l] @ x)
        for p in range(1, self.k + 1):
            x = self.Pp[p] @ x
            for _ in range(cycles):
                x = x + self.pmg(p, bp[p] - self.plevels[p].A @ x)
        out = np.zeros(top.ndof)
        out[top.idx] = x
        return out

    def vcycle(self, r_full):
        top = self.plevels[self.k]
        z = np.zeros(top.ndof)
        z[top.idx] = self.pmg(self.k, np.asarray(r_full)[top.idx])
        return z

    def apply(self, x_full):
        top = self.plevels[self.k]
        y = np.zeros(top.ndof)
        y[top.idx] = top.A @ np.asarray(x_full)[top.idx]
        return y

    def stationary(self, b_full, cycles):
        """Multigrid as a solver; returns x and the residual norm history."""
        x = np.zeros_like(b_full)
        hist = [np.linalg.norm(b_full)]
        for _ in range(cycles):
            r = b_full - self.apply(x)
            x = x + self.vcycle(r)
            hist.append(np.linalg.norm(b_full - self.apply(x)))
        return x, np.array(hist)

    def pcg(self, b_full, rtol=1e-10, maxit=200):
        """CG preconditioned by one V-cycle; stops at |r| / |b| <= rtol."""
        x = np.zeros_like(b_full)
        r = b_full.copy()
        bn = np.linalg.norm(b_full)
        hist = [1.0]
        if bn == 0.0:
            return x, 0, np.array(hist)
        z = self.vcycle(r)
        pdir = z.copy()
        rz = r @ z
        it = 0
        for it in range(1, maxit + 1):
            Ap = self.apply(pdir)
            alpha = rz / (pdir @ Ap)
            x += alpha * pdir
            r -= alpha * Ap
            rel = np.linalg.norm(r) / bn
            hist.append(rel)
            if rel <= rtol:
                break
            z = self.vcycle(r)
            rz_new = r @ z
            pdir = z + (rz_new / rz) * pdir
            rz = rz_new
        return x, it, np.array(hist)


def convergence_factor(hist, first=2, last=8):
    """Geometric mean of rho_k = |r_k| / |r_{k-1}| over cycles first..last."""
    h = np.asarray(hist)
    last = min(last, len(h) - 1)
    return (h[last] / h[first - 1]) ** (1.0 / (last - first + 1))
