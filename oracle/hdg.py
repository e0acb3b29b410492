"""HDG (LDG-H) discretisation of -div(kappa grad u) = f, u = 0 on the boundary, on a
Cartesian quad mesh; float64 CPU oracle (test infrastructure only).

Paper passages followed:
  * Eq. eq2: mixed form kappa^-1 q + grad u = 0, div q = f.
  * Eqs. eq_h1-eq_h3: the HDG weak form. Reading: the volume term of eq_h1 is
    (kappa^-1 q_h, v) (the paper drops K^-1; the strong form of Eq. eq2 and the
    LDG-H method it cites have it). With g_D = 0, P_h g_D = 0 and the trace is 0 on
    boundary edges, so the interior-edge and boundary-edge terms of eq_h2 merge
    into one sum over all faces with lambda = 0 on the boundary.
  * Eqs. static_1, static_2: element matrices A_K, B_K, C_K, D_K, E_K, F_K.
  * Eq. shur0: local solver [Q; U] = L_K^-1 (-[C; E] Lambda + [R; F]).
  * Eq. shur1: per interior edge, the sum over its two elements of
    G Q + tau H U - tau M Lambda vanishes. Multiplying out gives the condensed
    operator sum_K A_K^T S_K A_K with S_K = [G  tau H] L_K^-1 [C; E] + tau M_dK.
  * Procedure (i)-(iv) of Sec. 3 and Alg. 3 (the per-edge assembly-free apply).
  * tau = 1 on every facet (Sec. 5, for the model problem).

Layouts (shared only as a specification with the GPU library):
  volume unknowns per element: Q = [Qx (n), Qy (n)], U (n); n = (p+1)^2, nodal
  at the GLL tensor grid, index I = i + j (p+1) (i along x).
  trace unknowns per element: Lambda = [W, E, S, N] faces x (p+1) GL nodes.
  f input: samples at the (p+2) x (p+2) GL points of each element (any nq x nq
  GL tensor grid is accepted; Table 1 of Sec. 5 uses nq = p + 1),
  f_q[e, jy, ix] (x fastest).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import quadrature as qd
from .mesh import Mesh

FACES = ("W", "E", "S", "N")


class RefElement:
    """Reference-coordinate tables for degree p on an hx x hy rectangle."""

    def __init__(self, p, hx, hy, nquad=None):
        self.p = p
        self.hx, self.hy = hx, hy
        self.n1 = p + 1
        self.n = (p + 1) ** 2
        self.m = 4 * (p + 1)
        self.vnodes = qd.volume_nodes(p)
        self.tnodes = qd.trace_nodes(p)
        nq = p + 2 if nquad is None else nquad
        self.nq = nq
        self.xq, self.wq = qd.gauss_legendre(nq)
        # 1-D volume basis and its derivative at the quadrature points
        self.B1 = qd.lagrange_matrix(self.vnodes, self.xq)            # [nq, p+1]
        if p == 0:
            self.D1 = np.zeros((nq, 1))
        else:
            self.D1 = qd.lagrange_derivative_matrix(self.vnodes, self.xq)
        # trace basis at the quadrature points
        self.T1 = qd.lagrange_matrix(self.tnodes, self.xq)            # [nq, p+1]
        # volume basis at the ends of [-1, 1]
        self.B1m = qd.lagrange_matrix(self.vnodes, [-1.0])[0]         # [p+1]
        self.B1p = qd.lagrange_matrix(self.vnodes, [1.0])[0]

    def phi_at_quad(self):
        """V[qy*nq+qx, I] = phi_I at tensor quadrature point (qx, qy)."""
        return np.kron(self.B1, self.B1)   # row index qy*nq+qx, col i + j(p+1)

    def dphidx_at_quad(self):
        return np.kron(self.B1, self.D1) * (2.0 / self.hx)

    def dphidy_at_quad(self):
        return np.kron(self.D1, self.B1) * (2.0 / self.hy)

    def quad_weights(self):
        J = self.hx * self.hy / 4.0
        return np.kron(self.wq, self.wq) * J

    def face_tables(self, f):
        """For face f: (phi values at face quadrature points [nq, n],
        trace basis at those points [nq, p+1], line weights [nq], normal (nx, ny))."""
        p1 = self.n1
        if f in (0, 1):   # W / E: xi = -1 / +1, varying eta (along y)
            end = self.B1m if f == 0 else self.B1p
            phi = np.zeros((self.nq, self.n))
            for j in range(p1):
                for i in range(p1):
                    phi[:, i + j * p1] = end[i] * self.B1[:, j]
            w = self.wq * self.hy / 2.0
            nrm = (-1.0, 0.0) if f == 0 else (1.0, 0.0)
        else:             # S / N: eta = -1 / +1, varying xi (along x)
            end = self.B1m if f == 2 else self.B1p
            phi = np.zeros((self.nq, self.n))
            for j in range(p1):
                for i in range(p1):
                    phi[:, i + j * p1] = self.B1[:, i] * end[j]
            w = self.wq * self.hx / 2.0
            nrm = (0.0, -1.0) if f == 2 else (0.0, 1.0)
        return phi, self.T1, w, nrm


def element_matrices(ref, kappa, tau=1.0, kappa_q=None):
    """Element matrices of Eqs. static_1 / static_2 and the flux rows of Eq. shur1.

    Returns a dict with
      A  [2n, 2n]   (kappa^-1 q, v)
      B  [n, 2n]    B[i, (c, j)] = (phi_i, d_c phi_j)            (eq_h1 uses -B^T)
      B2 [n, 2n]    -(q, grad w) + <q.n, w>_dK, taken literally from eq_h2
      C  [2n, m]    C[(c, i), (f, a)] = <mu_a, phi_i n_c>_f
      D  [n, n]     tau <phi_j, phi_i>_dK
      E  [n, m]     -tau <mu_a, phi_i>_f
      G  [m, 2n]    <phi_i n_c, mu_a>_f   (= C^T)
      H  [m, n]     <phi_i, mu_a>_f
      Ml [m, m]     <mu_b, mu_a>_f (face mass)
    kappa_q: optional kappa values at the tensor quadrature points (for a
    coefficient that varies inside the element); otherwise kappa is constant.
    """
    n, m, p1 = ref.n, ref.m, ref.n1
    V = ref.phi_at_quad()
    Dx = ref.dphidx_at_quad()
    Dy = ref.dphidy_at_quad()
    wJ = ref.quad_weights()
    kinv = (1.0 / kappa) * np.ones_like(wJ) if kappa_q is None else 1.0 / np.asarray(kappa_q)
    M = V.T @ (wJ[:, None] * V)
    Mk = V.T @ ((wJ * kinv)[:, None] * V)
    A = np.zeros((2 * n, 2 * n))
    A[:n, :n] = Mk
    A[n:, n:] = Mk
    B = np.zeros((n, 2 * n))
    B[:, :n] = V.T @ (wJ[:, None] * Dx)
    B[:, n:] = V.T @ (wJ[:, None] * Dy)
    B2 = np.zeros((n, 2 * n))
    # -(q, grad w): row i (test w = phi_i), column (c, j) (q_c = phi_j)
    B2[:, :n] = -(Dx.T @ (wJ[:, None] * V))
    B2[:, n:] = -(Dy.T @ (wJ[:, None] * V))
    C = np.zeros((2 * n, m))
    D = np.zeros((n, n))
    E = np.zeros((n, m))
    H = np.zeros((m, n))
    Ml = np.zeros((m, m))
    for f in range(4):
        phi, T, w, (nx_, ny_) = ref.face_tables(f)
        sl = slice(f * p1, (f + 1) * p1)
        # <mu_a, phi_i n_c>
        PT = phi.T @ (w[:, None] * T)              # [n, p+1]
        C[:n, sl] += nx_ * PT
        C[n:, sl] += ny_ * PT
        # <q.n, w> part of eq_h2: row i, column (c, j): <phi_j n_c, phi_i>
        PP = phi.T @ (w[:, None] * phi)            # [n, n]
        B2[:, :n] += nx_ * PP
        B2[:, n:] += ny_ * PP
        D += tau * PP
        E[:, sl] += -tau * PT
        H[sl, :] += PT.T
        Ml[sl, sl] += T.T @ (w[:, None] * T)
    G = C.T.copy()
    return dict(A=A, B=B, B2=B2, C=C, D=D, E=E, G=G, H=H, Ml=Ml, M=M, tau=tau,
                V=V, wJ=wJ)


def local_system(mats):
    """L_K of Eq. shur0: [[A, -B^T], [B2, D]] (B2 is eq_h2's q-block)."""
    A, B, B2, D = mats["A"], mats["B"], mats["B2"], mats["D"]
    n = D.shape[0]
    L = np.zeros((3 * n, 3 * n))
    L[:2 * n, :2 * n] = A
    L[:2 * n, 2 * n:] = -B.T
    L[2 * n:, :2 * n] = B2
    L[2 * n:, 2 * n:] = D
    return L


def schur_block(mats):
    """S_K = [G  tau H] L_K^-1 [C; E] + tau M_dK  (from Eqs. shur0 and shur1; the
    sign makes S_K symmetric positive semi-definite)."""
    L = local_system(mats)
    CE = np.vstack([mats["C"], mats["E"]])
    GH = np.hstack([mats["G"], mats["tau"] * mats["H"]])
    return GH @ np.linalg.solve(L, CE) + mats["tau"] * mats["Ml"]


def rhs_block(mats, F):
    """b_K = [G  tau H] L_K^-1 [0; F] (the f-part of the edge flux, Eq. shur1)."""
    n = mats["D"].shape[0]
    L = local_system(mats)
    rhs = np.zeros(3 * n)
    rhs[2 * n:] = F
    GH = np.hstack([mats["G"], mats["tau"] * mats["H"]])
    return GH @ np.linalg.solve(L, rhs)


def local_solve(mats, lam_K, F):
    """Eq. shur0: (Q, U) from the element's trace values and load vector."""
    n = mats["D"].shape[0]
    L = local_system(mats)
    rhs = -np.vstack([mats["C"], mats["E"]]) @ lam_K
    rhs[2 * n:] += F
    sol = np.linalg.solve(L, rhs)
    return sol[:2 * n], sol[2 * n:]


def load_vector(ref, mats, f_q_e):
    """F_K[i] = (f, phi_i)_K from samples at the nq x nq GL points of the element
    (x fastest), nq read from the sample count: (p+2)^2 samples are the library's
    input format; (p+1)^2 samples give the (p+1)-point rule with which the paper's
    Table 1 was computed (Sec. 5)."""
    f_q_e = np.asarray(f_q_e).ravel()
    nq = int(round(np.sqrt(f_q_e.size)))
    if nq * nq != f_q_e.size:
        raise ValueError("f samples must form an nq x nq tensor grid")
    xq, wq = qd.gauss_legendre(nq)
    B1 = qd.lagrange_matrix(ref.vnodes, xq)
    V = np.kron(B1, B1)
    wJ = np.kron(wq, wq) * ref.hx * ref.hy / 4.0
    return V.T @ (wJ * f_q_e)


def f_quadrature_points(mesh, p, npts=None):
    """Physical coordinates of the npts x npts GL sample points of every element
    (npts = p + 2 by default, the library's input format): X, Y with shape
    [nel, npts, npts] (index [e, jy, ix])."""
    nq = p + 2 if npts is None else int(npts)
    xq, _ = qd.gauss_legendre(nq)
    X = np.zeros((mesh.nel, nq, nq))
    Y = np.zeros_like(X)
    for e in range(mesh.nel):
        ox, oy = mesh.elem_origin(e)
        gx = ox + mesh.hx * (xq + 1) / 2
        gy = oy + mesh.hy * (xq + 1) / 2
        X[e], Y[e] = np.meshgrid(gx, gy)
    return X, Y


class HDGProblem:
    """All element blocks of one mesh, degree p, per-element kappa.

    tau: the stabilisation on every face of every element, a positive number
    (1 in Sec. 5 for the model problem), or "kappa" for tau_K = kappa_K on the
    faces of element K (tau piecewise constant per element, Sec. 3)."""

    def __init__(self, mesh, p, kappa, tau=1.0, kappa_q_fn=None, nquad=None):
        self.mesh = mesh
        self.p = p
        self.kappa = np.asarray(kappa, dtype=np.float64).reshape(mesh.nel)
        if not (tau == "kappa" or (np.isscalar(tau) and float(tau) > 0.0)):
            raise ValueError("tau must be a positive number or 'kappa'")
        self.tau = tau
        self.ref = RefElement(p, mesh.hx, mesh.hy, nquad=nquad)
        self.n1 = p + 1
        self.m = 4 * (p + 1)
        self.e2e = mesh.elem_to_edge()
        self.edge_elem, self.edge_face = mesh.edge_to_elem()
        self.kappa_q_fn = kappa_q_fn
        self._S = None

    def mats(self, e):
        kq = None
        if self.kappa_q_fn is not None:
            ox, oy = self.mesh.elem_origin(e)
            gx = ox + self.mesh.hx * (self.ref.xq + 1) / 2
            gy = oy + self.mesh.hy * (self.ref.xq + 1) / 2
            X, Y = np.meshgrid(gx, gy)
            kq = self.kappa_q_fn(X.ravel(), Y.ravel())
        return element_matrices(self.ref, self.kappa[e], self.tau_of(e), kappa_q=kq)

    def tau_of(self, e):
        return float(self.kappa[e]) if self.tau == "kappa" else float(self.tau)

    def dofs(self, e):
        """Global trace dof indices of element e's local Lambda_K (the map A_K)."""
        p1 = self.n1
        return np.concatenate([self.e2e[e, f] * p1 + np.arange(p1) for f in range(4)])

    def schur_blocks(self, elems=None):
        """S_K for the given elements (all by default) [len, m, m]."""
        elems = range(self.mesh.nel) if elems is None else elems
        return np.array([schur_block(self.mats(e)) for e in elems])

    def S(self):
        if self._S is None:
            self._S = self.schur_blocks()
        return self._S

    @property
    def ndof(self):
        return self.mesh.n_edges * self.n1

    def interior_dofs(self):
        ie = self.mesh.interior_edges()
        return (ie[:, None] * self.n1 + np.arange(self.n1)).ravel()

    def assemble(self, S=None):
        """Condensed matrix over ALL trace dofs, sum_K A_K^T S_K A_K (step (ii))."""
        S = self.S() if S is None else S
        rows, cols, vals = [], [], []
        for e in range(self.mesh.nel):
            d = self.dofs(e)
            rows.append(np.repeat(d, len(d)))
            cols.append(np.tile(d, len(d)))
            vals.append(S[e].ravel())
        A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.ndof, self.ndof))
        A.sum_duplicates()
        return A

    def assemble_interior(self, S=None):
        """The trace system on interior dofs only (boundary trace = P_h g_D = 0)."""
        A = self.assemble(S)
        idx = self.interior_dofs()
        return A[idx][:, idx].tocsr(), idx

    def apply_assembled(self, x, A_int=None, idx=None):
        """y = A x on all dofs; boundary rows are 0 and boundary x is ignored."""
        if A_int is None:
            A_int, idx = self.assemble_interior()
        y = np.zeros(self.ndof)
        y[idx] = A_int @ np.asarray(x)[idx]
        return y

    def apply_per_edge(self, x, S=None):
        """Alg. 3: for every interior edge, y_e = sum over its two elements of the
        edge's row block of S_K times the element's gathered trace values."""
        S = self.S() if S is None else S
        p1 = self.n1
        y = np.zeros(self.ndof)
        x = np.asarray(x)
        xb = x.copy()
        xb[np.setdiff1d(np.arange(self.ndof), self.interior_dofs())] = 0.0
        for ed in range(self.mesh.n_edges):
            E1, E2 = self.edge_elem[ed]
            if E1 < 0 or E2 < 0:
                continue
            acc = np.zeros(p1)
            for K, f in ((E1, self.edge_face[ed, 0]), (E2, self.edge_face[ed, 1])):
                rows = S[K][f * p1:(f + 1) * p1, :]
                acc += rows @ xb[self.dofs(K)]
            y[ed * p1:(ed + 1) * p1] = acc
        return y

    def load_vectors(self, f_q):
        f_q = np.asarray(f_q).reshape(self.mesh.nel, -1)
        return np.array([load_vector(self.ref, self.mats(e), f_q[e]) for e in range(self.mesh.nel)])

    def condense_rhs(self, f_q):
        """b = sum_K A_K^T b_K on all dofs, boundary entries 0 (step (ii), RHS)."""
        F = self.load_vectors(f_q)
        b = np.zeros(self.ndof)
        for e in range(self.mesh.nel):
            b[self.dofs(e)] += rhs_block(self.mats(e), F[e])
        b[np.setdiff1d(np.arange(self.ndof), self.interior_dofs())] = 0.0
        return b

    def solve_direct(self, b):
        """Step (iii) with a sparse direct solver (SuperLU)."""
        A_int, idx = self.assemble_interior()
        lam = np.zeros(self.ndof)
        lam[idx] = spla.splu(A_int.tocsc()).solve(b[idx])
        return lam

    def recover(self, lam, f_q):
        """Step (iv), Eq. shur0. Returns u [nel, (p+1)^2] and q [nel, 2, (p+1)^2] as
        values at the GLL tensor nodes (the nodal coefficients)."""
        F = self.load_vectors(f_q)
        n = self.ref.n
        u = np.zeros((self.mesh.nel, n))
        q = np.zeros((self.mesh.nel, 2, n))
        for e in range(self.mesh.nel):
            Q, U = local_solve(self.mats(e), lam[self.dofs(e)], F[e])
            u[e] = U
            q[e, 0], q[e, 1] = Q[:n], Q[n:]
        return u, q


def uncondensed_solve(mesh, p, kappa, f_q, tau=1.0):
    """The full (Q, U, Lambda) HDG system of Eqs. eq_h1-eq_h3 (interior Lambda only),
    assembled and solved directly; for tiny meshes. Returns (lam, u, q) with lam
    on all trace dofs (0 on the boundary)."""
    prob = HDGProblem(mesh, p, kappa, tau)
    n, m, p1 = prob.ref.n, prob.m, prob.n1
    nel = mesh.nel
    idx = prob.interior_dofs()
    gmap = -np.ones(prob.ndof, dtype=np.int64)
    gmap[idx] = np.arange(len(idx))
    nvol = 3 * n * nel
    N = nvol + len(idx)
    K = np.zeros((N, N))
    rhs = np.zeros(N)
    F = prob.load_vectors(f_q)
    for e in range(nel):
        mt = prob.mats(e)
        L = local_system(mt)
        CE = np.vstack([mt["C"], mt["E"]])
        off = 3 * n * e
        K[off:off + 3 * n, off:off + 3 * n] = L
        d = prob.dofs(e)
        for a, gd in enumerate(d):
            g = gmap[gd]
            if g < 0:
                continue
            K[off:off + 3 * n, nvol + g] += CE[:, a]
        rhs[off + 2 * n:off + 3 * n] = F[e]
        # eq_h3 rows: sum over elements of G Q + tau H U - tau Ml Lambda = 0
        GH = np.hstack([mt["G"], mt["tau"] * mt["H"]])
        for a, gd in enumerate(d):
            g = gmap[gd]
            if g < 0:
                continue
            K[nvol + g, off:off + 3 * n] += GH[a]
            for b_, gd2 in enumerate(d):
                g2 = gmap[gd2]
                if g2 < 0:
                    continue
                K[nvol + g, nvol + g2] -= mt["tau"] * mt["Ml"][a, b_]
    sol = np.linalg.solve(K, rhs)
    lam = np.zeros(prob.ndof)
    lam[idx] = sol[nvol:]
    u = np.zeros((nel, n))
    q = np.zeros((nel, 2, n))
    for e in range(nel):
        off = 3 * n * e
        q[e, 0] = sol[off:off + n]
        q[e, 1] = sol[off + n:off + 2 * n]
        u[e] = sol[off + 2 * n:off + 3 * n]
    return lam, u, q


def l2_errors(prob, u, q, u_exact, q_exact, nquad=None, components=False):
    """L2 norms of u_h - u and q_h - q by nquad-point GL quadrature per element
    (p+4 points by default; Table 1 of Sec. 5 is reproduced with p+1 points).
    With components=True returns (|u_h - u|, |q_h,x - q_x|, |q_h,y - q_y|)."""
    ref = prob.ref
    nq = ref.p + 4 if nquad is None else nquad
    xq, wq = qd.gauss_legendre(nq)
    B1 = qd.lagrange_matrix(ref.vnodes, xq)
    V = np.kron(B1, B1)
    wJ = np.kron(wq, wq) * prob.mesh.hx * prob.mesh.hy / 4.0
    eu = 0.0
    eqx = 0.0
    eqy = 0.0
    for e in range(prob.mesh.nel):
        ox, oy = prob.mesh.elem_origin(e)
        X, Y = np.meshgrid(ox + prob.mesh.hx * (xq + 1) / 2, oy + prob.mesh.hy * (xq + 1) / 2)
        X, Y = X.ravel(), Y.ravel()
        uh = V @ u[e]
        eu += np.sum(wJ * (uh - u_exact(X, Y)) ** 2)
        qx, qy = q_exact(X, Y)
        eqx += np.sum(wJ * (V @ q[e, 0] - qx) ** 2)
        eqy += np.sum(wJ * (V @ q[e, 1] - qy) ** 2)
    if components:
        return np.sqrt(eu), np.sqrt(eqx), np.sqrt(eqy)
    return np.sqrt(eu), np.sqrt(eqx + eqy)


def postprocess(prob, u, q):
    """Element-local postprocessing of Sec. 3 step (v) and Sec. 5 (the filter of
    the cited LDG-H analysis): on each element K find u* in Q_{p+1}(K) with
        (kappa grad u*, grad w)_K = -(q_h, grad w)_K   for all w in Q_{p+1}(K),
        (u*, 1)_K = (u_h, 1)_K,
    i.e. a local Neumann problem whose gradient matches -kappa^-1 q_h and whose
    mean is that of u_h. Integrals by the (p+3)-point GL rule (exact: the
    integrands have degree <= 2p+2 in each variable). Returns u* as values at
    the (p+2)^2 GLL tensor nodes of each element, [nel, (p+2)^2] (index
    i + (p+2) j), and the postprocessed flux q* = -kappa grad u* is obtained
    from it (see postprocessed_flux). Table 1's u* and q* columns are reproduced
    with these definitions."""
    p, m = prob.p, prob.mesh
    ref = prob.ref
    xs = qd.volume_nodes(p + 1)
    nq = p + 3
    xq, wq = qd.gauss_legendre(nq)
    Bs = qd.lagrange_matrix(xs, xq)
    Ds = qd.lagrange_derivative_matrix(xs, xq)
    Vs = np.kron(Bs, Bs)
    Dxs = np.kron(Bs, Ds) * (2.0 / m.hx)
    Dys = np.kron(Ds, Bs) * (2.0 / m.hy)
    Bh = qd.lagrange_matrix(ref.vnodes, xq)
    Vh = np.kron(Bh, Bh)
    wJ = np.kron(wq, wq) * m.hx * m.hy / 4.0
    stiff = Dxs.T @ (wJ[:, None] * Dxs) + Dys.T @ (wJ[:, None] * Dys)
    mean_row = wJ @ Vs
    ns = Vs.shape[1]
    us = np.zeros((m.nel, ns))
    for e in range(m.nel):
        kap = prob.kappa[e]
        # the Neumann matrix is singular (constants); the mean condition closes it
        # through a Lagrange multiplier
        L = np.zeros((ns + 1, ns + 1))
        L[:ns, :ns] = kap * stiff
        L[ns, :ns] = mean_row
        L[:ns, ns] = mean_row
        rhs = np.zeros(ns + 1)
        rhs[:ns] = -(Dxs.T @ (wJ * (Vh @ q[e, 0])) + Dys.T @ (wJ * (Vh @ q[e, 1])))
        rhs[ns] = wJ @ (Vh @ u[e])
        us[e] = np.linalg.solve(L, rhs)[:ns]
    return us


def postprocessed_errors(prob, ustar, u_exact, q_exact, nquad=None, components=False):
    """L2 errors of u* and q* = -kappa grad u* (per element, nodal at the
    (p+2)^2 GLL nodes) by nquad-point GL quadrature (p+2 by default, the rule
    with which Table 1's u* and q* columns are reproduced)."""
    p, m = prob.p, prob.mesh
    xs = qd.volume_nodes(p + 1)
    nq = p + 2 if nquad is None else nquad
    xq, wq = qd.gauss_legendre(nq)
    B = qd.lagrange_matrix(xs, xq)
    D = qd.lagrange_derivative_matrix(xs, xq)
    V = np.kron(B, B)
    Dx = np.kron(B, D) * (2.0 / m.hx)
    Dy = np.kron(D, B) * (2.0 / m.hy)
    wJ = np.kron(wq, wq) * m.hx * m.hy / 4.0
    eu = ex = ey = 0.0
    for e in range(m.nel):
        ox, oy = m.elem_origin(e)
        X, Y = np.meshgrid(ox + m.hx * (xq + 1) / 2, oy + m.hy * (xq + 1) / 2)
        X, Y = X.ravel(), Y.ravel()
        kap = prob.kappa[e]
        eu += np.sum(wJ * (V @ ustar[e] - u_exact(X, Y)) ** 2)
        qx, qy = q_exact(X, Y)
        ex += np.sum(wJ * (-kap * (Dx @ ustar[e]) - qx) ** 2)
        ey += np.sum(wJ * (-kap * (Dy @ ustar[e]) - qy) ** 2)
    if components:
        return np.sqrt(eu), np.sqrt(ex), np.sqrt(ey)
    return np.sqrt(eu), np.sqrt(ex + ey)
