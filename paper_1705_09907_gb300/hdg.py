"""ctypes binding of libhdg.so (include/hdg.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels; PyTorch supplies
device memory and the current CUDA stream. The functions named like the C ABI
(hdg_setup, hdg_apply_trace, ...) take raw device pointers; the HDGSolver class
wraps them for torch tensors. Importing this module fails loudly if the library
has not been built (there is no CPU fallback).
"""
import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhdg.so")

HDG_OK = 0
HDG_ERR_INVALID_ARG = 1
HDG_ERR_CUDA = 2
HDG_ERR_OOM = 3
HDG_ERR_NOT_CONVERGED = 4
HDG_ERR_BREAKDOWN = 5
HDG_ERR_TIMEOUT = 6
HDG_ERR_UNSUPPORTED = 7

PREC = {"fp64": 0, "fp32": 1, "bf16": 2, "f32x2": 3}
VEC_DTYPE = {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.float32, "f32x2": torch.float64}


class hdg_mesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("x1", ctypes.c_double), ("y1", ctypes.c_double)]


class hdg_options(ctypes.Structure):
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("coarse_n", ctypes.c_int), ("tau", ctypes.c_double),
                ("cheb_degree", ctypes.c_int), ("mixed", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("autotune", ctypes.c_int), ("reduced", ctypes.c_int),
                ("tau_kappa", ctypes.c_int), ("smoother", ctypes.c_int), ("tensor_apply", ctypes.c_int),
                ("fmg_start", ctypes.c_int),
                ("max_device_bytes", ctypes.c_size_t),
                ("wait_probe", ctypes.c_int),
                ("coarse_fuse", ctypes.c_int),
                ("top_accum", ctypes.c_int)]


class hdg_info(ctypes.Structure):
    _fields_ = [("nel", ctypes.c_int), ("n_edges", ctypes.c_int), ("ndof", ctypes.c_int), ("k", ctypes.c_int),
                ("n_plevels", ctypes.c_int), ("n_hlevels", ctypes.c_int), ("coarse_dim", ctypes.c_int),
                ("device_bytes", ctypes.c_size_t), ("setup_ms", ctypes.c_double), ("vcycle_kernels", ctypes.c_int),
                ("apply_kernels", ctypes.c_int)]


class hdg_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("relres", ctypes.c_double),
                ("relres_history", ctypes.c_double * 256), ("solve_ms", ctypes.c_double)]


class HDGError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s failed: %s (status %d)" % (where, error_string(status), status))


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libhdg.so is not built; run paper_1705_09907_gb300.build.build() first (%s)" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "hdg_default_options": (None, [ctypes.POINTER(hdg_options)]),
        "hdg_error_string": (ctypes.c_char_p, [i]),
        "hdg_setup": (i, [ctypes.POINTER(hdg_mesh), i, vp, ctypes.POINTER(hdg_options), vp, ctypes.POINTER(vp)]),
        "hdg_get_info": (i, [vp, ctypes.POINTER(hdg_info)]),
        "hdg_get_maps": (i, [vp, vp, vp, vp, vp]),
        "hdg_condense_rhs": (i, [vp, vp, vp, i, vp]),
        "hdg_apply_trace": (i, [vp, vp, vp, i, i, vp]),
        "hdg_gmg_vcycle": (i, [vp, vp, vp, i, i, vp]),
        "hdg_solve": (i, [vp, vp, vp, i, d, i, i, ctypes.POINTER(hdg_solve_info), vp]),
        "hdg_recover_local": (i, [vp, vp, vp, vp, vp, vp]),
        "hdg_postprocess": (i, [vp, vp, vp, vp, vp, vp]),
        "hdg_fmg": (i, [vp, vp, vp, i, vp]),
        "hdg_adjoint_grad": (i, [vp, vp, vp, vp, d, i, vp, vp, vp, vp, vp]),
        "hdg_condense_rhs_noalloc": (i, [vp, vp, vp, i, vp]),
        "hdg_apply_shared_batched": (i, [vp, vp, vp, i, vp]),
        "hdg_apply_shared_fp64": (i, [vp, vp, vp, i, vp]),
        "hdg_apply_multi": (i, [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), i, vp]),
        "hdg_setup_batch": (i, [i, ctypes.POINTER(hdg_mesh), ctypes.POINTER(i), ctypes.POINTER(vp),
                                ctypes.POINTER(hdg_options), vp, ctypes.POINTER(vp)]),
        "hdg_solve_multi": (i, [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), d, i, i,
                                ctypes.POINTER(hdg_solve_info), ctypes.POINTER(i), vp]),
        "hdg_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()

# C ABI names, re-exported
hdg_default_options = _lib.hdg_default_options
hdg_error_string = _lib.hdg_error_string
hdg_setup = _lib.hdg_setup
hdg_get_info = _lib.hdg_get_info
hdg_get_maps = _lib.hdg_get_maps
hdg_condense_rhs = _lib.hdg_condense_rhs
hdg_apply_trace = _lib.hdg_apply_trace
hdg_gmg_vcycle = _lib.hdg_gmg_vcycle
hdg_solve = _lib.hdg_solve
hdg_recover_local = _lib.hdg_recover_local
hdg_postprocess = _lib.hdg_postprocess
hdg_fmg = _lib.hdg_fmg
hdg_adjoint_grad = _lib.hdg_adjoint_grad
hdg_condense_rhs_noalloc = _lib.hdg_condense_rhs_noalloc
hdg_apply_shared_batched = _lib.hdg_apply_shared_batched
hdg_apply_shared_fp64 = _lib.hdg_apply_shared_fp64
hdg_apply_multi = _lib.hdg_apply_multi
hdg_setup_batch = _lib.hdg_setup_batch
hdg_solve_multi = _lib.hdg_solve_multi


def setup_batch(problems, **options):
    """Set up several uneven problems in one call (hdg_setup_batch).
    problems: list of (nx, ny, k, kappa) with kappa a CUDA tensor of nx*ny
    entries (unit square meshes). Returns one HDGSolver per problem."""
    n = len(problems)
    meshes = (hdg_mesh * n)(*[hdg_mesh(int(nx), int(ny), 0.0, 0.0, 1.0, 1.0) for nx, ny, _, _ in problems])
    ks = (ctypes.c_int * n)(*[int(k) for _, _, k, _ in problems])
    kaps = [kap.to(device="cuda", dtype=torch.float64).contiguous() for _, _, _, kap in problems]
    kp = (ctypes.c_void_p * n)(*[_ptr(kap, torch.float64).value for kap in kaps])
    out = (ctypes.c_void_p * n)()
    opt = default_options(**options)
    _check(_lib.hdg_setup_batch(n, meshes, ks, kp, ctypes.byref(opt), _stream(), out), "hdg_setup_batch")
    return [HDGSolver._adopt(ctypes.c_void_p(out[q]), problems[q][0], problems[q][1], problems[q][2], meshes[q], opt)
            for q in range(n)]


def apply_multi(solvers, xs, prec="fp64", outs=None):
    """One launch of y_q = A_q x_q over several HDGSolver instances."""
    n = len(solvers)
    ys = [torch.empty_like(x) for x in xs] if outs is None else outs
    arr = ctypes.c_void_p * n
    ctxs = arr(*[s.ctx.value for s in solvers])
    xp = arr(*[_ptr(x, VEC_DTYPE[prec]).value for x in xs])
    yp = arr(*[_ptr(y, VEC_DTYPE[prec]).value for y in ys])
    _check(_lib.hdg_apply_multi(n, ctxs, xp, yp, PREC[prec], _stream()), "hdg_apply_multi")
    return ys


def solve_multi(solvers, bs, rtol=1e-10, maxit=200, inner="fp64", outs=None, raise_on_error=True):
    """hdg_solve_multi: every HDGSolver's system at once (each on its own stream).
    Returns the solutions and one info dict per instance."""
    n = len(solvers)
    lams = [torch.empty_like(b) for b in bs] if outs is None else outs
    arr = ctypes.c_void_p * n
    ctxs = arr(*[s.ctx.value for s in solvers])
    bp = arr(*[_ptr(b, torch.float64).value for b in bs])
    lp = arr(*[_ptr(x, torch.float64).value for x in lams])
    infos = (hdg_solve_info * n)()
    sts = (ctypes.c_int * n)()
    st = _lib.hdg_solve_multi(n, ctxs, bp, lp, float(rtol), int(maxit), PREC[inner], infos, sts, _stream())
    out = [{"status": sts[q], "iterations": infos[q].iterations, "relres": infos[q].relres,
            "solve_ms": infos[q].solve_ms} for q in range(n)]
    if raise_on_error:
        _check(st, "hdg_solve_multi")
    return lams, out


hdg_destroy = _lib.hdg_destroy


def library():
    return _lib


def error_string(status):
    return _lib.hdg_error_string(int(status)).decode()


def _check(status, where):
    if status != HDG_OK:
        raise HDGError(status, where)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype=None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError("expected dtype %s, got %s" % (dtype, t.dtype))
    return ctypes.c_void_p(t.data_ptr())


def default_options(**kw):
    o = hdg_options()
    _lib.hdg_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class HDGSolver:
    """Owns one hdg context: mesh nx x ny on [x0,x1]x[y0,y1], degree k,
    per-element kappa (a float64 CUDA tensor of nx*ny entries)."""

    def __init__(self, nx, ny, k, kappa, x0=0.0, y0=0.0, x1=1.0, y1=1.0, **options):
        self.nx, self.ny, self.k = int(nx), int(ny), int(k)
        self.mesh = hdg_mesh(self.nx, self.ny, x0, y0, x1, y1)
        self.opt = default_options(**options)
        kappa = kappa.to(device="cuda", dtype=torch.float64).contiguous()
        ctx = ctypes.c_void_p()
        st = _lib.hdg_setup(ctypes.byref(self.mesh), self.k, _ptr(kappa, torch.float64), ctypes.byref(self.opt),
                            _stream(), ctypes.byref(ctx))
        _check(st, "hdg_setup")
        self.ctx = ctx
        inf = hdg_info()
        _check(_lib.hdg_get_info(self.ctx, ctypes.byref(inf)), "hdg_get_info")
        self.info = {f: getattr(inf, f) for f, _ in hdg_info._fields_}
        self.nel, self.n_edges, self.ndof = inf.nel, inf.n_edges, inf.ndof

    @classmethod
    def _adopt(cls, ctx, nx, ny, k, mesh, opt):
        """Wrap a context created by hdg_setup_batch."""
        self = cls.__new__(cls)
        self.nx, self.ny, self.k = int(nx), int(ny), int(k)
        self.mesh, self.opt, self.ctx = mesh, opt, ctx
        inf = hdg_info()
        _check(_lib.hdg_get_info(self.ctx, ctypes.byref(inf)), "hdg_get_info")
        self.info = {f: getattr(inf, f) for f, _ in hdg_info._fields_}
        self.nel, self.n_edges, self.ndof = inf.nel, inf.n_edges, inf.ndof
        return self

    def get_info(self):
        inf = hdg_info()
        _check(_lib.hdg_get_info(self.ctx, ctypes.byref(inf)), "hdg_get_info")
        return {f: getattr(inf, f) for f, _ in hdg_info._fields_}

    def close(self):
        if getattr(self, "ctx", None):
            _lib.hdg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def maps(self):
        e2e = torch.empty((self.nel, 4), dtype=torch.int32, device="cuda")
        el = torch.empty((self.n_edges, 2), dtype=torch.int32, device="cuda")
        fc = torch.empty((self.n_edges, 2), dtype=torch.int32, device="cuda")
        _check(_lib.hdg_get_maps(self.ctx, _ptr(e2e), _ptr(el), _ptr(fc), _stream()), "hdg_get_maps")
        return e2e, el, fc

    def condense_rhs(self, f_q):
        f_q = f_q.to(device="cuda", dtype=torch.float64).contiguous()
        nrhs = 1 if f_q.dim() == 3 else f_q.shape[0]
        b = torch.empty((self.ndof,) if nrhs == 1 else (self.ndof, nrhs), dtype=torch.float64, device="cuda")
        _check(_lib.hdg_condense_rhs(self.ctx, _ptr(f_q), _ptr(b), nrhs, _stream()), "hdg_condense_rhs")
        return b

    def apply(self, x, prec="fp64", out=None):
        nrhs = 1 if x.dim() == 1 else x.shape[1]
        y = torch.empty_like(x) if out is None else out
        _check(_lib.hdg_apply_trace(self.ctx, _ptr(x, VEC_DTYPE[prec]), _ptr(y, VEC_DTYPE[prec]), nrhs, PREC[prec],
                                    _stream()), "hdg_apply_trace")
        return y

    def apply_shared_batched(self, X, out=None):
        """Y = A X for a uniform coefficient on the tensor cores: X BF16 [ndof, nrhs]
        (nrhs a multiple of 64), Y FP32 [ndof, nrhs]."""
        if X.dtype != torch.bfloat16 or X.dim() != 2:
            raise ValueError("X must be a 2-D bfloat16 CUDA tensor [ndof, nrhs]")
        Y = torch.empty(X.shape, dtype=torch.float32, device="cuda") if out is None else out
        _check(_lib.hdg_apply_shared_batched(self.ctx, _ptr(X), _ptr(Y, torch.float32), X.shape[1], _stream()),
               "hdg_apply_shared_batched")
        return Y

    def apply_shared_fp64(self, X, out=None):
        """Y = A X in FP64 for a uniform coefficient on the tensor cores (exact
        slice splitting): X, Y float64 [ndof, nrhs], nrhs a multiple of 64."""
        if X.dtype != torch.float64 or X.dim() != 2:
            raise ValueError("X must be a 2-D float64 CUDA tensor [ndof, nrhs]")
        Y = torch.empty_like(X) if out is None else out
        _check(_lib.hdg_apply_shared_fp64(self.ctx, _ptr(X), _ptr(Y, torch.float64), X.shape[1], _stream()),
               "hdg_apply_shared_fp64")
        return Y

    def vcycle(self, r, prec="fp64", out=None):
        nrhs = 1 if r.dim() == 1 else r.shape[1]
        z = torch.empty_like(r) if out is None else out
        _check(_lib.hdg_gmg_vcycle(self.ctx, _ptr(r, VEC_DTYPE[prec]), _ptr(z, VEC_DTYPE[prec]), nrhs, PREC[prec],
                                   _stream()), "hdg_gmg_vcycle")
        return z

    def solve(self, b, rtol=1e-10, maxit=200, inner="fp64", out=None, raise_on_error=True):
        """b: [ndof] or [ndof, nrhs] (right-hand side fastest); for nrhs > 1 all
        columns iterate together and `iterations` / `relres` are the largest
        over the columns."""
        nrhs = 1 if b.dim() == 1 else b.shape[1]
        lam = torch.empty_like(b) if out is None else out
        inf = hdg_solve_info()
        st = _lib.hdg_solve(self.ctx, _ptr(b, torch.float64), _ptr(lam, torch.float64), nrhs, float(rtol),
                            int(maxit), PREC[inner], ctypes.byref(inf), _stream())
        info = {"status": st, "iterations": inf.iterations, "relres": inf.relres, "solve_ms": inf.solve_ms,
                "history": list(inf.relres_history[: min(inf.iterations, 255) + 1])}
        if raise_on_error:
            _check(st, "hdg_solve")
        return lam, info

    def recover(self, lam, f_q):
        n = (self.k + 1) ** 2
        u = torch.empty((self.nel, n), dtype=torch.float64, device="cuda")
        q = torch.empty((self.nel, 2, n), dtype=torch.float64, device="cuda")
        f_q = f_q.to(device="cuda", dtype=torch.float64).contiguous()
        _check(_lib.hdg_recover_local(self.ctx, _ptr(lam, torch.float64), _ptr(f_q), _ptr(u), _ptr(q), _stream()),
               "hdg_recover_local")
        return u, q

    def fmg(self, b, cycles=1, out=None):
        """One full multigrid cycle (Sec. 7) with `cycles` V-cycles per level."""
        lam = torch.empty_like(b) if out is None else out
        _check(_lib.hdg_fmg(self.ctx, _ptr(b, torch.float64), _ptr(lam, torch.float64), int(cycles), _stream()),
               "hdg_fmg")
        return lam

    def postprocess(self, u, q, flux=True):
        """u*, and q* = -kappa grad u* if flux, from the recovered (u, q): values at
        the (k+2)^2 Gauss-Lobatto nodes of each element."""
        ns = (self.k + 2) ** 2
        us = torch.empty((self.nel, ns), dtype=torch.float64, device="cuda")
        qs = torch.empty((self.nel, 2, ns), dtype=torch.float64, device="cuda") if flux else None
        _check(_lib.hdg_postprocess(self.ctx, _ptr(u, torch.float64), _ptr(q, torch.float64), _ptr(us),
                                    _ptr(qs), _stream()), "hdg_postprocess")
        return (us, qs) if flux else us

    def adjoint_grad(self, f_q, lam, lam_obs, rtol=1e-12, maxit=200):
        f_q = f_q.to(device="cuda", dtype=torch.float64).contiguous()
        dth = torch.empty(self.nel, dtype=torch.float64, device="cuda")
        df = torch.empty((self.nel, self.k + 2, self.k + 2), dtype=torch.float64, device="cuda")
        J = torch.empty(1, dtype=torch.float64, device="cuda")
        psi = torch.empty(self.ndof, dtype=torch.float64, device="cuda")
        _check(_lib.hdg_adjoint_grad(self.ctx, _ptr(f_q), _ptr(lam, torch.float64), _ptr(lam_obs, torch.float64),
                                     float(rtol), int(maxit), _ptr(dth), _ptr(df), _ptr(J), _ptr(psi), _stream()),
               "hdg_adjoint_grad")
        return J, dth, df, psi
