"""Coarse Q1 levels fused into one launch (hdg_options.coarse_fuse, Alg. 1 on
the h-levels): the V-cycle whose coarse levels run as phases of one single-CTA
kernel equals the one-launch-per-step V-cycle up to the coarsest solve's
rounding (its inverse instead of the two substitutions), for one and many
right-hand sides, every vector type, hierarchies that end on an odd size or on
a coarsest mesh with many unknowns; it launches fewer kernels per V-cycle, and
a solve takes the same iterations to the same solution."""
import numpy as np
import pytest
import torch

from paper_1705_09907_gb300 import hdg, inputs

pytestmark = pytest.mark.gpu

# (nx, ny, k, options): power-of-two, ragged (48 x 40 ends at 6 x 5), coarsest
# 14 x 14 interior vertices (60 -> 30 -> 15), coarse_n = 8 (coarsest 7 x 7)
CASES = [(32, 32, 2, {}), (128, 128, 3, {}), (48, 40, 1, {}), (60, 60, 2, {}), (64, 64, 2, {"coarse_n": 8})]


def _pair(nx, ny, k, **kw):
    kap = torch.as_tensor(np.exp(inputs.gaussian_field(nx, seed=3, corr_len=0.2, ny=ny)), device="cuda")
    return hdg.HDGSolver(nx, ny, k, kap, **kw), hdg.HDGSolver(nx, ny, k, kap, coarse_fuse=0, **kw)


def _rhs(s, nrhs, seed):
    rng = np.random.default_rng(seed)
    shape = (s.ndof,) if nrhs == 1 else (s.ndof, nrhs)
    return torch.as_tensor(rng.normal(size=shape), device="cuda")


@pytest.mark.parametrize("nx,ny,k,opts", CASES)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("f32x2", 1e-12), ("fp32", 2e-5), ("bf16", 2e-5)])
def test_fused_vcycle_equals_unfused(nx, ny, k, opts, prec, tol):
    a, b = _pair(nx, ny, k, **opts)
    for nrhs in (1, 8):
        r = _rhs(a, nrhs, 40 + nrhs)
        r = r.to(hdg.VEC_DTYPE[prec])
        za = a.vcycle(r, prec=prec)
        zb = b.vcycle(r, prec=prec)
        assert torch.isfinite(za).all()
        err = (torch.linalg.norm((za - zb).double()) / torch.linalg.norm(zb.double())).item()
        assert err <= tol, (nrhs, err)
        # graph replay reproduces the fused cycle
        assert torch.equal(a.vcycle(r, prec=prec), za)
    a.close()
    b.close()


@pytest.mark.parametrize("prec,saved", [("fp32", 44), ("fp64", 33)])
def test_fused_cycle_launches_fewer_kernels(prec, saved):
    a, b = _pair(128, 128, 2)
    r = _rhs(a, 1, 7).to(hdg.VEC_DTYPE[prec])
    a.vcycle(r, prec=prec)
    b.vcycle(r, prec=prec)
    ka, kb = a.get_info()["vcycle_kernels"], b.get_info()["vcycle_kernels"]
    # 128^2: Q1 levels 128, 64, ..., 2 with 11 launches per smoothed level and
    # one coarsest solve; float cycles fuse levels 32 and below (961 vertices:
    # 80 KB of stencils and vectors), double cycles levels 16 and below (at
    # most 512 entries per level)
    assert ka == kb - saved, (ka, kb)
    a.close()
    b.close()


@pytest.mark.parametrize("inner", ["fp64", "fp32"])
def test_fused_solve_matches_unfused(inner):
    nx = ny = 128
    k = 3
    a, b = _pair(nx, ny, k)
    fq = torch.as_tensor(inputs.constant_f(nx, k), device="cuda")
    rhs = a.condense_rhs(fq)
    la, ia = a.solve(rhs, rtol=1e-10, inner=inner)
    lb, ib = b.solve(rhs, rtol=1e-10, inner=inner)
    assert abs(ia["iterations"] - ib["iterations"]) <= 1
    assert ia["relres"] <= 1e-10
    assert (torch.linalg.norm(la - lb) / torch.linalg.norm(lb)).item() <= 1e-9
    a.close()
    b.close()
