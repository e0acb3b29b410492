"""hdg_condense_rhs_noalloc: the allocation-free condensed right-hand side for
callers that cannot allocate device memory when they need it (code running
where an allocation would synchronise the device or is not permitted).

Checked through the C ABI against hdg_condense_rhs on two calls in a row (the
fixed scratch array keeps the previous call's contents), with one and with
several right-hand sides (the scratch is reused column by column), against the
oracle's condensed right-hand side, for unchanged free device memory across
calls, for the device check and for the size limit. This file is collected
last so that a failure here comes after every other test."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("nrhs", [1, 3])
def test_condense_noalloc_matches_condense(nrhs):
    from paper_1705_09907_gb300 import hdg, inputs
    nx, ny, k = 37, 12, 3
    kap = torch.as_tensor(np.exp(inputs.gaussian_field(nx, seed=3, corr_len=0.2, ny=ny)), device="cuda")
    s = hdg.HDGSolver(nx, ny, k, kap)
    rng = np.random.default_rng(21 + nrhs)
    for call in range(2):
        fq = torch.as_tensor(rng.normal(size=(nrhs, s.nel, k + 2, k + 2)), device="cuda")
        b_ref = torch.empty(s.ndof * nrhs, dtype=torch.float64, device="cuda")
        b_new = torch.full((s.ndof * nrhs,), float("nan"), dtype=torch.float64, device="cuda")
        st = hdg.hdg_condense_rhs(s.ctx, _vp(fq), _vp(b_ref), nrhs, _stream())
        assert st == hdg.HDG_OK
        st = hdg.hdg_condense_rhs_noalloc(s.ctx, _vp(fq), _vp(b_new), nrhs, _stream())
        assert st == hdg.HDG_OK, hdg.error_string(st)
        torch.cuda.synchronize()
        ref = b_ref.cpu().numpy()
        new = b_new.cpu().numpy()
        assert np.all(np.isfinite(new))
        # same arithmetic in the same order: the test's FP64 tolerance for b
        assert np.abs(new - ref).max() <= 1e-12 * np.abs(ref).max()
    s.close()


def test_condense_noalloc_matches_oracle():
    from oracle import hdg as ohdg, mesh as omesh
    from paper_1705_09907_gb300 import hdg, inputs
    nx, ny, k = 9, 6, 2
    kap = np.exp(inputs.gaussian_field(nx, seed=5, corr_len=0.3, ny=ny))
    s = hdg.HDGSolver(nx, ny, k, torch.as_tensor(kap, device="cuda"))
    rng = np.random.default_rng(8)
    fq = rng.normal(size=(s.nel, k + 2, k + 2))
    prob = ohdg.HDGProblem(omesh.Mesh(nx, ny), k, kap)
    expect = prob.condense_rhs(fq)
    fq_d = torch.as_tensor(fq, device="cuda")
    for call in range(2):
        b = torch.full((s.ndof,), float("nan"), dtype=torch.float64, device="cuda")
        assert hdg.hdg_condense_rhs_noalloc(s.ctx, _vp(fq_d), _vp(b), 1, _stream()) == hdg.HDG_OK
        torch.cuda.synchronize()
        got = b.cpu().numpy()
        assert np.abs(got - expect).max() <= 1e-12 * np.abs(expect).max()
    s.close()


def test_condense_noalloc_leaves_free_memory_unchanged():
    """Free device memory is the same before and after two calls: the calls
    commit no device memory (the scratch array was loaded at set-up)."""
    from paper_1705_09907_gb300 import hdg
    nx, ny, k = 64, 48, 4
    s = hdg.HDGSolver(nx, ny, k, torch.ones(nx * ny, dtype=torch.float64, device="cuda"), mixed=0)
    fq = torch.ones((s.nel, k + 2, k + 2), dtype=torch.float64, device="cuda")
    b = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for call in range(2):
        assert hdg.hdg_condense_rhs_noalloc(s.ctx, _vp(fq), _vp(b), 1, _stream()) == hdg.HDG_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    s.close()


def test_condense_noalloc_rejects_oversize():
    from paper_1705_09907_gb300 import hdg
    nx = ny = 256
    k = 2                                   # 65536 elements x 12 > 2^19 scratch entries
    s = hdg.HDGSolver(nx, ny, k, torch.ones(nx * ny, dtype=torch.float64, device="cuda"), mixed=0, autotune=0)
    fq = torch.zeros((s.nel, k + 2, k + 2), dtype=torch.float64, device="cuda")
    b = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    st = hdg.hdg_condense_rhs_noalloc(s.ctx, _vp(fq), _vp(b), 1, _stream())
    assert st == hdg.HDG_ERR_INVALID_ARG
    s.close()
