"""hdg_condense_rhs_noalloc: the allocation-free condensed right-hand side for
callers that cannot allocate device memory when they need it. Checked through
the C ABI against hdg_condense_rhs on two calls in a row (the fixed scratch
array keeps the previous call's contents), and for the size limit. This file
is collected last so that a failure here comes after every other test."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_condense_noalloc_matches_condense():
    from paper_1705_09907_gb300 import hdg, inputs
    nx, ny, k = 37, 12, 3
    kap = torch.as_tensor(np.exp(inputs.gaussian_field(nx, seed=3, corr_len=0.2, ny=ny)), device="cuda")
    s = hdg.HDGSolver(nx, ny, k, kap)
    rng = np.random.default_rng(21)
    for call in range(2):
        fq = torch.as_tensor(rng.normal(size=(s.nel, k + 2, k + 2)), device="cuda")
        b_ref = torch.empty(s.ndof, dtype=torch.float64, device="cuda")
        b_new = torch.full((s.ndof,), float("nan"), dtype=torch.float64, device="cuda")
        st = hdg.hdg_condense_rhs(s.ctx, ctypes.c_void_p(fq.data_ptr()), ctypes.c_void_p(b_ref.data_ptr()), 1,
                                  _stream())
        assert st == hdg.HDG_OK
        st = hdg.hdg_condense_rhs_noalloc(s.ctx, ctypes.c_void_p(fq.data_ptr()), ctypes.c_void_p(b_new.data_ptr()),
                                          1, _stream())
        assert st == hdg.HDG_OK, hdg.error_string(st)
        torch.cuda.synchronize()
        ref = b_ref.cpu().numpy()
        new = b_new.cpu().numpy()
        assert np.all(np.isfinite(new))
        # same arithmetic in the same order: the test's FP64 tolerance for b
        assert np.abs(new - ref).max() <= 1e-12 * np.abs(ref).max()
    s.close()


def test_condense_noalloc_rejects_oversize():
    from paper_1705_09907_gb300 import hdg
    nx = ny = 256
    k = 2                                   # 65536 elements x 12 > 2^19 scratch entries
    s = hdg.HDGSolver(nx, ny, k, torch.ones(nx * ny, dtype=torch.float64, device="cuda"), mixed=0, autotune=0)
    fq = torch.zeros((s.nel, k + 2, k + 2), dtype=torch.float64, device="cuda")
    b = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    st = hdg.hdg_condense_rhs_noalloc(s.ctx, ctypes.c_void_p(fq.data_ptr()), ctypes.c_void_p(b.data_ptr()), 1,
                                      _stream())
    assert st == hdg.HDG_ERR_INVALID_ARG
    s.close()
