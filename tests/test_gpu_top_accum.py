"""Float V-cycles with the finest level's correction kept as a double-float pair
(hdg_options.top_accum = 1, the default): every operator of the cycle stays in
FP32 / BF16, only the sum of the prolongated coarse correction and the
smoothing increments is wider. The preconditioned CG then takes the iterations
of the FP64 cycle (the float-rounded sum costs ~40% more on the 512^2 mesh),
for one and for many right-hand sides, and reaches the same solution."""
import numpy as np
import pytest
import torch

from paper_1705_09907_gb300 import hdg, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("inner", ["fp32", "bf16"])
def test_float_cycle_iterations_match_fp64_at_512(inner):
    N, k = 512, 4
    kap = torch.as_tensor(inputs.lognormal_kappa(N, 0), device="cuda")
    fq = torch.as_tensor(inputs.constant_f(N, k), device="cuda")
    s = hdg.HDGSolver(N, N, k, kap)
    b = s.condense_rhs(fq)
    l64, i64 = s.solve(b, rtol=1e-10)
    lf, iff = s.solve(b, rtol=1e-10, inner=inner)
    assert iff["iterations"] <= i64["iterations"] + 1, (iff["iterations"], i64["iterations"])
    assert (torch.linalg.norm(lf - l64) / torch.linalg.norm(l64)).item() < 1e-9
    s.close()
    s0 = hdg.HDGSolver(N, N, k, kap, top_accum=0)
    _, i0 = s0.solve(s0.condense_rhs(fq), rtol=1e-10, inner=inner)
    assert i0["iterations"] >= iff["iterations"] + 5, (i0["iterations"], iff["iterations"])
    s0.close()


@pytest.mark.parametrize("k", [1, 3])
def test_batched_float_cycle_with_wide_top_sum(k):
    N, nb = 128, 8
    kap = torch.as_tensor(np.exp(inputs.gaussian_field(N, seed=6, corr_len=0.1)), device="cuda")
    s = hdg.HDGSolver(N, N, k, kap)
    B = s.condense_rhs(torch.as_tensor(inputs.fourier_rhs(N, k, nb, seed=4), device="cuda"))
    L64, i64 = s.solve(B, rtol=1e-10)
    L32, i32 = s.solve(B, rtol=1e-10, inner="fp32")
    assert i32["iterations"] <= i64["iterations"] + 1
    for j in (0, nb - 1):
        assert (torch.linalg.norm(L32[:, j] - L64[:, j]) / torch.linalg.norm(L64[:, j])).item() < 1e-9
    # every column equals its own single solve's accuracy
    l0, _ = s.solve(B[:, 0].contiguous(), rtol=1e-10, inner="fp32")
    assert (torch.linalg.norm(l0 - L64[:, 0]) / torch.linalg.norm(L64[:, 0])).item() < 1e-9
    s.close()
