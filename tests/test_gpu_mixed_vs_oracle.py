"""Every V-cycle precision's solution against the FP64 oracle's direct solution
on the seeded lognormal workload (kappa = exp(g), correlation length 0.05,
seed 0, f = 1) at 128 x 128, k = 4 and k = 3: the stored SuperLU solutions of
tests/golden/ (written by the oracle alone). The outer CG runs on FP64 vectors
with an FP64 (or double-float, ~48-bit) operator in every mode, so at rtol
1e-12 the remaining difference is that of two independent FP64 computations of
the element blocks and the right-hand side: rounding of order eps in their
entries moves the solution by up to cond(A) eps, and cond(A) = 7.3e5 here
(128 x 128, k = 4; Lanczos extremes of the oracle's matrix), so the bound is
20 cond(A) eps = 1.6e-9 (measured: 4.7e-10 in FP64). The oracle's own CG and
its SuperLU solution agree to 2e-13, so the difference is not the stopping
test's."""
import os

import numpy as np
import pytest
import torch

from paper_1705_09907_gb300 import inputs

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("k", [4, 3])
@pytest.mark.parametrize("inner", ["fp64", "fp32", "bf16", "f32x2"])
def test_solution_vs_oracle(k, inner):
    from paper_1705_09907_gb300 import hdg
    N = 128
    ref = np.load(os.path.join(HERE, "golden", "oracle_lognormal_%d_k%d.npy" % (N, k)))
    s = hdg.HDGSolver(N, N, k, torch.as_tensor(inputs.lognormal_kappa(N, 0), device="cuda"))
    b = s.condense_rhs(torch.as_tensor(inputs.constant_f(N, k), device="cuda"))
    lam, info = s.solve(b, rtol=1e-12, maxit=400, inner=inner)
    err = np.linalg.norm(lam.cpu().numpy() - ref) / np.linalg.norm(ref)
    s.close()
    assert err < 1.6e-9, (inner, err, info["iterations"])
