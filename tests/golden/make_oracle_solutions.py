"""Writes the oracle's trace solutions used as expected values by the mixed-
precision checks (tests/test_gpu_mixed_vs_oracle.py and the benchmark's
err_vs_oracle keys). Calls only the FP64 CPU oracle (condensed right-hand
side, assembly of sum_K A_K^T S_K A_K, SuperLU) on the seeded lognormal
workload: kappa = exp(g), g the Gaussian field of correlation length 0.05 and
variance 1 on the element centres (seed 0), f = 1, N x N unit square, degree k.

Run from the repository root:  python tests/golden/make_oracle_solutions.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import hdg, mesh  # noqa: E402
from paper_1705_09907_gb300 import inputs  # noqa: E402

CASES = [(128, 4), (128, 3)]


def path(N, k):
    return os.path.join(HERE, "oracle_lognormal_%d_k%d.npy" % (N, k))


def main():
    for N, k in CASES:
        prob = hdg.HDGProblem(mesh.Mesh(N, N), k, inputs.lognormal_kappa(N, 0))
        lam = prob.solve_direct(prob.condense_rhs(inputs.constant_f(N, k)))
        np.save(path(N, k), lam)
        print("wrote", path(N, k), lam.shape)


if __name__ == "__main__":
    main()
