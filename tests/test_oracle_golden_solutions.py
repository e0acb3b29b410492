"""The stored oracle solutions (tests/golden/oracle_lognormal_*.npy, written by
tests/golden/make_oracle_solutions.py from the oracle alone) satisfy sampled
rows of the oracle's condensed system A lambda = b: each sampled interior
edge's rows, sum over its two elements of S_K[edge rows] lambda_K - b_e, built
here from the element blocks of those elements only."""
import os

import numpy as np
import pytest

from oracle import hdg, mesh as omesh
from paper_1705_09907_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("N,k", [(128, 4), (128, 3)])
def test_stored_solution_satisfies_sampled_rows(N, k):
    lam = np.load(os.path.join(HERE, "golden", "oracle_lognormal_%d_k%d.npy" % (N, k)))
    m = omesh.Mesh(N, N)
    prob = hdg.HDGProblem(m, k, inputs.lognormal_kappa(N, 0))
    assert lam.shape == (prob.ndof,)
    fq = inputs.constant_f(N, k)
    rng = np.random.default_rng(7)
    inner = m.interior_edges()
    p1 = k + 1
    worst = 0.0
    for ed in rng.choice(inner, size=40, replace=False):
        res = np.zeros(p1)
        scale = np.zeros(p1)
        for K, f in zip(prob.edge_elem[ed], prob.edge_face[ed]):
            mt = prob.mats(K)
            S = hdg.schur_block(mt)
            bK = hdg.rhs_block(mt, hdg.load_vector(prob.ref, mt, fq[K]))
            rows = slice(f * p1, (f + 1) * p1)
            lK = lam[prob.dofs(K)]
            res += S[rows] @ lK - bK[rows]
            scale += np.abs(S[rows]) @ np.abs(lK) + np.abs(bK[rows])
        worst = max(worst, np.max(np.abs(res) / scale))
    assert worst < 1e-12
    # boundary entries are zero
    bnd = np.setdiff1d(np.arange(prob.ndof), prob.interior_dofs())
    assert np.all(lam[bnd] == 0.0)
