"""The paper-like CPU baseline (baselines/cpu_kronecker.py: the factorised face operator of
Sec. 2.4 applied in the three steps of Sec. 2.5.1 with numpy) against the oracle's
explicit face matrices.  Agreement pins the baseline that bench.py times."""
import numpy as np
import pytest

from baselines.cpu_kronecker import KroneckerCPU, KroneckerOpenMP
from oracle.ghost_penalty import Oracle
from paper_2503_00246_gb300 import workloads as W


@pytest.mark.parametrize("dim,n,k", [(2, 12, 1), (2, 12, 4), (2, 10, 7), (3, 6, 1), (3, 6, 2), (3, 6, 3), (3, 5, 5)])
@pytest.mark.parametrize("paper", [False, True])
def test_kronecker_cpu_equals_oracle(dim, n, k, paper):
    pr = W.small_ball(dim, n, k, radius=0.6, seed=300 + k, weights=W.paper_weights(0.5, k) if paper else None)
    o = Oracle(pr)
    kc = KroneckerCPU(pr, o)
    x = W.x_vectors(pr, o.n_active)[0]
    ref = o.apply(x)
    y = kc.apply(x)
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)
    for nt in (1, 3):
        y2 = KroneckerOpenMP(pr, o, nthreads=nt).apply(x)
        assert np.linalg.norm(y2 - ref) <= 1e-12 * np.linalg.norm(ref)
