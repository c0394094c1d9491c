"""The package's crossing-benchmark scoring (vectorised) against the oracle's plain loops
(reading R31), on seeded predictions near and far from the ground truth."""
import numpy as np
import pytest

from oracle import metrics as M
from paper_2604_00250_gb300 import crossing


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


@pytest.mark.parametrize("K,F,seed", [(2, 2, 0), (3, 2, 1), (5, 2, 2), (1, 2, 3)])
def test_score_matches_oracle(K, F, seed):
    rng = np.random.default_rng(seed)
    V = 400
    gt = _unit(rng.standard_normal((V, F, 3)))
    ff = np.where(rng.random((V, F)) < 0.8, 0.5, 0.0)
    ff[:, 0] = 0.5                                        # at least one ground-truth fiber
    # predictions: noisy copies of the ground truth (some far off), random sign and order
    d = np.empty((V, K, 3))
    for k in range(K):
        src = gt[:, k % F] + rng.normal(0, rng.choice([0.02, 0.3, 2.0], size=(V, 1)), (V, 3))
        d[:, k] = _unit(src) * rng.choice([-1.0, 1.0], size=(V, 1))
    peaks = rng.random((V, K)) < 0.8
    peaks[:, 0] = True
    case = rng.integers(0, 5, V)
    per_a, all_a, r_a, p_a, f_a = crossing.score(d, peaks, gt, ff, case)
    per_b, all_b, r_b, p_b, f_b = M.crossing_scores(d, peaks, gt, ff, case)
    assert per_a.keys() == per_b.keys()
    for c in per_a:
        assert abs(per_a[c] - per_b[c]) < 1e-9
    assert abs(all_a - all_b) < 1e-9
    assert (r_a, p_a) == (r_b, p_b)
    assert abs(f_a - f_b) < 1e-12
