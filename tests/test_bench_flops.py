"""bench.py's algorithmic flop counts per voxel-iteration (the numerators of the roofline
fractions) against the counts stated with the kernels: the brain scheme (18 b = 0 + 3 x 90),
K = 3, shell loop 270 x (4 + 26 K) + 18 x 4 = 22,212 and per-measurement loop 270 x (17 + 28 K)
+ 18 x 5 = 27,360 (MSE); Rician NLL and calibration per measurement without the b = 0
shortcut."""
import numpy as np

import bench


def test_brain_scheme_counts():
    b = np.array([0.0] * 18 + [1000.0] * 90 + [2000.0] * 90 + [3000.0] * 90)
    assert bench.flops_per_voxel_iteration(b, "mse", False, 3, True) == 270 * 82 + 18 * 4 == 22212
    assert bench.flops_per_voxel_iteration(b, "mse", False, 3, False) == 270 * 101 + 18 * 5 == 27360
    assert bench.flops_per_voxel_iteration(b, "mse", True, 3, False) == 288 * (28 + 28 * 3)
    assert bench.flops_per_voxel_iteration(b, "nll", False, 3, False) == 288 * (85 + 28 * 3)
    assert bench.flops_per_voxel_iteration(b, "nll", True, 5, False) == 288 * (94 + 28 * 5)


def test_odd_b0_count_in_the_per_measurement_loop():
    # the per-measurement loop takes b = 0 measurements apart only in whole pairs
    b = np.array([0.0] * 5 + [1000.0] * 10)
    assert bench.flops_per_voxel_iteration(b, "mse", False, 3, False) == 11 * 101 + 4 * 5
