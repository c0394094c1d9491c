"""GPU parity on edge cases: a one-voxel volume (alone and in a batch), the largest accepted
measurement count, and the smallest and largest patch edges."""
import numpy as np
import pytest
import torch

import phantoms as P
from oracle import prism_oracle as O
from tests.helpers import inits_for, make_pair

pytestmark = pytest.mark.gpu


def _fit_pair(vols, K, T, **kw):
    inits = inits_for(vols, K, 31)
    f, ovs = make_pair(vols, inits, K=K, **kw)
    f.step(T)
    f.sync()
    res = O.fit(ovs, [torch.as_tensor(t).double() for t in inits], T)
    np.testing.assert_allclose(f.loss_history(), res.loss_history, rtol=1e-5)
    ref = np.concatenate([t.numpy() for t in res.theta])
    assert float(np.max(np.abs(f.params_host() - ref))) < 3e-4
    f.close()


def _one_voxel(seed, scheme):
    m = np.zeros((3, 3, 3), np.uint8)
    m[1, 2, 0] = 1
    v = P.random_volume((3, 3, 3), scheme=scheme, seed=seed, mask_density=1.0)
    sig = np.asarray(v.signal)[np.flatnonzero(v.mask.ravel())]
    keep = np.ravel_multi_index((1, 2, 0), (3, 3, 3))
    return P.Volume(mask=m, signal=np.ascontiguousarray(sig[[keep]]), bvals=v.bvals, bvecs=v.bvecs)


@pytest.mark.parametrize("loss,cal", [("mse", False), ("nll", True)])
def test_one_voxel_volume(loss, cal):
    sch = P.make_scheme(2, [(1000, 9), (2500, 10)], 4)
    _fit_pair([_one_voxel(0, sch)], 3, 3, loss=loss, calibration=cal, patch_dim=4, lam_sp=0.01, lam_dir=0.005)


def test_one_voxel_volume_in_a_batch_with_one_thread_per_voxel():
    sch = P.make_scheme(2, [(1000, 9), (2500, 10)], 4)
    big = P.random_volume((8, 8, 8), scheme=sch, seed=2, mask_density=0.9)
    _fit_pair([big, _one_voxel(1, sch)], 3, 3, loss="mse", patch_dim=4, lam_sp=0.01, lam_dir=0.005,
              threads_per_voxel=1)


@pytest.mark.parametrize("cal", [False, True])
def test_largest_measurement_count(cal):
    """N = 1024, the largest accepted (its tables need more than 48 KB of shared memory)."""
    sch = P.make_scheme(16, [(1000, 336), (2000, 336), (3000, 336)], 5)
    assert sch[0].shape[0] == 1024
    vol = P.random_volume((4, 4, 5), scheme=sch, seed=3, mask_density=0.8, calibration=cal)
    _fit_pair([vol], 3, 2, loss="mse", calibration=cal, patch_dim=4, threads_per_voxel=1)


@pytest.mark.parametrize("patch_dim", [1, 64])
def test_patch_edges(patch_dim):
    """patch_dim 1 leaves every voxel without neighbours; 64 puts the whole volume in one patch."""
    sch = P.make_scheme(2, [(1000, 9), (2500, 10)], 6)
    vol = P.random_volume((6, 5, 7), scheme=sch, seed=4, mask_density=0.7)
    _fit_pair([vol], 3, 3, loss="mse", patch_dim=patch_dim, lam_sp=0.01, lam_dir=0.005)
