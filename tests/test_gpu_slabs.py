"""GPU parity of the slab driver (Sec. 3 "Configuration", readings R28, R29):
prism_fit_init_slabs + prism_stitch_slabs against the oracle's slab split, per-slab fits
and stitching."""
import numpy as np
import pytest
import torch

import phantoms as P
from oracle import prism_oracle as O
from oracle import slabs as OS
from tests.helpers import oracle_opts

pytestmark = pytest.mark.gpu

K = 3


def _volume(seed=0, shape=(5, 4, 19)):
    sch = P.make_scheme(3, [(1000, 14), (2500, 15)], seed)
    return P.random_volume(shape, scheme=sch, seed=seed, mask_density=0.8)


def _slab_parts(vol, slab, overlap):
    """Oracle-side slab volumes: (ranges, [(sub_mask, signal_rows)]) for the non-empty slabs."""
    r = OS.slab_ranges(vol.mask.shape[-1], slab, overlap)
    z = np.argwhere(vol.mask)[:, -1]
    sig = np.asarray(vol.signal)
    parts = []
    keep = []
    for (z0, z1) in r:
        sel = (z >= z0) & (z < z1)
        if sel.any():
            parts.append((np.ascontiguousarray(vol.mask[..., z0:z1]), sig[sel]))
            keep.append((z0, z1))
    return keep, parts


def _fitter(vol, slab, overlap, **kw):
    import paper_2604_00250_gb300 as prism
    return prism.Fitter(vol, prism.options(K=K, patch_dim=4, **kw), slabs=(slab, overlap))


def _close_maps(gpu, ref, dir_mask=None, atol=2e-5):
    s0, fr, fin, d = gpu
    rs0, rfr, rfin, rd = ref
    np.testing.assert_allclose(s0, rs0, rtol=0, atol=atol * max(1.0, float(np.abs(rs0).max())))
    np.testing.assert_allclose(fr, rfr, rtol=0, atol=atol)
    np.testing.assert_allclose(fin, rfin, rtol=0, atol=atol)
    m = np.ones(d.shape[0], bool) if dir_mask is None else dir_mask
    np.testing.assert_allclose(d[m], rd[m], rtol=0, atol=10 * atol)


def _clear_matches(mask, ranges, thetas):
    """Voxels whose fiber matching (and hemisphere choice) has a clear winner, so that the
    FP32 and FP64 sides must take the same decision."""
    import itertools
    nz = mask.shape[-1]
    coords = np.argwhere(mask)
    per = []
    for (z0, z1), th in zip(ranges, thetas):
        c = np.argwhere(mask[..., z0:z1])
        c[:, -1] += z0
        per.append((OS.readout(th, K)[3], {tuple(x): i for i, x in enumerate(c)}))
    ok = np.ones(len(coords), bool)
    for v, cc in enumerate(coords):
        src = [(i, per[i][1][tuple(cc)]) for i, (z0, z1) in enumerate(ranges) if z0 <= cc[-1] < z1]
        if len(src) < 2:
            continue
        da = per[src[0][0]][0][src[0][1]]
        db = per[src[1][0]][0][src[1][1]]
        sums = sorted(sum(abs(float(da[k] @ db[p[k]])) for k in range(K)) for p in itertools.permutations(range(K)))
        p, _ = OS.match_fibers(da, db)
        dots = [abs(float(da[k] @ db[p[k]])) for k in range(K)]
        ok[v] = (sums[-1] - sums[-2] > 1e-4) and min(dots) > 1e-4
    return ok


def test_stitch_matches_oracle_on_given_parameters():
    vol = _volume(0)
    slab, overlap = 8, 3
    f = _fitter(vol, slab, overlap)
    ranges, parts = _slab_parts(vol, slab, overlap)
    assert f.n_groups == len(parts) >= 3
    rng = np.random.default_rng(4)
    th = rng.normal(0, 1, (f.n_vox, f.Q)).astype(np.float32)
    th[:, 0] += 1.0
    f.set_params(torch.as_tensor(th))
    gpu = f.stitch()
    counts = np.cumsum([0] + [p[1].shape[0] for p in parts])
    thetas = [th[counts[i]:counts[i + 1]].astype(np.float64) for i in range(len(parts))]
    ref = OS.stitch(vol.mask, ranges, thetas, K)
    _close_maps(gpu, ref, _clear_matches(vol.mask, ranges, thetas))
    f.close()


@pytest.mark.parametrize("loss,cal", [("mse", False), ("nll", False), ("nll", True)])
def test_slab_fit_matches_oracle(loss, cal):
    """Ten fused iterations on every slab (each its own volume, with its own sigma and, when
    calibrated, its own bias field and per-measurement affine) and the stitched maps, against
    the oracle's per-slab fits and stitching."""
    vol = _volume(1, shape=(4, 5, 17))
    slab, overlap = 7, 2
    kw = dict(loss=loss, calibration=cal, lam_sp=0.01, lam_dir=0.005)
    f = _fitter(vol, slab, overlap, **kw)
    ranges, parts = _slab_parts(vol, slab, overlap)
    th0 = f.params_host().astype(np.float64)
    f.step(10)
    f.sync()
    o = oracle_opts(K=K, patch_dim=4, **kw)
    ovs = [O.OracleVolume(m, s, vol.bvals, vol.bvecs, o) for m, s in parts]
    counts = np.cumsum([0] + [p[1].shape[0] for p in parts])
    res = O.fit(ovs, [torch.as_tensor(th0[counts[i]:counts[i + 1]]) for i in range(len(parts))], 10)
    np.testing.assert_allclose(f.loss_history(), res.loss_history, rtol=1e-5)
    thetas = [t.numpy() for t in res.theta]
    ref = OS.stitch(vol.mask, ranges, thetas, K)
    _close_maps(f.stitch(), ref, _clear_matches(vol.mask, ranges, thetas), atol=3e-4)
    f.close()


def test_slab_signal_in_device_memory_gives_the_same_fit():
    vol = _volume(2, shape=(4, 4, 13))
    f1 = _fitter(vol, 6, 2)
    dev = P.Volume(mask=vol.mask, signal=torch.as_tensor(np.asarray(vol.signal)).cuda(), bvals=vol.bvals,
                   bvecs=vol.bvecs)
    f2 = _fitter(dev, 6, 2)
    f1.step(5)
    f2.step(5)
    for a, b in zip(f1.stitch(), f2.stitch()):
        np.testing.assert_array_equal(a, b)
    f1.close()
    f2.close()


def test_stitch_into_given_arrays():
    """stitch(out=...) writes the same maps into caller arrays: numpy, pinned host tensors, or
    CUDA tensors; mismatched shapes or mixed memory spaces are refused before any call."""
    vol = _volume(4, shape=(4, 4, 13))
    f = _fitter(vol, 6, 2)
    f.step(3)
    ref = f.stitch()
    V = f.n_out
    shapes = ((V,), (V, K + 3), (V,), (V, K, 3))
    outs = [tuple(np.full(s, np.nan, np.float32) for s in shapes),
            tuple(torch.full(s, float("nan"), pin_memory=True) for s in shapes),
            tuple(torch.full(s, float("nan"), device="cuda") for s in shapes)]
    for out in outs:
        got = f.stitch(out=out)
        assert all(g is o for g, o in zip(got, out))
        for g, r in zip(got, ref):
            g = g.cpu().numpy() if isinstance(g, torch.Tensor) else g
            np.testing.assert_array_equal(g, r)
    with pytest.raises(ValueError):
        f.stitch(out=(np.empty((V + 1,), np.float32),) + outs[0][1:])
    with pytest.raises(ValueError):
        f.stitch(out=outs[0][:2] + outs[2][2:])
    f.close()


def test_stitch_on_a_plain_handle_is_a_state_error():
    import paper_2604_00250_gb300 as prism
    from paper_2604_00250_gb300._lib import PrismError
    vol = _volume(3, shape=(3, 3, 5))
    f = prism.Fitter(vol, prism.options(K=K, patch_dim=4))
    f.n_out = f.n_vox
    with pytest.raises(PrismError):
        f.stitch()
    f.close()
