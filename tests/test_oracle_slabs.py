"""Pins of the oracle's slab split and stitching (Sec. 3 "Configuration", readings R28, R29)
against hand values, invariants and constructed cases."""
import numpy as np
import pytest

from oracle import slabs as S



def _theta(rng, V, K):
    th = rng.normal(0, 1, (V, 4 * K + 5))
    th[:, 0] += 1.0
    return th


def _raw_from(s0, fr, fin, d):
    """Raw parameters reproducing given (S0, fractions, f_intra, unit directions) exactly
    up to rounding: inverse softplus, log fractions, logit, the directions themselves."""
    V, K = d.shape[0], d.shape[1]
    th = np.zeros((V, 4 * K + 5))
    th[:, 0] = np.log(np.expm1(s0))
    th[:, 1:K + 4] = np.log(fr)
    th[:, K + 4:4 * K + 4] = d.reshape(V, 3 * K)
    th[:, 4 * K + 4] = np.log(fin / (1 - fin))
    return th


def test_slab_ranges_hand_values():
    # 145 slices, 30-slice slabs with a 5-slice overlap: stride 25, the last slab clipped
    assert S.slab_ranges(145, 30, 5) == [(0, 30), (25, 55), (50, 80), (75, 105), (100, 130), (125, 145)]
    assert S.slab_ranges(20, 30, 5) == [(0, 20)]
    assert S.slab_ranges(30, 30, 5) == [(0, 30)]
    assert S.slab_ranges(31, 30, 5) == [(0, 30), (25, 31)]
    with pytest.raises(ValueError):
        S.slab_ranges(100, 10, 6)


def test_slab_weights_ramp_and_partition_of_unity():
    r = S.slab_ranges(60, 30, 5)
    w = S.slab_weights(60, r)
    np.testing.assert_allclose(w.sum(0), 1.0, rtol=0, atol=1e-15)
    # overlap of slabs 0 and 1 is slices 25..29: slab 1 ramps 0.1, 0.3, ..., 0.9
    np.testing.assert_allclose(w[1, 25:30], [0.1, 0.3, 0.5, 0.7, 0.9], atol=1e-15)
    np.testing.assert_allclose(w[0, 25:30], [0.9, 0.7, 0.5, 0.3, 0.1], atol=1e-15)
    assert np.all(w[0, :25] == 1) and np.all(w[1, 30:50] == 1)
    assert np.all(w[1, :25] == 0)


def test_match_fibers_hand_case():
    da = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    db = np.array([[0, 0, -1.0], [-1.0, 0, 0], [0, 0.8, 0.6]])
    p, s = S.match_fibers(da, db)
    assert p == (1, 2, 0)
    np.testing.assert_array_equal(s, [-1.0, 1.0, -1.0])


def test_single_slab_is_the_readout():
    rng = np.random.default_rng(0)
    mask = (rng.random((4, 3, 9)) < 0.7).astype(np.uint8)
    K = 2
    V = int(mask.sum())
    th = _theta(rng, V, K)
    r = S.slab_ranges(9, 30, 5)
    out = S.stitch(mask, r, [th], K)
    ref = S.readout(th, K)
    for a, b in zip(out, ref):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)


def test_permuted_flipped_copy_stitches_to_itself():
    """Slab B holds slab A's estimate with its fibers permuted and directions negated:
    in the overlap, matching and sign alignment must give back A exactly (weights sum to 1);
    where slab B is alone its own fiber labels stand (labels are per voxel)."""
    rng = np.random.default_rng(1)
    K = 3
    mask = np.ones((2, 2, 12), np.uint8)
    r = S.slab_ranges(12, 8, 3)                       # (0, 8), (5, 12): overlap slices 5..7
    assert r == [(0, 8), (5, 12)]
    s0, fr, fin, d = S.readout(_theta(rng, 2 * 2 * 12, K), K)
    vol = dict(s0=s0.reshape(2, 2, 12), fr=fr.reshape(2, 2, 12, K + 3), fin=fin.reshape(2, 2, 12),
               d=d.reshape(2, 2, 12, K, 3))
    perm = [2, 0, 1]

    def slab_params(z0, z1, permute):
        s = vol["s0"][:, :, z0:z1].reshape(-1)
        f = vol["fr"][:, :, z0:z1].reshape(-1, K + 3).copy()
        fi = vol["fin"][:, :, z0:z1].reshape(-1)
        dd = vol["d"][:, :, z0:z1].reshape(-1, K, 3).copy()
        if permute:
            f[:, 2:K + 2] = f[:, 2:K + 2][:, perm]
            dd = -dd[:, perm]
        return _raw_from(s, f, fi, dd)

    out = S.stitch(mask, r, [slab_params(0, 8, False), slab_params(5, 12, True)], K)
    z = np.argwhere(mask)[:, -1]
    a = z < 8                                        # slab A alone or the overlap: A's labels and signs
    b = ~a                                           # slab B alone: B's own labels and signs
    np.testing.assert_allclose(out[0], s0, atol=1e-12)
    np.testing.assert_allclose(out[2], fin, atol=1e-12)
    np.testing.assert_allclose(out[1][a], fr[a], atol=1e-12)
    np.testing.assert_allclose(out[3][a], d[a], atol=1e-12)
    fb = fr[b].copy()
    fb[:, 2:K + 2] = fb[:, 2:K + 2][:, perm]
    np.testing.assert_allclose(out[1][b], fb, atol=1e-12)
    np.testing.assert_allclose(out[3][b], -d[b][:, perm], atol=1e-12)


def test_overlap_interpolates_linearly():
    """Two slabs with the same directions and different fractions / S0: in the overlap the
    stitched value is (1 - w) a + w b with the ramp weights of R29."""
    K = 1
    mask = np.ones((1, 1, 10), np.uint8)
    r = S.slab_ranges(10, 6, 2)                       # (0, 6), (4, 10): overlap slices 4, 5
    d = np.tile(np.array([0.0, 0.6, 0.8]), (6, 1, 1))
    fa = np.tile([0.1, 0.2, 0.6, 0.1], (6, 1))
    fb = np.tile([0.3, 0.1, 0.4, 0.2], (6, 1))
    tha = _raw_from(np.full(6, 1.0), fa, np.full(6, 0.5), d)
    thb = _raw_from(np.full(6, 2.0), fb, np.full(6, 0.25), d)
    s0, fr, fin, dd = S.stitch(mask, r, [tha, thb], K)
    for z, wb in ((4, 0.25), (5, 0.75)):
        np.testing.assert_allclose(s0[z], (1 - wb) * 1.0 + wb * 2.0, atol=1e-12)
        np.testing.assert_allclose(fr[z], (1 - wb) * fa[0] + wb * fb[0], atol=1e-12)
        np.testing.assert_allclose(fin[z], (1 - wb) * 0.5 + wb * 0.25, atol=1e-12)
        np.testing.assert_allclose(dd[z, 0], [0.0, 0.6, 0.8], atol=1e-12)
    np.testing.assert_allclose(s0[:4], 1.0, atol=1e-12)
    np.testing.assert_allclose(s0[6:], 2.0, atol=1e-12)
