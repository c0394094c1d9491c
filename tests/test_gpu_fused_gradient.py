"""The fused kernel's own gradient against the oracle's, block by block.

The fused iteration (synthesis, data term, adjoint, priors and Adam in one persistent
kernel, replayed from a CUDA graph) never exposes its gradient. But one iteration from zero
Adam state leaves the first moment m = (1 - beta1) g (Adam, the Table 2 comparator), for
every voxel parameter and every group parameter. So g = m / (1 - beta1) is read from the
checkpoint blob (prism_get_state: header, theta, m, v in [V][Q] mask order, then the packed
group parameters and their two moments) and compared with the oracle's gradient at the
starting point, normwise per block (S0, logits, dirs, f_in, sigma, alpha, beta, b_lr).
Adam's step is invariant to a per-block scale of the gradient, so the trajectory tests
alone would not catch an adjoint off by a constant factor; this test does.
"""
import types

import numpy as np
import pytest
import torch

import phantoms as P
from oracle import prism_oracle as O
from tests.helpers import (TOL_GRAD, TOL_LOSS, block_slices, inits_for, make_pair, normwise, oracle_opts,
                           split_groups)

pytestmark = pytest.mark.gpu

HEADER = np.dtype([("magic", "<u4"), ("version", "<u4"), ("K", "<i4"), ("Q", "<i4"), ("G", "<i4"),
                   ("step", "<i4"), ("V", "<i8"), ("GP", "<i8")])


def parse_state(blob):
    """(header, theta, m, v, groups, gm, gv) of a prism_get_state blob."""
    hd = np.frombuffer(blob, HEADER, count=1)[0]
    V, Q, GP = int(hd["V"]), int(hd["Q"]), int(hd["GP"])
    body = np.frombuffer(blob, np.float32, offset=HEADER.itemsize)
    n = V * Q
    th, m, v = (body[i * n:(i + 1) * n].reshape(V, Q) for i in range(3))
    g0 = 3 * n
    gp, gm, gv = (body[g0 + i * GP:g0 + (i + 1) * GP] for i in range(3))
    return hd, th, m, v, gp, gm, gv


def _problem(cal, seed=0):
    sch = P.make_scheme(3, [(1000, 14), (2500, 15)], seed)       # N = 32
    sch2 = P.make_scheme(2, [(800, 9), (2000, 10)], seed + 1)    # N = 21 (odd: a partial pair)
    return [P.random_volume((7, 5, 6), scheme=sch, seed=seed, mask_density=0.75, calibration=cal),
            P.random_volume((5, 6, 4), scheme=sch2, seed=seed + 1, mask_density=0.6, calibration=cal)]


def _perturb(f, rng, cal, loss):
    packed = f.groups().copy()
    off = f.group_layout()
    for gi in range(f.n_groups):
        a, b, c, d = (int(x) for x in off[4 * gi:4 * gi + 4])
        N = f.n_meas[gi]
        if loss == "nll":
            packed[a] = np.log(0.05 + 0.02 * gi)
        if cal:
            packed[b:b + N] = rng.normal(0, 0.05, N)
            packed[c:c + N] = rng.normal(0, 0.02, N)
            packed[d:d + 512] = rng.normal(0, 0.1, 512)
    f.set_groups(packed)
    return packed


def fused_gradient(f, beta1):
    """(voxel gradient [V, Q], packed group gradient) of the handle's first iteration."""
    hd, _, m, _, _, gm, _ = parse_state(f.state())
    assert int(hd["step"]) == 1
    return m.astype(np.float64) / (1.0 - np.float64(np.float32(beta1))), gm.astype(np.float64) / (
        1.0 - np.float64(np.float32(beta1)))


CASES = [(loss, cal, tpv, K) for loss in ("mse", "nll") for cal in (False, True) for tpv in (1, 4, 16)
         for K in (3, 5)]


@pytest.mark.parametrize("loss,cal,tpv,K", CASES)
def test_fused_gradient_matches_oracle(loss, cal, tpv, K):
    rng = np.random.default_rng(100 + K + 10 * tpv)
    vols = _problem(cal)
    inits = [(t + rng.normal(0, 0.3, t.shape)).astype(np.float32) for t in inits_for(vols, K, 3)]
    kw = dict(K=K, loss=loss, calibration=cal, patch_dim=4, lam_sp=0.01, lam_dir=0.005, fused=1, use_graph=1,
              threads_per_voxel=tpv)
    f, ovs = make_pair(vols, inits, **kw)
    assert f.shape()["threads_per_voxel"] == tpv
    packed = _perturb(f, rng, cal, loss)
    gps = split_groups(packed, f)
    f.step(1)
    f.sync()
    g_vox, g_grp = fused_gradient(f, f.opts.beta1)
    hist = f.loss_history()
    off = f.group_layout()
    v0 = 0
    for gi, ov in enumerate(ovs):
        J, _, g, ggr = O.value_and_grad(ov, torch.as_tensor(inits[gi]).double(), gps[gi])
        assert abs(hist[0, gi] - float(J)) <= TOL_LOSS * abs(float(J)), (gi, hist[0, gi], float(J))
        for name, sl in block_slices(K).items():
            e = normwise(g_vox[v0:v0 + ov.n_vox, sl], g[:, sl].numpy())
            assert e <= TOL_GRAD, (gi, name, e)
        v0 += ov.n_vox
        a, b, c, d = (int(x) for x in off[4 * gi:4 * gi + 4])
        N = ov.n_meas
        if loss == "nll":
            e = normwise([g_grp[a]], [float(ggr["sigma_log"])])
            assert e <= TOL_GRAD, ("sigma", gi, e)
        if cal:
            assert normwise(g_grp[b:b + N], ggr["alpha"].numpy()) <= TOL_GRAD, ("alpha", gi)
            assert normwise(g_grp[c:c + N], ggr["beta"].numpy()) <= TOL_GRAD, ("beta", gi)
            assert normwise(g_grp[d:d + 512], ggr["blr"].numpy().ravel()) <= TOL_GRAD, ("blr", gi)
    f.close()


def _patch_ids(vol, patch_dim, n, seed=0):
    coords = np.argwhere(vol.mask.astype(bool))
    pshape = tuple(-(-s // patch_dim) for s in vol.mask.shape)
    pid = np.ravel_multi_index(tuple((coords // patch_dim).T), pshape)
    ids, counts = np.unique(pid, return_counts=True)
    rng = np.random.default_rng(seed)
    rest = rng.choice(ids, size=max(0, n - 2), replace=False)
    return np.unique(np.concatenate([[ids[np.argmax(counts)], ids[np.argmin(counts)]], rest]))


def test_brain_bench_configuration_fused_gradient():
    """The HCP-shaped brain (740,110 voxels, N = 288, MSE, neighbour priors) in the launch
    configuration bench.py times (fused, one thread per voxel, 128-voxel tiles, CUDA graph):
    the first iteration's gradient on sampled whole 16^3 patches (the fullest, the emptiest
    and two more) against the oracle's, with the volume's |M| as the normaliser."""
    import paper_2604_00250_gb300 as prism
    vol = P.brain_phantom(0, device="cuda")
    K = 3
    kw = dict(K=K, loss="mse", patch_dim=16, lam_sp=0.01, lam_dir=0.005)
    v = types.SimpleNamespace(mask=vol.mask, signal=torch.as_tensor(vol.signal).cuda(), bvals=vol.bvals,
                              bvecs=vol.bvecs, init=None)
    f = prism.Fitter([v], prism.options(fused=1, use_graph=1, **kw))
    assert f.shape()["threads_per_voxel"] == 1 and f.shape()["tile_voxels"] == 128
    assert f.shape()["shell_loop"] == 1
    th0 = f.params_host()
    f.step(1)
    f.sync()
    g_vox, _ = fused_gradient(f, f.opts.beta1)
    f.close()
    ids = _patch_ids(vol, 16, 4)
    ov = O.OracleVolume(vol.mask, vol.signal, vol.bvals, vol.bvecs, oracle_opts(**kw), patches=ids)
    _, _, g, _ = O.value_and_grad(ov, torch.as_tensor(th0[ov.sel]).double(), O.group_init(ov), n_norm=ov.n_mask)
    for name, sl in block_slices(K).items():
        e = normwise(g_vox[ov.sel][:, sl], g[:, sl].numpy())
        assert e <= TOL_GRAD, (name, e)
