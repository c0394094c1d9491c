"""GPU parity: the CUDA library (through the C-ABI) against the FP64 oracle.

Element-wise y_hat, objective per group, gradient per parameter block, one Adam
step (fused and plain paths), and a 200-iteration fit of the one-patch crossing
workload. Sizes span several tiles with ragged tails.
"""
import numpy as np
import pytest
import torch

import phantoms as P
from oracle import metrics as M
from oracle import prism_oracle as O
from tests.helpers import (TOL_GRAD, TOL_LOSS, TOL_SIGNAL, block_slices, inits_for, make_pair, normwise,
                           signal_rel, split_groups)

pytestmark = pytest.mark.gpu

CASES = [
    # loss, calibration, K, threads per voxel, extra options
    ("mse", False, 3, 1, dict(lam_sp=0.01, lam_dir=0.005)),
    ("mse", False, 3, 4, dict(lam_sp=0.01, lam_dir=0.005)),
    ("mse", False, 3, 16, dict()),
    ("nll", False, 2, 1, dict()),
    ("nll", False, 3, 4, dict(lam_sp=0.01)),
    ("mse", True, 3, 1, dict(lam_dir=0.005)),
    ("nll", True, 3, 1, dict(lam_sp=0.01, lam_dir=0.005)),
    ("nll", True, 2, 16, dict()),
    ("mse", False, 1, 1, dict()),
    ("mse", False, 5, 4, dict(lam_sp=0.01)),
    # remaining stabilisers of Sec. 2.4 and the 26-neighbourhood
    ("mse", False, 3, 1, dict(lam_sp=0.01, lam_dir=0.005, lam_orphan=0.01, lam_order=0.01, connectivity=26)),
    ("nll", True, 3, 4, dict(lam_sp=0.01, lam_orphan=0.01, s_orphan=0.5, lam_order=0.01, connectivity=26)),
]


def _problem(cal, seed=0, nvol=2):
    sch = P.make_scheme(3, [(1000, 14), (2500, 15)], seed)       # N = 32
    sch2 = P.make_scheme(2, [(800, 9), (2000, 10)], seed + 1)    # N = 21
    vols = [P.random_volume((7, 5, 6), scheme=sch, seed=seed, mask_density=0.75, calibration=cal)]
    if nvol > 1:
        vols.append(P.random_volume((5, 6, 4), scheme=sch2, seed=seed + 1, mask_density=0.6, calibration=cal))
    return vols


def _perturb_groups(f, rng, cal, loss):
    packed = f.groups().copy()
    for gi, g in enumerate(f.group_view(packed)):
        off = f.group_layout()
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


@pytest.mark.parametrize("loss,cal,K,tpv,extra", CASES)
def test_forward_and_gradient(loss, cal, K, tpv, extra):
    rng = np.random.default_rng(1)
    vols = _problem(cal)
    inits = [th + rng.normal(0, 0.3, th.shape).astype(np.float32) for th in inits_for(vols, K, 3)]
    kw = dict(K=K, loss=loss, calibration=cal, patch_dim=4, threads_per_voxel=tpv, **extra)
    f, ovs = make_pair(vols, inits, **kw)
    packed = _perturb_groups(f, rng, cal, loss)
    gps = split_groups(packed, f)
    loss_g, yhat = f.forward(want_yhat=True)
    gth, gg = f.backward()
    torch.cuda.synchronize()
    yhat = yhat.cpu().numpy()
    gth = gth.cpu().numpy()
    gg = gg.cpu().numpy()
    off = f.group_layout()
    pos = 0
    vpos = 0
    for gi, ov in enumerate(ovs):
        th = torch.as_tensor(inits[gi]).double()
        yref, _ = O.predict(ov, th, gps[gi])
        n = ov.n_vox * ov.n_meas
        assert signal_rel(yhat[pos:pos + n].reshape(ov.n_vox, ov.n_meas), yref.numpy()) <= TOL_SIGNAL
        pos += n
        J, parts, g, ggr = O.value_and_grad(ov, th, gps[gi])
        assert abs(float(loss_g[gi]) - float(J)) <= TOL_LOSS * abs(float(J)), (gi, float(loss_g[gi]), float(J), parts)
        gv = gth[vpos:vpos + ov.n_vox]
        vpos += ov.n_vox
        for name, sl in block_slices(K).items():
            e = normwise(gv[:, sl], g[:, sl].numpy())
            assert e <= TOL_GRAD, (gi, name, e)
        a, b, c, d = (int(x) for x in off[4 * gi:4 * gi + 4])
        N = ov.n_meas
        if loss == "nll":
            e = normwise([gg[a]], [float(ggr["sigma_log"])])
            assert e <= TOL_GRAD, ("sigma", e, gg[a], float(ggr["sigma_log"]))
        if cal:
            assert normwise(gg[b:b + N], ggr["alpha"].numpy()) <= TOL_GRAD
            assert normwise(gg[c:c + N], ggr["beta"].numpy()) <= TOL_GRAD
            assert normwise(gg[d:d + 512], ggr["blr"].numpy().ravel()) <= TOL_GRAD
    f.close()


@pytest.mark.parametrize("fused,tpv", [(1, 1), (1, 4), (1, 16), (0, 1), (0, 4)])
@pytest.mark.parametrize("loss,cal", [("mse", False), ("nll", True), ("nll", False), ("mse", True)])
def test_adam_steps_match_oracle(fused, tpv, loss, cal):
    """Three iterations (objective, gradient, Adam) on the fused path (packed two-measurement
    steps for one thread per voxel with MSE and no calibration) and the plain path; one volume
    has an odd measurement count (21), so masked partial chunks and pairs are exercised."""
    vols = _problem(cal)
    K = 3
    inits = inits_for(vols, K, 5)
    kw = dict(K=K, loss=loss, calibration=cal, patch_dim=4, lam_sp=0.01, lam_dir=0.005, fused=fused,
              use_graph=fused, threads_per_voxel=tpv)
    f, ovs = make_pair(vols, inits, **kw)
    f.step(3)
    f.sync()
    th = f.params_host()
    res = O.fit(ovs, [torch.as_tensor(t).double() for t in inits], 3)
    hist = f.loss_history()
    np.testing.assert_allclose(hist, res.loss_history, rtol=1e-5)
    ref = np.concatenate([t.numpy() for t in res.theta])
    # each Adam step moves a parameter by ~lr; three steps agree to float32 rounding
    assert float(np.max(np.abs(th - ref))) < 3e-4
    f.close()


@pytest.mark.parametrize("tpv", [16, 1])
def test_fit_crossing_patch_200_iterations(tpv):
    """One 8^3 patch of crossings, 96 measurements, MSE, 200 Adam iterations: median
    matched angular deviation <= 0.5 deg and identical peak counts per voxel."""
    vol = P.crossing_patch(0)
    K = 3
    th0 = P.default_init(vol.n_vox, K, 0)
    f, ovs = make_pair([vol], [th0], K=K, patch_dim=8, threads_per_voxel=tpv)
    f.step(200)
    f.sync()
    th_gpu = f.params_host()
    res = O.fit(ovs, [torch.as_tensor(th0).double()], 200)
    dev, pa, pb = M.matched_deviation(res.theta[0].numpy(), th_gpu, K)
    assert float(np.median(dev)) <= 0.5, float(np.median(dev))
    assert np.array_equal(pa, pb), int(np.sum(pa != pb))
    np.testing.assert_allclose(f.loss_history()[:, 0], res.loss_history[:, 0], rtol=1e-3)
    f.close()


@pytest.mark.parametrize("loss,cal,tpv", [("nll", True, 0), ("mse", False, 1)])
def test_fused_is_deterministic_and_resumable(loss, cal, tpv):
    vols = _problem(cal)
    K = 3
    inits = inits_for(vols, K, 9)
    kw = dict(K=K, loss=loss, calibration=cal, patch_dim=4, lam_sp=0.01, lam_dir=0.005, threads_per_voxel=tpv)
    f1, _ = make_pair(vols, inits, **kw)
    f1.step(6)
    blob = f1.state()
    f1.step(6)
    a = f1.params_host()
    f2, _ = make_pair(vols, inits, **kw)
    f2.step(12)
    b = f2.params_host()
    assert np.array_equal(a, b)
    f3, _ = make_pair(vols, inits, **kw)
    f3.load_state(blob)
    f3.step(6)
    c = f3.params_host()
    assert np.array_equal(a, c)
    assert np.array_equal(f1.groups(), f3.groups())
    for f in (f1, f2, f3):
        f.close()


def test_nonfinite_signal_is_rejected():
    import paper_2604_00250_gb300 as prism
    vol = P.random_volume((3, 3, 3), seed=2)
    sig = vol.signal.copy()
    sig[4, 7] = np.nan
    from tests.helpers import gpu_volume
    v = gpu_volume(vol)
    v.signal = sig
    with pytest.raises(prism.PrismError) as e:
        prism.Fitter([v], prism.options(K=2))
    assert e.value.code == 5


@pytest.mark.parametrize("fused,tpv,loss,cal", [(1, 1, "mse", False), (1, 4, "nll", True), (1, 1, "nll", False),
                                                (0, 4, "mse", True)])
def test_rprop_steps_match_oracle(fused, tpv, loss, cal):
    """Three Rprop iterations (the paper's solver, Sec. 2.5) of every parameter, group ones
    included. Rprop moves each parameter by +-step whatever the gradient's size, so a
    parameter whose gradient sign is decided by rounding may take the other branch; all
    others agree to float32 rounding."""
    vols = _problem(cal)
    K = 3
    inits = inits_for(vols, K, 6)
    kw = dict(K=K, loss=loss, calibration=cal, patch_dim=4, lam_sp=0.01, lam_dir=0.005, fused=fused,
              use_graph=fused, threads_per_voxel=tpv, optimizer="rprop")
    f, ovs = make_pair(vols, inits, **kw)
    f.step(3)
    f.sync()
    th = f.params_host()
    res = O.fit(ovs, [torch.as_tensor(t).double() for t in inits], 3, optimizer="rprop")
    np.testing.assert_allclose(f.loss_history(), res.loss_history, rtol=1e-4)
    d = np.abs(th - np.concatenate([t.numpy() for t in res.theta]))
    assert float(np.mean(d < 1e-5)) >= 0.99, float(np.mean(d < 1e-5))
    f.close()



@pytest.mark.parametrize("tpv,loss,cal", [(1, "mse", False), (4, "nll", True)])
def test_stabilisers_26_connectivity_steps(tpv, loss, cal):
    """Three fused iterations with orphan-WM suppression, fiber ordering and 26-connected
    neighbour priors against the oracle's trajectory."""
    vols = _problem(cal)
    K = 3
    inits = inits_for(vols, K, 13)
    kw = dict(K=K, loss=loss, calibration=cal, patch_dim=4, lam_sp=0.01, lam_dir=0.005, lam_orphan=0.01,
              s_orphan=0.5, lam_order=0.01, connectivity=26, threads_per_voxel=tpv)
    f, ovs = make_pair(vols, inits, **kw)
    f.step(3)
    f.sync()
    res = O.fit(ovs, [torch.as_tensor(t).double() for t in inits], 3)
    np.testing.assert_allclose(f.loss_history(), res.loss_history, rtol=1e-5)
    th = f.params_host()
    assert float(np.max(np.abs(th - np.concatenate([t.numpy() for t in res.theta])))) < 3e-4
    f.close()



def test_fiber_readout_matches_oracle_metrics():
    """prism_get_fibers: directions, fractions and peak flags against the oracle's readout."""
    vols = _problem(False)
    K = 3
    rng = np.random.default_rng(17)
    inits = [(t + rng.normal(0, 0.8, t.shape)).astype(np.float32) for t in inits_for(vols, K, 17)]
    f, _ = make_pair(vols, inits, K=K, patch_dim=4)
    d, fr, pk = f.fibers(0.15)
    th = np.concatenate(inits)
    dref, fwm = M.fibers(th, K)
    np.testing.assert_allclose(d, dref, rtol=0, atol=TOL_SIGNAL)
    np.testing.assert_allclose(fr[:, 2:K + 2], fwm, rtol=TOL_SIGNAL, atol=1e-7)
    np.testing.assert_allclose(fr.sum(1), 1.0, atol=TOL_SIGNAL)
    share = fwm / fwm.sum(1, keepdims=True)
    clear = np.abs(share - 0.15) > 1e-4          # away from the threshold the decision is unique
    assert np.array_equal(pk[clear], M.peak_mask(fwm, 0.15)[clear])
    f.close()


def _interleave_b0(vols, seed):
    """The same volumes with their measurements in a seeded random order (b = 0 volumes
    scattered through the scheme, as scanners interleave them)."""
    out = []
    for i, v in enumerate(vols):
        perm = np.random.default_rng(seed + i).permutation(v.n_meas)
        out.append(P.Volume(mask=v.mask, signal=np.ascontiguousarray(np.asarray(v.signal)[:, perm]),
                            bvals=v.bvals[perm].copy(), bvecs=v.bvecs[perm].copy(), gt=v.gt))
    return out


@pytest.mark.parametrize("loss,tpv", [("mse", 1), ("nll", 4)])
def test_interleaved_b0_scheme(loss, tpv):
    """Without calibration the library moves the b = 0 measurements to the front of its table
    (the packed path then takes their pairs without the fiber terms); y_hat comes back in the
    caller's order, and a permuted scheme gives the oracle's objective, gradient and steps."""
    vols = _interleave_b0(_problem(False), 11)
    assert any(np.flatnonzero(v.bvals == 0).max() > 8 for v in vols)
    K = 3
    rng = np.random.default_rng(2)
    inits = [th + rng.normal(0, 0.3, th.shape).astype(np.float32) for th in inits_for(vols, K, 7)]
    kw = dict(K=K, loss=loss, patch_dim=4, threads_per_voxel=tpv, lam_sp=0.01, lam_dir=0.005)
    f, ovs = make_pair(vols, inits, **kw)
    packed = _perturb_groups(f, rng, False, loss)
    gps = split_groups(packed, f)
    loss_g, yhat = f.forward(want_yhat=True)
    gth, _ = f.backward()
    torch.cuda.synchronize()
    yhat, gth = yhat.cpu().numpy(), gth.cpu().numpy()
    pos = vpos = 0
    for gi, ov in enumerate(ovs):
        th = torch.as_tensor(inits[gi]).double()
        yref, _ = O.predict(ov, th, gps[gi])
        n = ov.n_vox * ov.n_meas
        assert signal_rel(yhat[pos:pos + n].reshape(ov.n_vox, ov.n_meas), yref.numpy()) <= TOL_SIGNAL
        pos += n
        J, _, g, _ = O.value_and_grad(ov, th, gps[gi])
        assert abs(float(loss_g[gi]) - float(J)) <= TOL_LOSS * abs(float(J))
        for name, sl in block_slices(K).items():
            assert normwise(gth[vpos:vpos + ov.n_vox, sl], g[:, sl].numpy()) <= TOL_GRAD, (gi, name)
        vpos += ov.n_vox
    f.close()
    # three fused iterations against the oracle's
    f, ovs = make_pair(vols, inits, **kw)
    f.step(3)
    f.sync()
    res = O.fit(ovs, [torch.as_tensor(t).double() for t in inits], 3)
    np.testing.assert_allclose(f.loss_history(), res.loss_history, rtol=1e-5)
    ref = np.concatenate([t.numpy() for t in res.theta])
    assert float(np.max(np.abs(f.params_host() - ref))) < 3e-4
    f.close()


@pytest.mark.parametrize("loss,cal", [("mse", False), ("nll", False), ("mse", True), ("nll", True)])
def test_adam_steps_five_fibers(loss, cal):
    """K = 5 (the paper's DiSCo1 setting) through the fused kernel with one thread per voxel:
    packed steps for the MSE, NLL and calibrated MSE, the scalar loop for the calibrated NLL,
    all compiled for 3 CTAs per SM."""
    vols = _problem(cal)
    K = 5
    inits = inits_for(vols, K, 9)
    kw = dict(K=K, loss=loss, calibration=cal, patch_dim=4, lam_sp=0.01, lam_dir=0.005, fused=1, use_graph=1,
              threads_per_voxel=1, lam_order=0.01)
    f, ovs = make_pair(vols, inits, **kw)
    f.step(3)
    f.sync()
    res = O.fit(ovs, [torch.as_tensor(t).double() for t in inits], 3)
    np.testing.assert_allclose(f.loss_history(), res.loss_history, rtol=1e-5)
    ref = np.concatenate([t.numpy() for t in res.theta])
    assert float(np.max(np.abs(f.params_host() - ref))) < 3e-4
    f.close()
