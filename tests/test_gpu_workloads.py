"""GPU parity on the benchmark workloads at their real sizes.

- crossing sweep: 16 volumes of 10^3, N = 96, MSE and Rician NLL (sigma per volume):
  objective, gradient per block and group gradients in full, then Adam iterations.
- bundle phantom: 64^3 (262,144 voxels), N = 360, NLL + calibration + neighbour priors:
  y_hat and the voxel gradient on sampled whole patches (the oracle evaluates them one patch
  at a time with the volume's normaliser and the library's group parameters); group
  gradients on a calibrated volume the oracle finishes in seconds.
- HCP-shaped brain: 740,110 voxels, N = 288, MSE + neighbour priors, in the launch
  configuration bench.py times (fused, one thread per voxel, CUDA graph): two iterations,
  then the parameters of sampled whole patches against the oracle's two iterations.
- DiSCo1-shaped fit: 40^3, N = 364, K = 5, Rician NLL with the topology and smoothness priors,
  in its default launch configuration: one iteration, sampled whole patches.
- mixed batch: 8 volumes with 96/288/360-measurement schemes, NLL + calibration, in full.
"""
import types

import numpy as np
import pytest
import torch

import phantoms as P
from oracle import prism_oracle as O
from tests.helpers import (TOL_GRAD, TOL_LOSS, TOL_SIGNAL, block_slices, make_pair, normwise, oracle_opts,
                           signal_rel, split_groups)
from tests.test_gpu_fused_gradient import fused_gradient

pytestmark = pytest.mark.gpu


def _patch_ids(vol, patch_dim, n, seed=0):
    mask = vol.mask.astype(bool)
    coords = np.argwhere(mask)
    pshape = tuple(-(-s // patch_dim) for s in mask.shape)
    pid = np.ravel_multi_index(tuple((coords // patch_dim).T), pshape)
    ids, counts = np.unique(pid, return_counts=True)
    rng = np.random.default_rng(seed)
    full = ids[np.argmax(counts)]
    ragged = ids[np.argmin(counts)]
    rest = rng.choice(ids, size=max(0, n - 2), replace=False)
    return np.unique(np.concatenate([[full, ragged], rest])), pid


@pytest.mark.parametrize("loss", ["mse", "nll"])
def test_crossing_sweep_full(loss):
    vols = P.crossing_sweep(0)
    K = 3
    rng = np.random.default_rng(2)
    inits = [(P.default_init(v.n_vox, K, 10 + i) + rng.normal(0, 0.2, (v.n_vox, 4 * K + 5))).astype(np.float32)
             for i, v in enumerate(vols)]
    f, ovs = make_pair(vols, inits, K=K, loss=loss, patch_dim=10)
    gps = split_groups(f.groups(), f)
    loss_g, _ = f.forward()
    gth, gg = f.backward()
    torch.cuda.synchronize()
    gth = gth.cpu().numpy()
    gg = gg.cpu().numpy()
    off = f.group_layout()
    v0 = 0
    for gi, ov in enumerate(ovs):
        th = torch.as_tensor(inits[gi]).double()
        J, _, g, ggr = O.value_and_grad(ov, th, gps[gi])
        assert abs(float(loss_g[gi]) - float(J)) <= TOL_LOSS * abs(float(J))
        for name, sl in block_slices(K).items():
            assert normwise(gth[v0:v0 + ov.n_vox, sl], g[:, sl].numpy()) <= TOL_GRAD, (gi, name)
        if loss == "nll":
            assert normwise([gg[int(off[4 * gi])]], [float(ggr["sigma_log"])]) <= TOL_GRAD
        v0 += ov.n_vox
    # five fused iterations against the oracle's trajectory
    f.set_params(torch.as_tensor(np.concatenate(inits)).cuda())
    f.step(5)
    f.sync()
    res = O.fit(ovs, [torch.as_tensor(t).double() for t in inits], 5)
    np.testing.assert_allclose(f.loss_history(), res.loss_history, rtol=1e-5)
    th = f.params_host()
    assert float(np.max(np.abs(th - np.concatenate([t.numpy() for t in res.theta])))) < 5e-4
    f.close()


def test_bundle_phantom_sampled_patches():
    vol = P.bundle_phantom(0, device="cuda")
    K = 3
    kw = dict(K=K, loss="nll", calibration=True, lam_sp=0.01, lam_dir=0.005, patch_dim=16)
    th0 = P.default_init(vol.n_vox, K, 7)
    rng = np.random.default_rng(3)
    th0 = (th0 + rng.normal(0, 0.2, th0.shape)).astype(np.float32)
    import paper_2604_00250_gb300 as prism
    v = types.SimpleNamespace(mask=vol.mask, signal=torch.as_tensor(vol.signal).cuda(), bvals=vol.bvals,
                              bvecs=vol.bvecs, init=th0)
    f = prism.Fitter([v], prism.options(**kw))
    packed = f.groups().copy()
    off = f.group_layout()
    N = vol.n_meas
    packed[int(off[1]):int(off[1]) + N] = rng.normal(0, 0.03, N)
    packed[int(off[2]):int(off[2]) + N] = rng.normal(0, 0.01, N)
    packed[int(off[3]):int(off[3]) + 512] = rng.normal(0, 0.05, 512)
    f.set_groups(packed)
    gp = split_groups(packed, f)[0]
    _, yhat = f.forward(want_yhat=True)
    gth, _ = f.backward()
    torch.cuda.synchronize()
    yhat = yhat.cpu().numpy().reshape(vol.n_vox, N)
    gth = gth.cpu().numpy()
    ids, pid = _patch_ids(vol, 16, 4)
    ov = O.OracleVolume(vol.mask, vol.signal, vol.bvals, vol.bvecs, oracle_opts(**kw), patches=ids)
    th = torch.as_tensor(th0[ov.sel]).double()
    yref, _ = O.predict(ov, th, gp)
    assert signal_rel(yhat[ov.sel], yref.numpy()) <= TOL_SIGNAL
    _, _, g, _ = O.value_and_grad(ov, th, gp, n_norm=ov.n_mask)
    for name, sl in block_slices(K).items():
        assert normwise(gth[ov.sel][:, sl], g[:, sl].numpy()) <= TOL_GRAD, name
    f.close()


def test_calibrated_volume_group_gradients():
    """A 24^3 bundle phantom, N = 360, NLL + calibration: sigma, alpha, beta and b_lr gradients
    and the objective in full (the oracle finishes in seconds; 108 tiles span two reduction splits)."""
    vol = P.bundle_phantom(1, edge=24, device="cpu")
    K = 3
    kw = dict(K=K, loss="nll", calibration=True, lam_sp=0.01, lam_dir=0.005, patch_dim=8, threads_per_voxel=1)
    th0 = P.default_init(vol.n_vox, K, 8)
    f, ovs = make_pair([vol], [th0], **kw)
    rng = np.random.default_rng(4)
    packed0 = f.groups().copy()
    packed = packed0.copy()
    off = f.group_layout()
    N = vol.n_meas
    packed[int(off[1]):int(off[1]) + N] = rng.normal(0, 0.03, N)
    packed[int(off[2]):int(off[2]) + N] = rng.normal(0, 0.01, N)
    packed[int(off[3]):int(off[3]) + 512] = rng.normal(0, 0.05, 512)
    f.set_groups(packed)
    gp = split_groups(packed, f)[0]
    loss_g, _ = f.forward()
    _, gg = f.backward()
    torch.cuda.synchronize()
    gg = gg.cpu().numpy()
    J, _, _, ggr = O.value_and_grad(ovs[0], torch.as_tensor(th0).double(), gp)
    assert abs(float(loss_g[0]) - float(J)) <= TOL_LOSS * abs(float(J))
    a, b, c, d = (int(x) for x in off[:4])
    assert normwise([gg[a]], [float(ggr["sigma_log"])]) <= TOL_GRAD
    assert normwise(gg[b:b + N], ggr["alpha"].numpy()) <= TOL_GRAD
    assert normwise(gg[c:c + N], ggr["beta"].numpy()) <= TOL_GRAD
    assert normwise(gg[d:d + 512], ggr["blr"].numpy().ravel()) <= TOL_GRAD
    # and three fused iterations of every parameter, group ones included, from the initial state
    f.set_groups(packed0)
    f.step(3)
    f.sync()
    res = O.fit(ovs, [torch.as_tensor(th0).double()], 3)
    np.testing.assert_allclose(f.loss_history()[:, 0], res.loss_history[:, 0], rtol=1e-5)
    f.close()


def test_brain_bench_configuration_sampled_patches():
    vol = P.brain_phantom(0, device="cuda")
    K = 3
    kw = dict(K=K, loss="mse", patch_dim=16, lam_sp=0.01, lam_dir=0.005)
    import paper_2604_00250_gb300 as prism
    v = types.SimpleNamespace(mask=vol.mask, signal=torch.as_tensor(vol.signal).cuda(), bvals=vol.bvals,
                              bvecs=vol.bvecs, init=None)
    f = prism.Fitter([v], prism.options(fused=1, use_graph=1, **kw))
    assert f.shape()["threads_per_voxel"] == 1 and f.shape()["tile_voxels"] == 128
    assert f.shape()["shell_loop"] == 1            # 18 b = 0 + 3 x 90: every shell even
    th0 = f.params_host()
    f.step(2)
    f.sync()
    th2 = f.params_host()
    hist = f.loss_history()
    f.close()
    assert np.isfinite(hist).all() and hist[1, 0] < hist[0, 0]
    ids, _ = _patch_ids(vol, 16, 3)
    ov = O.OracleVolume(vol.mask, vol.signal, vol.bvals, vol.bvecs, oracle_opts(**kw), patches=ids)
    th = torch.as_tensor(th0[ov.sel]).double()
    adam = O.Adam(ov.opts)
    gp = O.group_init(ov)
    for _ in range(2):
        adam.t += 1
        _, _, g, _ = O.value_and_grad(ov, th, gp, n_norm=ov.n_mask)
        th = adam.step("theta", th, g)
    diff = np.abs(th2[ov.sel] - th.numpy())
    assert float(diff.max()) < 3e-4, float(diff.max())


def test_disco_shaped_configuration_sampled_patches():
    """The DiSCo1-shaped fit of bench.py --workload disco (40^3, N = 364 up to b = 13,192, K = 5,
    Rician NLL, topology and smoothness priors) in its default launch configuration (on a GB300
    four lanes per voxel: 500 tiles of 128 voxels would fill 456 resident CTAs 1.1 times), one
    graph-replayed iteration from the default start: the gradient of sampled whole patches (read
    from Adam's first moment, m = (1 - beta1) g after one step) against the oracle's, normwise
    per parameter block. (Comparing the stepped parameters instead would test rounding noise:
    Adam's first step turns every gradient component above eps into +-lr, among them the radial
    components of the raw directions, which are zero up to rounding.)"""
    sch = P.make_scheme(4, [(1000, 90), (3000, 90), (7000, 90), (13192, 90)], 0)
    vol = P.bundle_phantom(0, edge=40, snr=50.0, scheme=sch, device="cuda")
    K = 5
    kw = dict(K=K, loss="nll", patch_dim=16, lam_rep=0.01, lam_sparse=0.02, lam_sp=0.01, lam_dir=0.005,
              lam_orphan=0.01, lam_order=0.01)
    import paper_2604_00250_gb300 as prism
    v = types.SimpleNamespace(mask=vol.mask, signal=torch.as_tensor(vol.signal).cuda(), bvals=vol.bvals,
                              bvecs=vol.bvecs, init=None)
    f = prism.Fitter([v], prism.options(fused=1, use_graph=1, **kw))
    # the default shape: four lanes per voxel where 128-voxel tiles fill the resident CTAs
    # (three per SM for five fibers) 0.75-1.25 times
    waves = vol.n_vox / 128 / (torch.cuda.get_device_properties(0).multi_processor_count * 3)
    assert f.shape()["threads_per_voxel"] == (4 if 0.75 < waves <= 1.25 else 1)
    th0 = f.params_host()
    gp = split_groups(f.groups().copy(), f)[0]
    f.step(1)
    f.sync()
    g_vox, _ = fused_gradient(f, f.opts.beta1)
    f.close()
    ids, _ = _patch_ids(vol, 16, 4)
    ov = O.OracleVolume(vol.mask, vol.signal, vol.bvals, vol.bvecs, oracle_opts(**kw), patches=ids)
    th = torch.as_tensor(th0[ov.sel]).double()
    _, _, g, _ = O.value_and_grad(ov, th, gp, n_norm=ov.n_mask)
    for name, sl in block_slices(K).items():
        e = normwise(g_vox[ov.sel][:, sl], g[:, sl].numpy())
        assert e <= TOL_GRAD, (name, e)


def test_mixed_batch_full():
    edges = (12, 14, 16, 18, 20, 22, 24, 26)
    vols = P.multi_volume_batch(0, edges=edges)
    K = 3
    kw = dict(K=K, loss="nll", calibration=True, lam_sp=0.01, lam_dir=0.005, patch_dim=8, threads_per_voxel=1)
    inits = [P.default_init(v.n_vox, K, 20 + i) for i, v in enumerate(vols)]
    f, ovs = make_pair(vols, inits, **kw)
    f.step(3)
    f.sync()
    res = O.fit(ovs, [torch.as_tensor(t).double() for t in inits], 3)
    np.testing.assert_allclose(f.loss_history(), res.loss_history, rtol=1e-5)
    th = f.params_host()
    assert float(np.max(np.abs(th - np.concatenate([t.numpy() for t in res.theta])))) < 5e-4
    f.close()
