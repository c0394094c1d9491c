"""FP32 (GPU) against FP64 (oracle) error of each benchmark configuration, stated per quantity.

For every configuration of the workloads (crossing patch, crossing sweep, bundle phantom, HCP-
shaped brain, multi-volume batch) this measures, through the C-ABI, at a perturbed starting
point and after a fit from the same start as the oracle's:
- the signal y_hat: max element-wise |dy| / max(|y_hat|, 1e-3);
- the objective J per volume: relative error;
- the gradient: normwise relative error per parameter block (S0, logits, dirs, f_in, and the
  group blocks sigma, alpha, beta, b_lr where the configuration learns them);
- the fitted fiber directions: the median over voxels of the angle between the GPU's and the
  oracle's fitted fibers after optimal matching (sign- and permutation-free), and the share of
  voxels with the same number of peaks (a fiber is a peak at >= 15 % of the white matter).
Where the oracle cannot evaluate the whole workload in seconds, the voxel quantities are taken on
sampled whole 16^3 patches (with the volume's |M| and the library's group parameters), J on the
whole volume in patch chunks, and the fit on the patches (without calibration patches are
independent problems) or on a smaller volume of the same kind, as each test says.

Each test asserts the tolerances of the parity tests (signal and J 1e-5, gradient 1e-4, median
direction 0.5 deg). With PRISM_ACCURACY_OUT set, the measured errors are appended to that file,
one JSON object per configuration.
"""
import json
import os
import types

import numpy as np
import pytest
import torch

import phantoms as P
from oracle import metrics as M
from oracle import prism_oracle as O
from tests.helpers import (TOL_GRAD, TOL_LOSS, TOL_SIGNAL, block_slices, make_pair, normwise, oracle_opts,
                           signal_rel, split_groups)

pytestmark = pytest.mark.gpu

TOL_DIR_DEG = 0.5
PATCH = 16


def _record(name, **kw):
    out = os.environ.get("PRISM_ACCURACY_OUT")
    if out:
        with open(out, "a") as fh:
            fh.write(json.dumps({"config": name, **kw}) + "\n")


def _patches(mask, n, seed=0, patch_dim=PATCH):
    coords = np.argwhere(np.asarray(mask).astype(bool))
    pshape = tuple(-(-s // patch_dim) for s in mask.shape)
    pid = np.ravel_multi_index(tuple((coords // patch_dim).T), pshape)
    ids, counts = np.unique(pid, return_counts=True)
    rng = np.random.default_rng(seed)
    pick = [ids[np.argmax(counts)], ids[np.argmin(counts)]]
    rest = [i for i in ids if i not in pick]
    pick += list(rng.choice(rest, size=min(len(rest), max(0, n - 2)), replace=False))
    return np.unique(np.asarray(pick)), ids


def _groups_of(f, packed):
    return split_groups(packed, f)


def _grad_errors(gth, g, K, gg=None, ggr=None, off=None, N=None, loss="mse", cal=False):
    e = {name: normwise(gth[:, sl], g[:, sl]) for name, sl in block_slices(K).items()}
    if gg is not None:
        a, b, c, d = (int(x) for x in off)
        if loss == "nll":
            e["sigma"] = normwise([gg[a]], [float(ggr["sigma_log"])])
        if cal:
            e["alpha"] = normwise(gg[b:b + N], ggr["alpha"].numpy())
            e["beta"] = normwise(gg[c:c + N], ggr["beta"].numpy())
            e["blr"] = normwise(gg[d:d + 512], ggr["blr"].numpy().ravel())
    return e


def _fit_compare(th_gpu, th_ref, K):
    dev, pa, pb = M.matched_deviation(th_ref, th_gpu, K)
    return float(np.median(dev)), float(np.mean(pa == pb))


def _chunked_objective(vol, opts, theta, gp, chunk_patches=8):
    """J of a whole volume from the oracle evaluated one chunk of whole patches at a time: the
    voxel sums (data term, priors, TV) add over chunks, the calibration L2 terms count once."""
    _, ids = _patches(vol.mask, 0, patch_dim=opts.patch_dim)
    ids = np.unique(ids)
    total = 0.0
    once = 0.0
    for i in range(0, len(ids), chunk_patches):
        ov = O.OracleVolume(vol.mask, vol.signal, vol.bvals, vol.bvecs, opts, patches=ids[i:i + chunk_patches])
        with torch.no_grad():
            _, parts = O.objective(ov, torch.as_tensor(theta[ov.sel]).double(), gp)
        for k, v in parts.items():
            if k in ("cal_alpha", "cal_beta", "cal_blr"):
                once = float(v)
            else:
                total += float(v)
    return total + once


def _perturb(f, rng, loss, cal, scale=1.0):
    packed = f.groups().copy()
    off = f.group_layout()
    for gi in range(f.n_groups):
        a, b, c, d = (int(x) for x in off[4 * gi:4 * gi + 4])
        N = f.n_meas[gi]
        if loss == "nll":
            packed[a] = np.log(0.05)
        if cal:
            packed[b:b + N] = rng.normal(0, 0.03 * scale, N)
            packed[c:c + N] = rng.normal(0, 0.01 * scale, N)
            packed[d:d + 512] = rng.normal(0, 0.05 * scale, 512)
    f.set_groups(packed)
    return packed


def test_crossing_patch_accuracy():
    """8^3 crossing patch, N = 96, K = 3, MSE: whole patch, 200 Adam iterations."""
    vol = P.crossing_patch(0)
    K = 3
    th0 = P.default_init(vol.n_vox, K, 0)
    rng = np.random.default_rng(1)
    thp = (th0 + rng.normal(0, 0.3, th0.shape)).astype(np.float32)
    f, ovs = make_pair([vol], [thp], K=K, patch_dim=8)
    gp = split_groups(f.groups(), f)[0]
    loss, yhat = f.forward(want_yhat=True)
    gth, _ = f.backward()
    torch.cuda.synchronize()
    yref, _ = O.predict(ovs[0], torch.as_tensor(thp).double(), gp)
    J, _, g, _ = O.value_and_grad(ovs[0], torch.as_tensor(thp).double(), gp)
    ey = signal_rel(yhat.cpu().numpy().reshape(vol.n_vox, -1), yref.numpy())
    eJ = abs(float(loss[0]) - float(J)) / abs(float(J))
    eg = _grad_errors(gth.cpu().numpy(), g.numpy(), K)
    f.set_params(torch.as_tensor(th0).cuda())
    f.step(200)
    f.sync()
    res = O.fit(ovs, [torch.as_tensor(th0).double()], 200)
    ddeg, peaks = _fit_compare(f.params_host(), res.theta[0].numpy(), K)
    f.close()
    _record("c1 crossing patch 8^3 N96 MSE", signal=ey, J=eJ, grad=eg, dir_median_deg=ddeg, peak_count_agree=peaks,
            iterations=200, voxels=vol.n_vox)
    assert ey <= TOL_SIGNAL and eJ <= TOL_LOSS and max(eg.values()) <= TOL_GRAD
    assert ddeg <= TOL_DIR_DEG and peaks == 1.0


@pytest.mark.parametrize("loss", ["mse", "nll"])
def test_crossing_sweep_accuracy(loss):
    """16 volumes of 10^3 (crossing angles 20-90 deg), N = 96, K = 3, sigma per volume for the
    NLL: every volume, 60 Adam iterations."""
    vols = P.crossing_sweep(0)
    K = 3
    inits = [P.default_init(v.n_vox, K, 10 + i) for i, v in enumerate(vols)]
    rng = np.random.default_rng(2)
    pert = [(t + rng.normal(0, 0.2, t.shape)).astype(np.float32) for t in inits]
    f, ovs = make_pair(vols, pert, K=K, loss=loss, patch_dim=10)
    packed = _perturb(f, rng, loss, False)
    gps = split_groups(packed, f)
    lossg, yhat = f.forward(want_yhat=True)
    gth, gg = f.backward()
    torch.cuda.synchronize()
    yhat, gth, gg = yhat.cpu().numpy(), gth.cpu().numpy(), gg.cpu().numpy()
    off = f.group_layout()
    ey = eJ = 0.0
    eg = {}
    pos = v0 = 0
    for gi, ov in enumerate(ovs):
        th = torch.as_tensor(pert[gi]).double()
        yref, _ = O.predict(ov, th, gps[gi])
        n = ov.n_vox * ov.n_meas
        ey = max(ey, signal_rel(yhat[pos:pos + n].reshape(ov.n_vox, ov.n_meas), yref.numpy()))
        pos += n
        J, _, g, ggr = O.value_and_grad(ov, th, gps[gi])
        eJ = max(eJ, abs(float(lossg[gi]) - float(J)) / abs(float(J)))
        e = _grad_errors(gth[v0:v0 + ov.n_vox], g.numpy(), K, gg, ggr, off[4 * gi:4 * gi + 4], ov.n_meas, loss)
        for k, v in e.items():
            eg[k] = max(eg.get(k, 0.0), v)
        v0 += ov.n_vox
    f.close()
    f, ovs = make_pair(vols, inits, K=K, loss=loss, patch_dim=10)
    f.step(60)
    f.sync()
    res = O.fit(ovs, [torch.as_tensor(t).double() for t in inits], 60)
    th = f.params_host()
    f.close()
    ddeg, peaks = _fit_compare(th, np.concatenate([t.numpy() for t in res.theta]), K)
    _record(f"c2 crossing sweep 16x10^3 N96 {loss.upper()}", signal=ey, J=eJ, grad=eg, dir_median_deg=ddeg,
            peak_count_agree=peaks, iterations=60, voxels=int(sum(v.n_vox for v in vols)))
    assert ey <= TOL_SIGNAL and eJ <= TOL_LOSS and max(eg.values()) <= TOL_GRAD
    assert ddeg <= TOL_DIR_DEG and peaks >= 0.99


def test_bundle_phantom_accuracy():
    """64^3 bundle phantom, N = 360, NLL + calibration + neighbour priors: y_hat and the voxel
    gradient on 4 sampled patches, J of the whole volume (patch chunks); the group gradients and
    a 40-iteration fit on the 24^3 phantom of the same kind (calibration couples the voxels)."""
    import paper_2604_00250_gb300 as prism
    vol = P.bundle_phantom(0, device="cpu")
    K = 3
    kw = dict(K=K, loss="nll", calibration=True, lam_sp=0.01, lam_dir=0.005, patch_dim=PATCH)
    rng = np.random.default_rng(3)
    th0 = (P.default_init(vol.n_vox, K, 7) + rng.normal(0, 0.2, (vol.n_vox, 4 * K + 5))).astype(np.float32)
    v = types.SimpleNamespace(mask=vol.mask, signal=torch.as_tensor(vol.signal).cuda(), bvals=vol.bvals,
                              bvecs=vol.bvecs, init=th0)
    f = prism.Fitter([v], prism.options(**kw))
    packed = _perturb(f, rng, "nll", True)
    gp = split_groups(packed, f)[0]
    lossg, yhat = f.forward(want_yhat=True)
    gth, _ = f.backward()
    torch.cuda.synchronize()
    N = vol.n_meas
    ids, _ = _patches(vol.mask, 4)
    o = oracle_opts(**kw)
    ov = O.OracleVolume(vol.mask, vol.signal, vol.bvals, vol.bvecs, o, patches=ids)
    sel = torch.as_tensor(ov.sel, device="cuda")
    ys = yhat.view(vol.n_vox, N)[sel].cpu().numpy()
    th = torch.as_tensor(th0[ov.sel]).double()
    yref, _ = O.predict(ov, th, gp)
    ey = signal_rel(ys, yref.numpy())
    _, _, g, _ = O.value_and_grad(ov, th, gp, n_norm=ov.n_mask)
    eg = _grad_errors(gth[sel].cpu().numpy(), g.numpy(), K)
    Jref = _chunked_objective(vol, o, th0, gp)
    eJ = abs(float(lossg[0]) - Jref) / abs(Jref)
    f.close()
    # group gradients and a fit on the 24^3 phantom
    small = P.bundle_phantom(1, edge=24, device="cpu")
    th1 = P.default_init(small.n_vox, K, 8)
    kw24 = dict(kw, patch_dim=8)
    f, ovs = make_pair([small], [th1], **kw24)
    packed = _perturb(f, rng, "nll", True)
    gp = split_groups(packed, f)[0]
    f.forward()
    _, gg = f.backward()
    torch.cuda.synchronize()
    _, _, _, ggr = O.value_and_grad(ovs[0], torch.as_tensor(th1).double(), gp)
    egg = _grad_errors(np.zeros((1, 4 * K + 5)), np.zeros((1, 4 * K + 5)), K, gg.cpu().numpy(), ggr,
                       f.group_layout()[:4], small.n_meas, "nll", True)
    egg = {k: v for k, v in egg.items() if k in ("sigma", "alpha", "beta", "blr")}
    f.close()
    f, ovs = make_pair([small], [th1], **kw24)
    f.step(40)
    f.sync()
    res = O.fit(ovs, [torch.as_tensor(th1).double()], 40)
    ddeg, peaks = _fit_compare(f.params_host(), res.theta[0].numpy(), K)
    f.close()
    eg.update(egg)
    _record("c3 bundle phantom 64^3 N360 NLL + calibration", signal=ey, J=eJ, grad=eg, dir_median_deg=ddeg,
            peak_count_agree=peaks, iterations=40, voxels=vol.n_vox,
            note="y_hat and voxel gradient on 4 sampled 16^3 patches; J of the whole volume; group gradients "
                 "and the fit on the 24^3 phantom of the same kind")
    assert ey <= TOL_SIGNAL and eJ <= TOL_LOSS and max(eg.values()) <= TOL_GRAD
    assert ddeg <= TOL_DIR_DEG and peaks >= 0.99


def test_brain_accuracy():
    """HCP-shaped brain, 740,110 voxels, N = 288, MSE + neighbour priors, the bench's launch
    configuration: y_hat and gradient on 4 sampled patches, J of the whole volume (patch chunks),
    and 100 iterations of 3 sampled patches (independent problems without calibration)."""
    import paper_2604_00250_gb300 as prism
    vol = P.brain_phantom(0, device="cpu")
    K = 3
    kw = dict(K=K, loss="mse", patch_dim=PATCH, lam_sp=0.01, lam_dir=0.005)
    v = types.SimpleNamespace(mask=vol.mask, signal=torch.as_tensor(vol.signal).cuda(), bvals=vol.bvals,
                              bvecs=vol.bvecs, init=None)
    f = prism.Fitter([v], prism.options(fused=1, use_graph=1, **kw))
    th0 = f.params_host()
    rng = np.random.default_rng(4)
    thp = (th0 + rng.normal(0, 0.2, th0.shape)).astype(np.float32)
    gp = split_groups(f.groups(), f)[0]
    lossg, yhat = f.forward(theta=torch.as_tensor(thp).cuda(), want_yhat=True)
    gth, _ = f.backward()
    torch.cuda.synchronize()
    N = vol.n_meas
    ids, _ = _patches(vol.mask, 4)
    o = oracle_opts(**kw)
    ov = O.OracleVolume(vol.mask, vol.signal, vol.bvals, vol.bvecs, o, patches=ids)
    sel = torch.as_tensor(ov.sel, device="cuda")
    ys = yhat.view(vol.n_vox, N)[sel].cpu().numpy()
    del yhat
    th = torch.as_tensor(thp[ov.sel]).double()
    yref, _ = O.predict(ov, th, gp)
    ey = signal_rel(ys, yref.numpy())
    _, _, g, _ = O.value_and_grad(ov, th, gp, n_norm=ov.n_mask)
    eg = _grad_errors(gth[sel].cpu().numpy(), g.numpy(), K)
    Jref = _chunked_objective(vol, o, thp, gp, chunk_patches=16)
    eJ = abs(float(lossg[0]) - Jref) / abs(Jref)
    # 100 iterations from the library's start; 3 sampled patches of the oracle's
    f.set_params(torch.as_tensor(th0).cuda())
    f.step(100)
    f.sync()
    thf = f.params_host()
    f.close()
    ids3, _ = _patches(vol.mask, 3, seed=1)
    ov3 = O.OracleVolume(vol.mask, vol.signal, vol.bvals, vol.bvecs, o, patches=ids3)
    adam = O.Adam(o)
    t = torch.as_tensor(th0[ov3.sel]).double()
    gp0 = O.group_init(ov3)
    for _ in range(100):
        adam.t += 1
        _, _, gr, _ = O.value_and_grad(ov3, t, gp0, n_norm=ov3.n_mask)
        t = adam.step("theta", t, gr)
    ddeg, peaks = _fit_compare(thf[ov3.sel], t.numpy(), K)
    _record("c4 HCP-shaped brain 740,110 voxels N288 MSE", signal=ey, J=eJ, grad=eg, dir_median_deg=ddeg,
            peak_count_agree=peaks, iterations=100, voxels=vol.n_vox,
            note="y_hat and gradient on 4 sampled 16^3 patches; J of the whole volume; the fit on 3 sampled "
                 "patches")
    assert ey <= TOL_SIGNAL and eJ <= TOL_LOSS and max(eg.values()) <= TOL_GRAD
    assert ddeg <= TOL_DIR_DEG and peaks >= 0.99


def test_multi_volume_batch_accuracy():
    """12 volumes of edge 32..128 (3.9 M voxels, N = 96/288/360), NLL + calibration + neighbour
    priors, one batch: per volume y_hat and the voxel gradient on 2 sampled patches; J of the 6
    smallest volumes in full (patch chunks); the fit on the 8-volume batch of edges 12..26."""
    import paper_2604_00250_gb300 as prism
    vols = P.multi_volume_batch(0)
    K = 3
    kw = dict(K=K, loss="nll", calibration=True, lam_sp=0.01, lam_dir=0.005, patch_dim=PATCH)
    rng = np.random.default_rng(5)
    inits = [(P.default_init(vv.n_vox, K, 20 + i) + rng.normal(0, 0.2, (vv.n_vox, 4 * K + 5))).astype(np.float32)
             for i, vv in enumerate(vols)]
    gv = [types.SimpleNamespace(mask=vv.mask, signal=torch.as_tensor(vv.signal).cuda(), bvals=vv.bvals,
                                bvecs=vv.bvecs, init=t) for vv, t in zip(vols, inits)]
    f = prism.Fitter(gv, prism.options(**kw))
    packed = _perturb(f, rng, "nll", True)
    gps = split_groups(packed, f)
    lossg, yhat = f.forward(want_yhat=True)
    gth, _ = f.backward()
    torch.cuda.synchronize()
    o = oracle_opts(**kw)
    per = []
    pos = v0 = 0
    order = np.argsort([vv.n_vox for vv in vols])
    full_J = set(int(i) for i in order[:6])
    for gi, vv in enumerate(vols):
        N = vv.n_meas
        ids, _ = _patches(vv.mask, 2, seed=gi)
        ov = O.OracleVolume(vv.mask, vv.signal, vv.bvals, vv.bvecs, o, patches=ids)
        sel = torch.as_tensor(ov.sel, device="cuda")
        ys = yhat[pos:pos + vv.n_vox * N].view(vv.n_vox, N)[sel].cpu().numpy()
        th = torch.as_tensor(inits[gi][ov.sel]).double()
        yref, _ = O.predict(ov, th, gps[gi])
        _, _, g, _ = O.value_and_grad(ov, th, gps[gi], n_norm=ov.n_mask)
        rec = {"volume": gi, "edge": int(vv.mask.shape[0]), "voxels": vv.n_vox, "n_meas": N,
               "signal": signal_rel(ys, yref.numpy()),
               "grad": _grad_errors(gth[v0:v0 + vv.n_vox][ov.sel.tolist()].cpu().numpy(), g.numpy(), K)}
        if gi in full_J:
            Jref = _chunked_objective(vv, o, inits[gi], gps[gi])
            rec["J"] = abs(float(lossg[gi]) - Jref) / abs(Jref)
        per.append(rec)
        pos += vv.n_vox * N
        v0 += vv.n_vox
    f.close()
    small = P.multi_volume_batch(0, edges=(12, 14, 16, 18, 20, 22, 24, 26))
    si = [P.default_init(vv.n_vox, K, 30 + i) for i, vv in enumerate(small)]
    f, ovs = make_pair(small, si, **dict(kw, patch_dim=8))
    f.step(30)
    f.sync()
    res = O.fit(ovs, [torch.as_tensor(t).double() for t in si], 30)
    ddeg, peaks = _fit_compare(f.params_host(), np.concatenate([t.numpy() for t in res.theta]), K)
    f.close()
    _record("c5 multi-volume batch 12 volumes NLL + calibration", per_volume=per, dir_median_deg=ddeg,
            peak_count_agree=peaks, iterations=30,
            note="per volume: y_hat and voxel gradient on 2 sampled 16^3 patches, J in full for the 6 smallest "
                 "volumes; the fit on the 8-volume batch of edges 12..26")
    for rec in per:
        assert rec["signal"] <= TOL_SIGNAL and max(rec["grad"].values()) <= TOL_GRAD, rec
        if "J" in rec:
            assert rec["J"] <= TOL_LOSS, rec
    assert ddeg <= TOL_DIR_DEG and peaks >= 0.99
