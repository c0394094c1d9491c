"""The launch-shape autotuner (prism_options.autotune): it times lanes per voxel (1, 4, 16)
and, where it applies, the shell loop against the per-measurement loop, and must pick a shape
whose fused kernel is within 5 % of the fastest shape forced by hand; a fit with the tuned shape
must still follow the oracle: its first-step gradient (Adam's first moment, every voxel and
group block) normwise, and the objective over three iterations. Above about 311k voxels the
candidates are timed on a bounded sample of whole patches (the brain exercises that path)."""
import types

import numpy as np
import pytest
import torch

import phantoms as P
from oracle import prism_oracle as O
from tests.helpers import TOL_GRAD, block_slices, inits_for, make_pair, normwise, split_groups
from tests.test_gpu_fused_gradient import fused_gradient

pytestmark = pytest.mark.gpu


def _fused_ms(vol_ns, kw, **force):
    import paper_2604_00250_gb300 as prism
    f = prism.Fitter([vol_ns], prism.options(**kw, **force))
    f.step(3)
    ms = min(f.profile(10)["fused_ms"] for _ in range(3))
    shape = f.shape()
    f.close()
    return ms, shape


def _forced(vol_ns, kw):
    out = []
    for tpv in (1, 4, 16):
        for shells in ((0, -1) if tpv == 1 else (0,)):
            ms, shape = _fused_ms(vol_ns, kw, threads_per_voxel=tpv, shells=shells)
            out.append((ms, shape["threads_per_voxel"], shape["shell_loop"]))
    return out


@pytest.mark.parametrize("case", ["mse_shells", "nll_calibrated"])
def test_autotune_picks_a_shape_near_the_fastest(case):
    if case == "mse_shells":
        vol = P.bundle_phantom(0, edge=40, scheme=P.scheme_288(0), device="cpu")
        kw = dict(K=3, loss="mse", patch_dim=16, lam_sp=0.01, lam_dir=0.005)
    else:
        vol = P.bundle_phantom(0, edge=40, device="cpu")
        kw = dict(K=3, loss="nll", calibration=True, patch_dim=16, lam_sp=0.01, lam_dir=0.005)
    v = types.SimpleNamespace(mask=vol.mask, signal=torch.as_tensor(vol.signal).cuda(), bvals=vol.bvals,
                              bvecs=vol.bvecs, init=None)
    forced = _forced(v, kw)
    best = min(m for m, _, _ in forced)
    tuned_ms, shape = _fused_ms(v, kw, autotune=1)
    assert tuned_ms <= 1.05 * best, (tuned_ms, shape, forced)
    # the tuned shape still follows the oracle: the first step's gradient, then three iterations
    K = 3
    init = inits_for([vol], K, 3)
    f, ovs = make_pair([vol], init, autotune=1, **kw)
    assert (f.shape()["threads_per_voxel"], f.shape()["shell_loop"]) == (shape["threads_per_voxel"],
                                                                        shape["shell_loop"])
    gp = split_groups(f.groups(), f)[0]
    f.step(1)
    f.sync()
    g_vox, g_grp = fused_gradient(f, f.opts.beta1)
    _, _, g, ggr = O.value_and_grad(ovs[0], torch.as_tensor(init[0]).double(), gp)
    for name, sl in block_slices(K).items():
        e = normwise(g_vox[:, sl], g[:, sl].numpy())
        assert e <= TOL_GRAD, (name, e)
    a, b, c, d = (int(x) for x in f.group_layout()[0:4])
    N = ovs[0].n_meas
    if kw["loss"] == "nll":
        assert normwise([g_grp[a]], [float(ggr["sigma_log"])]) <= TOL_GRAD
    if kw.get("calibration"):
        assert normwise(g_grp[b:b + N], ggr["alpha"].numpy()) <= TOL_GRAD
        assert normwise(g_grp[c:c + N], ggr["beta"].numpy()) <= TOL_GRAD
        assert normwise(g_grp[d:d + 512], ggr["blr"].numpy().ravel()) <= TOL_GRAD
    f.step(2)
    f.sync()
    res = O.fit(ovs, [torch.as_tensor(t).double() for t in init], 3)
    np.testing.assert_allclose(f.loss_history(), res.loss_history, rtol=1e-5)
    f.close()


def test_autotune_on_a_bounded_sample_of_the_brain():
    """740,110 voxels: the candidates are timed on about 311k voxels of the fullest patches."""
    vol = P.brain_phantom(0, device="cpu")
    kw = dict(K=3, loss="mse", patch_dim=16, lam_sp=0.01, lam_dir=0.005)
    v = types.SimpleNamespace(mask=vol.mask, signal=torch.as_tensor(vol.signal).cuda(), bvals=vol.bvals,
                              bvecs=vol.bvecs, init=None)
    forced = [(_fused_ms(v, kw, threads_per_voxel=t, shells=s)[0], t, s) for t, s in ((1, 0), (1, -1), (4, 0))]
    best = min(m for m, _, _ in forced)
    tuned_ms, shape = _fused_ms(v, kw, autotune=1)
    assert tuned_ms <= 1.05 * best, (tuned_ms, shape, forced)
