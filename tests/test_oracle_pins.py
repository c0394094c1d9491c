"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-runs the oracle's own formula as its expectation: each checks
a closed form, a special case that reduces to a library routine, an invariant,
a value printed in the paper, or brute-force finite differences.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import phantoms as P
from oracle import metrics as M
from oracle import prism_oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
F64 = torch.float64


def _vol(mask, signal, bvals, bvecs, **kw):
    o = O.Options(**kw)
    return O.OracleVolume(mask, signal, bvals, bvecs, o)


def _line_scheme(b, angles_deg):
    """b=0 first, then gradient directions in the x-y plane at the given angles to x."""
    a = np.radians(np.asarray(angles_deg, dtype=np.float64))
    g = np.stack([np.cos(a), np.sin(a), np.zeros_like(a)], 1)
    bv = np.concatenate([[0.0], np.full(len(a), float(b))])
    gv = np.concatenate([np.zeros((1, 3)), g])
    return bv, gv


def test_paper_constants():
    """Diffusivities, prior weights and the Huber delta are the printed ones."""
    gold = json.load(open(os.path.join(GOLD, "paper_constants.json")))
    assert O.D_CSF == gold["D_csf"]["value"]
    assert O.D_GM == gold["D_gm"]["value"]
    assert O.D_RES == gold["D_res"]["value"]
    assert O.D_PAR == gold["D_par"]["value"]
    assert O.D_PERP == gold["D_perp"]["value"]
    o = O.Options()
    assert o.huber_delta == gold["huber_delta"]["value"]
    assert o.lam_rep == gold["lambda_rep"]["value"]
    assert o.lam_sparse == gold["lambda_sparse"]["value"]
    assert o.tau == gold["tau"]["value"]
    assert o.lr == gold["adam_lr"]["value"]
    # f_intra raw init 0 -> sigmoid(0) = 0.5 (Sec. 2.2)
    th = P.default_init(3, 2, 0)
    assert np.all(th[:, -1] == 0.0)
    assert abs(1.0 / (1.0 + math.exp(-float(th[0, -1]))) - gold["f_intra_init"]["value"]) == 0


def _single_fiber_theta(V, K, vraw, u_in, s0=1.0):
    Q = O.n_params(K)
    th = torch.zeros(V, Q, dtype=F64)
    th[:, 0] = math.log(math.expm1(s0))
    th[:, 1:K + 4] = -60.0
    th[:, 3] = 0.0                          # wm_1 logit
    th[:, K + 4:K + 7] = torch.as_tensor(vraw, dtype=F64)
    for k in range(1, K):
        th[:, K + 4 + 3 * k:K + 7 + 3 * k] = torch.tensor([0.0, 0.0, 1.0], dtype=F64)
    th[:, 4 * K + 4] = u_in
    return th


@pytest.mark.parametrize("K", [1, 3])
def test_single_stick_closed_form(K):
    """f_wm=1, f_intra=1, S0=1, no calibration => y_hat = exp(-b D_par cos^2) (Eq. 5)."""
    angles = [0.0, 30.0, 45.0, 60.0, 90.0]
    bv, gv = _line_scheme(1000.0, angles)
    mask = np.ones((1, 1, 1), np.uint8)
    sig = np.ones((1, len(bv)), np.float32)
    ov = _vol(mask, sig, bv, gv, K=K, lam_rep=0, lam_sparse=0)
    th = _single_fiber_theta(1, K, [0.3, 0.0, 0.0], 60.0)   # raw direction not unit
    yhat, _ = O.predict(ov, th, O.group_init(ov))
    # hand values: exp(-1000 * 1.7e-3 * cos^2)
    want = [1.0, math.exp(-1.7), math.exp(-1.7 * 0.75), math.exp(-0.85), math.exp(-1.7 * 0.25), 1.0]
    got = yhat[0].numpy()
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-15)
    assert abs(got[2] - 0.2794310) < 1e-6        # exp(-1.275), computed by hand


def test_highest_shell_closed_forms():
    """At the highest b of the DiSCo1 scheme (13,192 s/mm^2, Sec. 3 "Datasets") the stick and
    the zeppelin still follow Eq. 5 in FP64 down to their smallest values: stick exp(-b D_par
    cos^2) at 0 / 45 / 90 deg, zeppelin exp(-b (D_par cos^2 + D_perp sin^2)) at 45 and 90 deg."""
    bv, gv = _line_scheme(13192.0, [0.0, 45.0, 90.0])
    mask = np.ones((1, 1, 1), np.uint8)
    ov = _vol(mask, np.ones((1, len(bv)), np.float32), bv, gv, K=1, lam_rep=0, lam_sparse=0)
    stick, _ = O.predict(ov, _single_fiber_theta(1, 1, [1.0, 0.0, 0.0], 60.0), O.group_init(ov))
    zep, _ = O.predict(ov, _single_fiber_theta(1, 1, [1.0, 0.0, 0.0], -60.0), O.group_init(ov))
    # hand values: b D_par = 22.4264, b D_perp = 5.2768
    np.testing.assert_allclose(stick[0].numpy()[1:], [1.8211186041263214e-10, 1.3494882749125023e-05, 1.0],
                               rtol=1e-12)
    np.testing.assert_allclose(zep[0].numpy()[2:], [9.645540179499184e-07, 0.005108752672315215], rtol=1e-12)


def test_zeppelin_only_closed_form():
    """f_intra = 0: E = exp(-b (D_par cos^2 + D_perp sin^2)); at 90 deg exp(-b D_perp)."""
    bv, gv = _line_scheme(2000.0, [90.0, 0.0])
    mask = np.ones((1, 1, 1), np.uint8)
    ov = _vol(mask, np.ones((1, 3), np.float32), bv, gv, K=1)
    th = _single_fiber_theta(1, 1, [1.0, 0.0, 0.0], -60.0)
    yhat, _ = O.predict(ov, th, O.group_init(ov))
    np.testing.assert_allclose(yhat[0].numpy(), [1.0, math.exp(-0.8), math.exp(-3.4)], rtol=1e-14)


def test_isotropic_closed_form():
    """All fraction in one isotropic pool gives exp(-b D) of that pool (Eq. 4)."""
    bv, gv = _line_scheme(1500.0, [10.0])
    mask = np.ones((1, 1, 1), np.uint8)
    ov = _vol(mask, np.ones((1, 2), np.float32), bv, gv, K=2)
    for pool, D in [(1, 3.0e-3), (2, 0.9e-3), (2 + 2 + 1, 0.2e-3)]:
        th = torch.zeros(1, O.n_params(2), dtype=F64)
        th[:, 0] = math.log(math.expm1(2.5))
        th[:, 1:6] = -60.0
        th[:, pool] = 0.0
        th[:, 6:12] = 1.0
        yhat, _ = O.predict(ov, th, O.group_init(ov))
        np.testing.assert_allclose(yhat[0].numpy(), [2.5, 2.5 * math.exp(-1500.0 * D)], rtol=1e-14)


def test_b0_gives_s0():
    """At b = 0 every compartment is 1 and softmax sums to 1: y_hat = S0 = softplus(s)."""
    rng = np.random.default_rng(1)
    K = 3
    bv = np.array([0.0, 0.0, 1000.0, 3000.0])
    gv = np.array([[0, 0, 0], [0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.float64)
    mask = np.ones((2, 3, 1), np.uint8)
    ov = _vol(mask, np.ones((6, 4), np.float32), bv, gv, K=K)
    th = torch.as_tensor(rng.normal(0, 2, size=(6, O.n_params(K))))
    th[0, 0] = 40.0                              # large s: softplus(s) ~ s
    th[1, 0] = -30.0                             # tiny S0
    yhat, _ = O.predict(ov, th, O.group_init(ov))
    want = np.array([math.log1p(math.exp(s)) for s in th[:, 0].tolist()])
    np.testing.assert_allclose(yhat[:, 0].numpy(), want, rtol=1e-14)
    np.testing.assert_allclose(yhat[:, 1].numpy(), want, rtol=1e-14)


def test_trilinear_matches_interpolate():
    """upsample(b_lr) equals torch's trilinear interpolation, align_corners=False."""
    rng = np.random.default_rng(2)
    grid = torch.as_tensor(rng.normal(size=(8, 8, 8)))
    shape = (13, 7, 20)
    ref = F.interpolate(grid[None, None], size=shape, mode="trilinear", align_corners=False)[0, 0]
    coords = np.argwhere(np.ones(shape, bool))
    got = O.bias_log(grid, coords, shape)
    np.testing.assert_allclose(got.numpy(), ref.reshape(-1).numpy(), rtol=1e-12, atol=1e-14)


def test_calibration_identity_and_constant_bias():
    """alpha = beta = b_lr = 0 => y_hat = S; constant b_lr = c => y_hat = e^c S (Sec. 2.3)."""
    vol = P.random_volume((3, 3, 3), seed=3)
    ov = _vol(vol.mask, vol.signal, vol.bvals, vol.bvecs, K=3, calibration=True)
    th = torch.as_tensor(P.default_init(ov.n_vox, 3, 3)).double()
    gp = O.group_init(ov)
    yhat, S = O.predict(ov, th, gp)
    np.testing.assert_array_equal(yhat.numpy(), S.numpy())
    gp["blr"] = torch.full((8, 8, 8), 0.3, dtype=F64)
    gp["alpha"] = torch.full((ov.n_meas,), -0.2, dtype=F64)
    gp["beta"] = torch.full((ov.n_meas,), 0.05, dtype=F64)
    yhat, S = O.predict(ov, th, gp)
    np.testing.assert_allclose(yhat.numpy(), math.exp(0.1) * S.numpy() + 0.05, rtol=1e-13)


def _rotation(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


@pytest.mark.parametrize("loss", ["mse", "nll"])
def test_joint_rotation_invariance(loss):
    """Rotating all fiber directions and b-vectors together leaves y_hat, J and the
    priors unchanged, and rotates dJ/dv with them."""
    rng = np.random.default_rng(4)
    vol = P.random_volume((3, 3, 2), seed=4)
    K = 3
    kw = dict(K=K, loss=loss, lam_sp=0.01, lam_dir=0.005, patch_dim=2)
    ov = _vol(vol.mask, vol.signal, vol.bvals, vol.bvecs, **kw)
    R = _rotation(rng)
    ov_r = _vol(vol.mask, vol.signal, vol.bvals, (vol.bvecs.astype(np.float64) @ R.T), **kw)
    th = torch.as_tensor(rng.normal(0, 1, size=(ov.n_vox, O.n_params(K))))
    th_r = th.clone()
    v = th[:, K + 4:4 * K + 4].reshape(-1, K, 3)
    th_r[:, K + 4:4 * K + 4] = (v @ torch.as_tensor(R).T).reshape(-1, 3 * K)
    gp = O.group_init(ov)
    gp["sigma_log"] = torch.tensor(math.log(0.04), dtype=F64)
    J, parts, g, _ = O.value_and_grad(ov, th, gp)
    Jr, parts_r, gr, _ = O.value_and_grad(ov_r, th_r, gp)
    assert abs(float(J - Jr)) <= 1e-12 * abs(float(J))
    for k in parts:
        assert abs(float(parts[k] - parts_r[k])) <= 1e-12 * max(1.0, abs(float(parts[k])))
    gv = g[:, K + 4:4 * K + 4].reshape(-1, K, 3)
    gvr = gr[:, K + 4:4 * K + 4].reshape(-1, K, 3)
    np.testing.assert_allclose((gv @ torch.as_tensor(R).T).numpy(), gvr.numpy(), rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(g[:, :K + 4].numpy(), gr[:, :K + 4].numpy(), rtol=1e-9, atol=1e-12)


def test_noiseless_ground_truth_is_stationary():
    """Data made by the (independent) phantom simulator with the fit model's own
    diffusivities: theta = ground truth reproduces it and dL_MSE/dtheta = 0."""
    rng = np.random.default_rng(5)
    K = 2
    V = 27
    bvals, bvecs = P.scheme_96(5)
    d1 = rng.normal(size=(V, 3)); d1 /= np.linalg.norm(d1, axis=1, keepdims=True)
    d2 = rng.normal(size=(V, 3)); d2 /= np.linalg.norm(d2, axis=1, keepdims=True)
    fr = rng.dirichlet([2, 2, 1, 1, 1], size=V)
    fin = rng.uniform(0.3, 0.7, V)
    s0 = np.ones(V)
    clean = P.volumes._simulate(bvals, bvecs, np.stack([d1, d2], 1), fr[:, :2], fr[:, 2:],
                                np.full(V, O.D_PAR), np.full(V, O.D_PERP), fin, s0)
    mask = np.ones((3, 3, 3), np.uint8)
    ov = O.OracleVolume(mask, clean, bvals, bvecs, O.Options(K=K, lam_rep=0, lam_sparse=0))
    ov.y = torch.as_tensor(clean)                 # keep float64 exactly (b0 mean is 1)
    th = torch.zeros(V, O.n_params(K), dtype=F64)
    th[:, 0] = math.log(math.expm1(1.0))
    # logits [csf, gm, wm1, wm2, res] = log fractions
    th[:, 1] = torch.as_tensor(np.log(fr[:, 2]))
    th[:, 2] = torch.as_tensor(np.log(fr[:, 3]))
    th[:, 3] = torch.as_tensor(np.log(fr[:, 0]))
    th[:, 4] = torch.as_tensor(np.log(fr[:, 1]))
    th[:, 5] = torch.as_tensor(np.log(fr[:, 4]))
    th[:, 6:9] = torch.as_tensor(d1 * 2.0)
    th[:, 9:12] = torch.as_tensor(-d2)
    th[:, 12] = torch.as_tensor(np.log(fin / (1 - fin)))
    yhat, _ = O.predict(ov, th, O.group_init(ov))
    np.testing.assert_allclose(yhat.numpy(), clean, rtol=1e-13, atol=1e-15)
    J, _, g, _ = O.value_and_grad(ov, th, O.group_init(ov))
    assert float(J) < 1e-26
    assert float(g.abs().max()) < 1e-14


def test_log_i0_against_scipy_and_series():
    sp = pytest.importorskip("scipy.special")
    z = np.logspace(-6, 4, 400)
    got = O.log_i0(torch.as_tensor(z)).numpy()
    ref = np.log(sp.i0e(z)) + z
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-15)
    # small z: log I0(z) = z^2/4 - z^4/64 + O(z^6)
    zs = np.array([1e-3, 1e-2])
    np.testing.assert_allclose(O.log_i0(torch.as_tensor(zs)).numpy(), zs ** 2 / 4 - zs ** 4 / 64,
                               rtol=1e-9)
    # large z (A&S 9.7.1): I0(z) ~ e^z / sqrt(2 pi z) (1 + 1/(8z) + 9/(128 z^2) + 225/(3072 z^3));
    # the first omitted term, 11025/(98304 z^4), bounds the difference
    zl = np.array([200.0, 2000.0])
    asym = zl - 0.5 * np.log(2 * np.pi * zl) + np.log1p(1 / (8 * zl) + 9 / (128 * zl ** 2)
                                                      + 225 / (3072 * zl ** 3))
    np.testing.assert_allclose(O.log_i0(torch.as_tensor(zl)).numpy(), asym, rtol=0,
                               atol=2 * 11025 / (98304 * 200.0 ** 4) + 1e-12)


def test_rician_tends_to_gaussian():
    """High SNR: NLL -> log s^2 + (y - yh)^2 / 2s^2 + 1/2 log(2 pi y yh / s^2), and
    s^2 dNLL/dyh -> (yh - y) + s^2 / (2 yh)."""
    bv, gv = _line_scheme(1000.0, [0.0, 40.0, 80.0])
    mask = np.ones((1, 1, 1), np.uint8)
    sig = np.array([[1.0, 0.3, 0.5, 0.8]], np.float32)
    ov = _vol(mask, sig, bv, gv, K=1, loss="nll", lam_rep=0, lam_sparse=0)
    th = _single_fiber_theta(1, 1, [1.0, 0.0, 0.0], 0.0)
    for s in [1e-2, 1e-3]:
        gp = O.group_init(ov)
        gp["sigma_log"] = torch.tensor(math.log(s), dtype=F64)
        yhat, _ = O.predict(ov, th, gp)
        y = ov.y
        J, parts, _, _ = O.value_and_grad(ov, th, gp)
        gauss = (math.log(s * s) + (y - yhat) ** 2 / (2 * s * s)
                 + 0.5 * torch.log(2 * math.pi * y * yhat / (s * s))).sum()
        zmin = float((y * yhat).min()) / (s * s)
        assert abs(float(parts["data"] - gauss)) < 4 * 0.125 / zmin
        yh = yhat.detach().clone().requires_grad_(True)
        l = (2 * gp["sigma_log"] + (y * y + yh * yh) / (2 * s * s) - O.log_i0(y * yh / (s * s))).sum()
        (gy,) = torch.autograd.grad(l, yh)
        lhs = (s * s * gy - (yh - y)).detach()
        np.testing.assert_allclose(lhs.numpy(), (s * s / (2 * yhat)).numpy(), rtol=0.2)


def test_huber_matches_library():
    r = torch.linspace(-0.2, 0.2, 401, dtype=F64)
    np.testing.assert_allclose(O.huber(r, 0.05).numpy(),
                               F.huber_loss(r, torch.zeros_like(r), reduction="none", delta=0.05).numpy(),
                               rtol=1e-15, atol=1e-18)


def _frac_theta(V, K, wm_logits, iso_logit=-60.0, dirs=None):
    th = torch.zeros(V, O.n_params(K), dtype=F64)
    th[:, 0] = math.log(math.expm1(1.0))
    th[:, 1] = iso_logit
    th[:, 2] = iso_logit
    th[:, K + 3] = iso_logit
    th[:, 3:K + 3] = torch.as_tensor(wm_logits, dtype=F64)
    if dirs is not None:
        th[:, K + 4:4 * K + 4] = torch.as_tensor(np.asarray(dirs, dtype=np.float64).reshape(V, 3 * K))
    return th


def _prior_parts(mask, th, K, **kw):
    N = 2
    bv, gv = _line_scheme(1000.0, [0.0])
    sig = np.ones((int(mask.sum()), N), np.float32)
    ov = _vol(mask, sig, bv, gv, K=K, **kw)
    _, parts = O.objective(ov, th, O.group_init(ov))
    return parts


def test_repulsion_hand_value():
    """R_rep = sum_{i<j} f_i f_j |d_i . d_j| (Sec. 2.4): f = .5/.5 at 60 deg -> .125."""
    mask = np.ones((1, 1, 1), np.uint8)
    d = [[1, 0, 0], [-0.5, math.sqrt(3) / 2, 0]]
    th = _frac_theta(1, 2, [0.0, 0.0], dirs=[d])
    parts = _prior_parts(mask, th, 2, lam_rep=0.01, lam_sparse=0)
    assert abs(float(parts["rep"]) - 0.01 * 0.125) < 1e-15
    # three orthogonal fibers repel nothing
    th = _frac_theta(1, 3, [0.0, 0.0, 0.0], dirs=[[[1, 0, 0], [0, 1, 0], [0, 0, 1]]])
    assert abs(float(_prior_parts(mask, th, 3, lam_rep=0.01, lam_sparse=0)["rep"])) < 1e-18


def test_sparsity_hand_value():
    """L1 on minor fiber fractions below tau = 0.15 (reading R15)."""
    mask = np.ones((1, 1, 1), np.uint8)
    # wm fractions 0.8, 0.1, 0.1 (iso pools ~0)
    lg = [math.log(0.8), math.log(0.1), math.log(0.1)]
    th = _frac_theta(1, 3, lg, dirs=[[[1, 0, 0], [0, 1, 0], [0, 0, 1]]])
    parts = _prior_parts(mask, th, 3, lam_rep=0, lam_sparse=0.02)
    assert abs(float(parts["sparse"]) - 0.02 * 0.2) < 1e-14


def test_spatial_prior_hand_values():
    """Eq. 7 on a 3-voxel line: constant fractions give 0; one bump gives the Huber value."""
    mask = np.ones((3, 1, 1), np.uint8)
    K = 1
    th = _frac_theta(3, K, [0.0], iso_logit=0.0, dirs=[[1, 0, 0]] * 3)
    parts = _prior_parts(mask, th, K, lam_rep=0, lam_sparse=0, lam_sp=0.01, patch_dim=4)
    assert abs(float(parts["spatial"])) < 1e-20
    # middle voxel all-wm, ends all-csf (K=1: pools csf, gm, wm, res)
    th = torch.zeros(3, O.n_params(K), dtype=F64)
    th[:, 1:5] = -60.0
    th[0, 1] = 0.0
    th[2, 1] = 0.0
    th[1, 3] = 0.0
    th[:, 5:8] = torch.tensor([1.0, 0, 0], dtype=F64)
    parts = _prior_parts(mask, th, K, lam_rep=0, lam_sparse=0, lam_sp=0.01, patch_dim=4)
    # residuals: end voxels r = e_csf - e_wm (|N|=1): csf +1, wm -1 -> two Huber(1) each;
    # middle r = e_wm - e_csf: same. Huber(1) = 0.05 * (1 - 0.025) = 0.04875.
    want = 0.01 / 3 * (6 * 0.04875)
    assert abs(float(parts["spatial"]) - want) < 1e-15
    # neighbours in another patch do not count (reading R13)
    parts = _prior_parts(mask, th, K, lam_rep=0, lam_sparse=0, lam_sp=0.01, patch_dim=1)
    assert abs(float(parts["spatial"])) < 1e-20


def test_direction_continuity_hand_values():
    """Identical or antipodal neighbour directions cost 0; orthogonal ones cost 1 per fiber."""
    mask = np.ones((2, 1, 1), np.uint8)
    K = 2
    d_a = [[1, 0, 0], [0, 1, 0]]
    d_b = [[-1, 0, 0], [0, 2, 0]]
    th = _frac_theta(2, K, [0.0, 0.0], dirs=[d_a, d_b])
    parts = _prior_parts(mask, th, K, lam_rep=0, lam_sparse=0, lam_dir=0.005, patch_dim=4)
    assert abs(float(parts["dir"])) < 1e-18
    d_c = [[0, 0, 1], [1, 0, 0]]
    th = _frac_theta(2, K, [0.0, 0.0], dirs=[d_a, d_c])
    parts = _prior_parts(mask, th, K, lam_rep=0, lam_sparse=0, lam_dir=0.005, patch_dim=4)
    assert abs(float(parts["dir"]) - 0.005 * (2 * 2) / 2) < 1e-15


def test_b0_normalisation_is_scale_free():
    vol = P.random_volume((2, 2, 2), seed=6)
    ov1 = _vol(vol.mask, vol.signal, vol.bvals, vol.bvecs)
    scale = np.linspace(0.5, 3.0, vol.n_vox)[:, None]
    ov2 = _vol(vol.mask, vol.signal * scale, vol.bvals, vol.bvecs)
    np.testing.assert_allclose(ov1.y.numpy(), ov2.y.numpy(), rtol=1e-6)
    assert np.allclose(ov1.y.numpy()[:, vol.bvals <= 50].mean(1), 1.0)


def test_sigma_init_pooled_b0():
    """Pooled std of normalised b=0 repeats recovers the Rician sigma at SNR 30."""
    vol = P.crossing_patch(0)
    ov = _vol(vol.mask, vol.signal, vol.bvals, vol.bvecs)
    assert abs(ov.sigma0 - 1 / 30.0) < 0.1 / 30.0


def test_adam_matches_torch_optim():
    """Adam equals torch.optim.Adam on float64, and its first step is lr * sign(g)."""
    rng = np.random.default_rng(7)
    o = O.Options()
    p0 = torch.as_tensor(rng.normal(size=20))
    ours = O.Adam(o)
    p = p0.clone()
    ref = p0.clone().requires_grad_(True)
    opt = torch.optim.Adam([ref], lr=o.lr, betas=(o.beta1, o.beta2), eps=o.eps)
    for it in range(6):
        g = torch.as_tensor(rng.normal(size=20)) * 10 ** (it - 3)
        ours.t += 1
        p_new = ours.step("p", p, g)
        if it == 0:
            np.testing.assert_allclose((p - p_new).numpy(),
                                       (o.lr * g / (g.abs() + o.eps)).numpy(), rtol=1e-12)
        p = p_new
        opt.zero_grad()
        ref.grad = g.clone()
        opt.step()
        np.testing.assert_allclose(p.numpy(), ref.detach().numpy(), rtol=1e-13, atol=1e-15)


def _fd_check(ov, th, gp, rng, n_checks=40, h=1e-6):
    J, _, g, gg = O.value_and_grad(ov, th, gp)

    def Jof(t, q):
        return float(O.objective(ov, t, q)[0])

    V, Q = th.shape
    picks = [(int(rng.integers(V)), int(rng.integers(Q))) for _ in range(n_checks)]
    for v, q in picks:
        tp = th.clone(); tp[v, q] += h
        tm = th.clone(); tm[v, q] -= h
        fd = (Jof(tp, gp) - Jof(tm, gp)) / (2 * h)
        assert abs(fd - float(g[v, q])) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (v, q, fd, float(g[v, q]))
    for name, gk in gg.items():
        flat = gp[name].reshape(-1)
        for i in rng.choice(flat.numel(), size=min(6, flat.numel()), replace=False):
            qp = {k: x.clone() for k, x in gp.items()}
            qm = {k: x.clone() for k, x in gp.items()}
            qp[name].view(-1)[i] += h
            qm[name].view(-1)[i] -= h
            fd = (Jof(th, qp) - Jof(th, qm)) / (2 * h)
            an = float(gk.reshape(-1)[i])
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (name, i, fd, an)


@pytest.mark.parametrize("loss,cal,K", [("mse", False, 2), ("mse", True, 3), ("nll", True, 3),
                                        ("nll", False, 2)])
def test_gradient_central_differences(loss, cal, K):
    """Autograd gradient of the full objective vs central differences (FP64)."""
    rng = np.random.default_rng(8)
    bv, gv = P.make_scheme(2, [(1000, 5), (2500, 5)], 8)
    vol = P.random_volume((2, 2, 2), scheme=(bv, gv), seed=8, calibration=cal)
    kw = dict(K=K, loss=loss, calibration=cal, lam_sp=0.01, lam_dir=0.005, patch_dim=2,
              tau=0.15, lam_orphan=0.01, lam_order=0.01, connectivity=26 if cal else 6)
    ov = _vol(vol.mask, vol.signal, vol.bvals, vol.bvecs, **kw)
    # keep every WM fraction away from the sparsity gate (a jump) by >> h
    while True:
        th = torch.as_tensor(rng.normal(0, 0.7, size=(ov.n_vox, O.n_params(K))))
        _, fr, _, _ = O.transforms(th, K)
        fw = fr[:, 2:K + 2]
        if float((fw - 0.15).abs().min()) > 1e-3 and (K < 2 or float((fw[:, 1:] - fw[:, :-1]).abs().min()) > 1e-3):
            break
    gp = O.group_init(ov)
    gp["sigma_log"] = torch.tensor(math.log(0.06), dtype=F64)
    if cal:
        gp["alpha"] = torch.as_tensor(rng.normal(0, 0.05, ov.n_meas))
        gp["beta"] = torch.as_tensor(rng.normal(0, 0.02, ov.n_meas))
        gp["blr"] = torch.as_tensor(rng.normal(0, 0.1, (8, 8, 8)))
    _fd_check(ov, th, gp, rng)


def test_metrics_permutation_and_sign_free():
    rng = np.random.default_rng(9)
    K = 3
    th = rng.normal(size=(50, O.n_params(K)))
    th2 = th.copy()
    perm = [2, 0, 1]
    v = th[:, K + 4:4 * K + 4].reshape(-1, K, 3)
    th2[:, K + 4:4 * K + 4] = (-v[:, perm]).reshape(-1, 3 * K)
    lg = th[:, 3:K + 3]
    th2[:, 3:K + 3] = lg[:, perm]
    dev, pa, pb = M.matched_deviation(th, th2, K)
    assert dev.max() < 1e-5          # arccos(1 - ulp) ~ 1e-6 deg
    np.testing.assert_array_equal(pa, pb)


def test_planted_mistakes_are_caught(monkeypatch):
    """Swapping the two fiber diffusivities, or dropping the restricted pool, breaks a pin."""
    monkeypatch.setattr(O, "D_PAR", 0.4e-3)
    with pytest.raises(AssertionError):
        test_single_stick_closed_form(1)
    monkeypatch.setattr(O, "D_PAR", 1.7e-3)
    monkeypatch.setattr(O, "D_RES", 0.0)
    with pytest.raises(AssertionError):
        test_isotropic_closed_form()


def test_rprop_matches_torch_optim():
    """Rprop equals torch.optim.Rprop (float64) over steps with sign changes, and its first
    step is -lr * sign(g)."""
    rng = np.random.default_rng(12)
    o = O.Options(lr=0.01)
    p0 = torch.as_tensor(rng.normal(size=30))
    ours = O.Rprop(o)
    p = p0.clone()
    ref = p0.clone().requires_grad_(True)
    opt = torch.optim.Rprop([ref], lr=o.lr, etas=(0.5, 1.2), step_sizes=(1e-6, 50.0))
    signs = rng.choice([-1.0, 1.0], size=(8, 30))
    signs[:, :5] = 1.0                     # these keep their sign: steps grow by 1.2 each time
    for it in range(8):
        g = torch.as_tensor(signs[it] * rng.uniform(0.1, 2.0, 30))
        p_new = ours.step("p", p, g)
        if it == 0:
            np.testing.assert_allclose((p - p_new).numpy(), (o.lr * torch.sign(g)).numpy(), rtol=0, atol=1e-15)
        p = p_new
        opt.zero_grad()
        ref.grad = g.clone()
        opt.step()
        np.testing.assert_allclose(p.numpy(), ref.detach().numpy(), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(ours.state["p"][1][:5].numpy(), o.lr * 1.2 ** 7, rtol=1e-13)


def test_orphan_and_ordering_hand_values():
    """R25: exp(-S0 / 0.05) sum_k f_wm (S0 = 0.05 -> e^-1); R26: hinge on ascending fractions."""
    mask = np.ones((1, 1, 1), np.uint8)
    K = 3
    # wm fractions 0.2, 0.5, 0.3 (iso pools ~0): ordering violations 0.5-0.2 = 0.3
    lg = [math.log(0.2), math.log(0.5), math.log(0.3)]
    th = _frac_theta(1, K, lg, dirs=[[[1, 0, 0], [0, 1, 0], [0, 0, 1]]])
    th[:, 0] = math.log(math.expm1(0.05))          # S0 = 0.05
    parts = _prior_parts(mask, th, K, lam_rep=0, lam_sparse=0, lam_orphan=0.01, lam_order=0.01)
    assert abs(float(parts["orphan"]) - 0.01 * math.exp(-1.0) * 1.0) < 1e-14
    assert abs(float(parts["order"]) - 0.01 * 0.3) < 1e-14
    # descending fractions: no ordering cost
    th2 = _frac_theta(1, K, [math.log(0.5), math.log(0.3), math.log(0.2)], dirs=[[[1, 0, 0], [0, 1, 0], [0, 0, 1]]])
    assert float(_prior_parts(mask, th2, K, lam_rep=0, lam_sparse=0, lam_order=0.01)["order"]) == 0.0


def test_26_connectivity_neighbours():
    """The 3x3x3 cube: an interior voxel has 26 neighbours, a corner 7; patches still bound them."""
    mask = np.ones((3, 3, 3), np.uint8)
    bv, gv = _line_scheme(1000.0, [0.0])
    ov = _vol(mask, np.ones((27, 2), np.float32), bv, gv, K=1, connectivity=26, patch_dim=4)
    cnt = (ov.nbr >= 0).sum(1).numpy()
    # 8 corners x 7 + 12 edges x 11 + 6 faces x 17 + centre 26
    assert cnt[13] == 26 and cnt[0] == 7 and cnt.sum() == 8 * 7 + 12 * 11 + 6 * 17 + 26
    ov6 = _vol(mask, np.ones((27, 2), np.float32), bv, gv, K=1, connectivity=6, patch_dim=4)
    assert (ov6.nbr >= 0).sum(1).numpy()[13] == 6
    ov_split = _vol(mask, np.ones((27, 2), np.float32), bv, gv, K=1, connectivity=26, patch_dim=2)
    c2 = (ov_split.nbr >= 0).sum(1).numpy()
    assert c2[0] == 7 and c2[13] == 7 and c2[26] == 0      # (2,2,2) is alone in its 2^3 patch


def test_ordering_kink_has_zero_derivative():
    """R26 at equal fractions (the equal-logit start): value 0 and no gradient from the hinge."""
    mask = np.ones((1, 1, 1), np.uint8)
    bv, gv = _line_scheme(1000.0, [0.0])
    ov = _vol(mask, np.ones((1, 2), np.float32), bv, gv, K=3, lam_rep=0, lam_sparse=0, lam_order=0.01)
    th = _frac_theta(1, 3, [0.0, 0.0, 0.0], dirs=[[[1, 0, 0], [0, 1, 0], [0, 0, 1]]]).requires_grad_(True)
    _, parts = O.objective(ov, th, O.group_init(ov))
    (g,) = torch.autograd.grad(parts["order"], th)
    assert float(parts["order"].detach()) == 0.0 and float(g.abs().max()) == 0.0


def test_crossing_scores_hand_cases():
    """Crossing-benchmark scoring (R31): a single peak on the bisector of a 30 deg crossing
    has best-match error 15 deg for both fibers and detects one of the two; an exact fit
    scores 0 deg and F1 = 1; a spurious third peak lowers precision only."""
    from oracle import metrics as M
    a = np.deg2rad(30.0)
    g1 = np.array([1.0, 0.0, 0.0])
    g2 = np.array([np.cos(a), np.sin(a), 0.0])
    bis = (g1 + g2) / np.linalg.norm(g1 + g2)
    z = np.array([0.0, 0.0, 1.0])
    gt = np.stack([np.stack([g1, g2]), np.stack([g1, g2])])
    ff = np.array([[0.5, 0.5], [0.5, 0.5]])
    case = np.array([3, 5])
    # voxel 0: one peak on the bisector (second fiber below threshold); voxel 1: exact, negated
    dirs = np.stack([np.stack([bis, z, z]), np.stack([-g2, g1, z])])
    peaks = np.array([[True, False, False], [True, True, False]])
    per, overall, rec, prec, f1 = M.crossing_scores(dirs, peaks, gt, ff, case)
    assert abs(per[3] - 15.0) < 1e-9 and abs(per[5]) < 1e-6
    assert abs(overall - 7.5) < 1e-9
    assert rec == 3 / 4 and prec == 1.0
    assert abs(f1 - 2 * 0.75 / 1.75) < 1e-12
    # a spurious orthogonal peak in voxel 1
    peaks2 = peaks.copy()
    peaks2[1, 2] = True
    _, overall2, rec2, prec2, _ = M.crossing_scores(dirs, peaks2, gt, ff, case)
    assert overall2 == overall and rec2 == rec and prec2 == 3 / 4
    # single-fiber ground truth (second gt fraction 0) ignores the second gt direction
    ff1 = np.array([[1.0, 0.0], [1.0, 0.0]])
    per1, _, rec1, _, _ = M.crossing_scores(dirs, peaks, gt, ff1, np.array([0, 0]))
    assert abs(per1[0] - 7.5) < 1e-9 and rec1 == 1.0
