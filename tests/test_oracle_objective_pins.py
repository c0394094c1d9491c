"""Hand-value pins of the oracle's data-term normaliser (Eq. 8) and of the calibration
regularisers (Sec. 2.3 "Scale control", Sec. 2.4 "Calibration regularizers"), with
planted mistakes.

Each pin compares the oracle with numbers worked out by hand from the paper's definitions
(closed-form exponentials of known b-values and diffusivities, a b_lr ramp whose trilinear
upsampling is linear and so known at every voxel). The planted-mistake test edits the
oracle's source text on the CPU (one plausible slip at a time: a divisor, an index shift, a
swapped weight, a pair that leaves the mask, a dropped smoothing constant), loads the edited
copy as a separate module and checks that a pin turns red.
"""
import math
import os
import sys
import types

import numpy as np
import pytest
import torch

from oracle import prism_oracle as O

F64 = torch.float64
ORACLE_SRC = open(O.__file__).read()


def _scheme3():
    """b = 0, 1000, 2000 s/mm^2 (the two weighted directions are irrelevant to isotropic pools)."""
    bv = np.array([0.0, 1000.0, 2000.0])
    gv = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    return bv, gv


def _csf_only_theta(Om, V, K=1):
    """S0 = 1 and every fraction in the CSF pool: y_hat = exp(-b D_csf) = 1, e^-3, e^-6 (Eq. 4)."""
    th = torch.zeros(V, Om.n_params(K), dtype=F64)
    th[:, 0] = math.log(math.expm1(1.0))
    th[:, 1:K + 4] = -60.0
    th[:, 1] = 0.0
    th[:, K + 4:4 * K + 4] = 1.0
    return th


def _mse_volume(Om, patches=None):
    """Three voxels on a line, the middle one outside the mask (|M| = 2), patch edge 1."""
    mask = np.array([1, 0, 1], np.uint8).reshape(3, 1, 1)
    sig = np.array([[2.0, 1.0, 0.5], [4.0, 1.0, 1.0]], np.float32)   # b0-normalised: [1, .5, .25], [1, .25, .25]
    bv, gv = _scheme3()
    o = Om.Options(K=1, loss="mse", lam_rep=0.0, lam_sparse=0.0, patch_dim=1)
    return Om.OracleVolume(mask, sig, bv, gv, o, patches=patches)


def pin_mse_value(Om):
    """Eq. 8: (1/|M|) sum_{x,n} (y_hat - y)^2 with |M| = 2 masked voxels (not |M| N = 6)."""
    ov = _mse_volume(Om)
    _, parts = Om.objective(ov, _csf_only_theta(Om, 2), Om.group_init(ov))
    e3, e6 = math.exp(-3.0), math.exp(-6.0)
    by_hand = ((e3 - 0.5) ** 2 + (e6 - 0.25) ** 2 + (e3 - 0.25) ** 2 + (e6 - 0.25) ** 2) / 2.0
    assert abs(by_hand - 0.18265521902478854) < 1e-15
    assert abs(float(parts["data"]) - by_hand) < 1e-14, float(parts["data"])


def pin_mse_subset_normaliser(Om):
    """A volume restricted to one patch (voxel 2 alone, patch id 2) keeps the whole volume's
    |M| = 2 as the divisor: the patch's share of Eq. 8 is its sum / 2, not its sum / 1."""
    ov = _mse_volume(Om, patches=[2])
    assert ov.n_vox == 1
    _, parts = Om.objective(ov, _csf_only_theta(Om, 1), Om.group_init(ov))
    e3, e6 = math.exp(-3.0), math.exp(-6.0)
    by_hand = ((e3 - 0.25) ** 2 + (e6 - 0.25) ** 2) / 2.0
    assert abs(by_hand - 0.050675993058377264) < 1e-15
    assert abs(float(parts["data"]) - by_hand) < 1e-14, float(parts["data"])


W = dict(w_alpha=2e-3, w_beta=3e-3, w_blr=5e-3, w_tv=7e-3, tv_eps=1e-6)


def _ramp_blr(Om):
    """b_lr[a, b, c] = 0.1 a: trilinear upsampling of a linear ramp is the ramp itself, so at
    grid coordinate u (Sec. 2.3, align_corners = False) log B = 0.1 u."""
    return (0.1 * torch.arange(8, dtype=F64))[:, None, None].expand(8, 8, 8).contiguous()


def _cal_volume(Om, shape, mask_flat):
    mask = np.asarray(mask_flat, np.uint8).reshape(shape)
    bv, gv = _scheme3()
    sig = np.ones((int(mask.sum()), 3), np.float32)
    o = Om.Options(K=1, calibration=True, lam_rep=0.0, lam_sparse=0.0, patch_dim=4, **W)
    ov = Om.OracleVolume(mask, sig, bv, gv, o)
    gp = Om.group_init(ov)
    gp["alpha"] = torch.tensor([0.1, -0.2, 0.3], dtype=F64)
    gp["beta"] = torch.tensor([0.05, 0.0, -0.05], dtype=F64)
    gp["blr"] = _ramp_blr(Om)
    _, parts = Om.objective(ov, _csf_only_theta(Om, ov.n_vox), gp)
    return parts


def pin_calibration_l2(Om):
    """w_alpha mean alpha^2, w_beta mean beta^2, w_blr mean b_lr^2 over the N = 3 measurements
    and the 8^3 grid: alpha^2 = (.01 + .04 + .09)/3, beta^2 = .005/3, b_lr^2 = .01 (0+1+...+49)/8."""
    p = _cal_volume(Om, (4, 1, 1), [1, 1, 1, 0])
    assert abs(float(p["cal_alpha"]) - 2e-3 * 0.14 / 3) < 1e-18
    assert abs(float(p["cal_beta"]) - 3e-3 * 0.005 / 3) < 1e-19
    assert abs(float(p["cal_blr"]) - 5e-3 * 0.175) < 1e-17


def pin_tv_line(Om):
    """TV on B = exp(upsampled b_lr) along x on a 4-voxel line whose last voxel is outside the
    mask (|M| = 3). Grid coordinate u = 2i + 1/2 (n = 4), so log B = 0.05, 0.25, 0.45 (0.65 at
    the unmasked voxel). Pairs (0,1), (1,2) count; (2,3) leaves the mask and does not.
    TV = w_tv / 3 (sqrt((e^.25 - e^.05)^2 + eps) + sqrt((e^.45 - e^.25)^2 + eps))."""
    p = _cal_volume(Om, (4, 1, 1), [1, 1, 1, 0])
    d1 = math.exp(0.25) - math.exp(0.05)
    d2 = math.exp(0.45) - math.exp(0.25)
    assert abs(d1 - 0.23275432031171728) < 1e-15 and abs(d2 - 0.28428676880242754) < 1e-15
    by_hand = 7e-3 / 3 * (math.sqrt(d1 * d1 + 1e-6) + math.sqrt(d2 * d2 + 1e-6))
    assert abs(by_hand - 0.0012064383241728405) < 1e-17
    assert abs(float(p["cal_tv"]) - by_hand) < 1e-16, float(p["cal_tv"])


def pin_tv_flat_axis(Om):
    """A 3-voxel line along y with the ramp along x: n_x = 1 puts every voxel at u = 3.5, so B
    is the same everywhere and each of the two y-pairs costs sqrt(eps) = 1e-3."""
    p = _cal_volume(Om, (1, 3, 1), [1, 1, 1])
    assert abs(float(p["cal_tv"]) - 7e-3 / 3 * 2e-3) < 1e-18, float(p["cal_tv"])


PINS = [pin_mse_value, pin_mse_subset_normaliser, pin_calibration_l2, pin_tv_line, pin_tv_flat_axis]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_pin_holds(pin):
    pin(O)


def _mutant(edits):
    """The oracle's source with each (old, new) replacement applied once, as a fresh module."""
    src = ORACLE_SRC
    for old, new in edits:
        assert src.count(old) >= 1, old
        src = src.replace(old, new)
    name = "oracle_planted_mistake"
    mod = types.ModuleType(name)
    mod.__file__ = O.__file__
    sys.modules[name] = mod
    try:
        exec(compile(src, name, "exec"), mod.__dict__)
    finally:
        del sys.modules[name]
    return mod


MISTAKES = {
    # Eq. 8 divided by the number of residuals |M| N instead of the masked-voxel count
    "mse_over_M_times_N": ([('((yhat - y) ** 2).sum() / M', '((yhat - y) ** 2).sum() / (M * ov.n_meas)')],
                           [pin_mse_value]),
    # a patch subset normalised by its own voxel count instead of the volume's
    "mse_over_subset": ([("M = float(n_norm if n_norm is not None else ov.n_mask)",
                          "M = float(n_norm if n_norm is not None else ov.n_vox)")],
                        [pin_mse_subset_normaliser]),
    # sum instead of mean over measurements / grid cells
    "alpha_sum": ([('(gp["alpha"] ** 2).mean()', '(gp["alpha"] ** 2).sum()')], [pin_calibration_l2]),
    "blr_sum": ([('(gp["blr"] ** 2).mean()', '(gp["blr"] ** 2).sum()')], [pin_calibration_l2]),
    # the alpha and beta weights swapped
    "weights_swapped": ([('o.w_alpha * (gp["alpha"]', 'o.w_beta * (gp["alpha"]'),
                         ('o.w_beta * (gp["beta"]', 'o.w_alpha * (gp["beta"]')], [pin_calibration_l2]),
    # TV against x - e instead of x + e
    "tv_backward_neighbour": ([("c1[:, a] += 1", "c1[:, a] -= 1")], [pin_tv_line]),
    # TV counting pairs whose x + e leaves the mask
    "tv_pairs_leave_mask": ([("up[ok, a] = mask[tuple(c[ok].T)]", "up[ok, a] = True")], [pin_tv_line]),
    # TV without the smoothing constant
    "tv_no_eps": ([("torch.sqrt(diff * diff + o.tv_eps)", "torch.sqrt(diff * diff)")], [pin_tv_flat_axis]),
    # TV on the log-bias b_lr upsampled instead of on B = exp(.)
    "tv_on_log_bias": ([("B0 = torch.exp(bias_log(gp[\"blr\"], ov.coords, ov.shape))",
                         "B0 = bias_log(gp[\"blr\"], ov.coords, ov.shape)"),
                        ("B1 = torch.exp(bias_log(gp[\"blr\"], c1, ov.shape))",
                         "B1 = bias_log(gp[\"blr\"], c1, ov.shape)")], [pin_tv_line]),
}


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_planted_mistake_turns_a_pin_red(name):
    edits, pins = MISTAKES[name]
    mod = _mutant(edits)
    for pin in pins:
        with pytest.raises(AssertionError):
            pin(mod)
    # the untouched oracle loaded the same way passes the same pins
    clean = _mutant([])
    for pin in pins:
        pin(clean)
