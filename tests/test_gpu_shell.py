"""The fused kernel's shell loop (one thread per voxel, MSE, no calibration, K <= 3) against
the oracle.

With every shell of the scheme holding an even number of measurements, the library sorts the
measurements by b-value and takes the shell loop, which forms the isotropic mixture and the
exponent constants of each b-value shell once per voxel (Eqs. 4-5 with the scaled cosine).
Checked here, on schemes whose measurements arrive interleaved in the caller's order:
- the first iteration's gradient (Adam's first moment) per block against the oracle's;
- three iterations against the oracle's trajectory, and against the per-measurement loop of
  the same library (shells = -1);
- a scheme without b = 0 whose shells span b = 5 to 6000 (the direction sums' rescaling);
- the shapes that cannot take the loop fall back to the per-measurement loop (an odd shell,
  more than 16 shells) and still match the oracle.
"""
import numpy as np
import pytest
import torch

import phantoms as P
from oracle import prism_oracle as O
from tests.helpers import TOL_GRAD, TOL_LOSS, block_slices, inits_for, make_pair, normwise, split_groups
from tests.test_gpu_fused_gradient import fused_gradient

pytestmark = pytest.mark.gpu


def _shuffled(vol, seed):
    perm = np.random.default_rng(seed).permutation(vol.n_meas)
    return P.Volume(mask=vol.mask, signal=np.ascontiguousarray(np.asarray(vol.signal)[:, perm]),
                    bvals=vol.bvals[perm].copy(), bvecs=vol.bvecs[perm].copy(), gt=vol.gt)


def _even_shell_problem(seed=0):
    sch = P.make_scheme(2, [(1000, 14), (2500, 16)], seed)               # N = 32: 2 + 14 + 16
    sch2 = P.make_scheme(4, [(700, 8), (1500, 6), (3000, 4)], seed + 1)  # N = 22 (NP = 24): 4 + 8 + 6 + 4
    v1 = P.random_volume((7, 5, 6), scheme=sch, seed=seed, mask_density=0.75)
    v2 = P.random_volume((5, 6, 4), scheme=sch2, seed=seed + 1, mask_density=0.6)
    return [_shuffled(v1, 3), _shuffled(v2, 4)]


KW = dict(loss="mse", patch_dim=4, lam_sp=0.01, lam_dir=0.005, fused=1, use_graph=1, threads_per_voxel=1)


@pytest.mark.parametrize("K", [1, 2, 3])
def test_shell_loop_gradient_matches_oracle(K):
    rng = np.random.default_rng(70 + K)
    vols = _even_shell_problem()
    inits = [(t + rng.normal(0, 0.3, t.shape)).astype(np.float32) for t in inits_for(vols, K, 2)]
    f, ovs = make_pair(vols, inits, K=K, **KW)
    assert f.shape()["shell_loop"] == 1
    gps = split_groups(f.groups(), f)
    f.step(1)
    f.sync()
    g_vox, _ = fused_gradient(f, f.opts.beta1)
    hist = f.loss_history()
    v0 = 0
    for gi, ov in enumerate(ovs):
        J, _, g, _ = O.value_and_grad(ov, torch.as_tensor(inits[gi]).double(), gps[gi])
        assert abs(hist[0, gi] - float(J)) <= TOL_LOSS * abs(float(J))
        for name, sl in block_slices(K).items():
            e = normwise(g_vox[v0:v0 + ov.n_vox, sl], g[:, sl].numpy())
            assert e <= TOL_GRAD, (gi, name, e)
        v0 += ov.n_vox
    f.close()


@pytest.mark.parametrize("K", [2, 3])
def test_shell_loop_trajectory_matches_oracle_and_the_measurement_loop(K):
    vols = _even_shell_problem(1)
    inits = inits_for(vols, K, 5)
    f, ovs = make_pair(vols, inits, K=K, **KW)
    assert f.shape()["shell_loop"] == 1
    f.step(3)
    f.sync()
    res = O.fit(ovs, [torch.as_tensor(t).double() for t in inits], 3)
    np.testing.assert_allclose(f.loss_history(), res.loss_history, rtol=1e-5)
    th = f.params_host()
    ref = np.concatenate([t.numpy() for t in res.theta])
    assert float(np.max(np.abs(th - ref))) < 3e-4
    f.close()
    g, _ = make_pair(vols, inits, K=K, shells=-1, **KW)
    assert g.shape()["shell_loop"] == 0
    g.step(3)
    g.sync()
    assert float(np.max(np.abs(g.params_host() - th))) < 3e-4
    np.testing.assert_allclose(g.loss_history(), res.loss_history, rtol=1e-5)
    g.close()


def test_shell_loop_without_b0_and_with_a_low_b_shell():
    """No b = 0 measurement: the first shell the loop opens has b > 0, and a b = 5 shell next to
    b = 6000 gives the largest ratio between two shells' dE/dc factors (ap is proportional to
    sqrt(b)), by which the direction sums are rescaled at each shell change. The b = 5 shell
    also serves as the b0 reference of the normalisation (b <= 50)."""
    K = 3
    sch = P.make_scheme(0, [(5, 4), (1000, 6), (6000, 8)], 5)
    v = P.random_volume((6, 5, 4), scheme=sch, seed=11, mask_density=0.8)
    vols = [_shuffled(v, 6)]
    rng = np.random.default_rng(77)
    inits = [(t + rng.normal(0, 0.3, t.shape)).astype(np.float32) for t in inits_for(vols, K, 2)]
    f, ovs = make_pair(vols, inits, K=K, **KW)
    assert f.shape()["shell_loop"] == 1
    gps = split_groups(f.groups(), f)
    f.step(1)
    f.sync()
    g_vox, _ = fused_gradient(f, f.opts.beta1)
    J, _, g, _ = O.value_and_grad(ovs[0], torch.as_tensor(inits[0]).double(), gps[0])
    assert abs(f.loss_history()[0, 0] - float(J)) <= TOL_LOSS * abs(float(J))
    for name, sl in block_slices(K).items():
        e = normwise(g_vox[:, sl], g[:, sl].numpy())
        assert e <= TOL_GRAD, (name, e)
    f.close()


@pytest.mark.parametrize("scheme", ["odd_shell", "many_shells"])
def test_schemes_outside_the_shell_loop(scheme):
    if scheme == "odd_shell":
        sch = P.make_scheme(3, [(1000, 14), (2500, 16)], 2)                # b = 0 shell of 3
    else:
        sch = P.make_scheme(2, [(400 + 100 * i, 2) for i in range(17)], 2)  # 18 shells
    vols = [P.random_volume((6, 5, 4), scheme=sch, seed=9, mask_density=0.8)]
    K = 3
    inits = inits_for(vols, K, 9)
    f, ovs = make_pair(vols, inits, K=K, **KW)
    assert f.shape()["shell_loop"] == 0
    f.step(2)
    f.sync()
    res = O.fit(ovs, [torch.as_tensor(t).double() for t in inits], 2)
    np.testing.assert_allclose(f.loss_history(), res.loss_history, rtol=1e-5)
    assert float(np.max(np.abs(f.params_host() - res.theta[0].numpy()))) < 3e-4
    f.close()
