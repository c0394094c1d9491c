"""PrismLoss (the torch.autograd.Function over prism_forward / prism_backward) on the GPU.

Sec. 2.1: every component of the forward model is differentiable, so tissue and calibration
parameters can be updated jointly by gradient descent. The gradient that PrismLoss hands to
autograd is the library's hand-written adjoint; it is checked against
- the oracle's analytic (autograd FP64) gradient, per parameter block, for theta and the
  packed group parameters (sigma, alpha, beta, b_lr), with and without explicit groups;
- central finite differences of the FP64 oracle objective (h = 1e-4) over every raw voxel
  parameter and sampled group parameters of a 2x2x2 patch;
- two PrismLoss nodes on one handle in one graph (each gets the gradient at its own point).
"""
import math

import numpy as np
import pytest
import torch

import phantoms as P
from oracle import prism_oracle as O
from tests.helpers import TOL_GRAD, TOL_LOSS, block_slices, inits_for, make_pair, normwise, split_groups

pytestmark = pytest.mark.gpu


def _problem(cal, seed=0):
    sch = P.make_scheme(3, [(1000, 14), (2500, 15)], seed)       # N = 32
    sch2 = P.make_scheme(2, [(800, 9), (2000, 10)], seed + 1)    # N = 21
    return [P.random_volume((7, 5, 6), scheme=sch, seed=seed, mask_density=0.75, calibration=cal),
            P.random_volume((5, 6, 4), scheme=sch2, seed=seed + 1, mask_density=0.6, calibration=cal)]


def _perturbed_groups(f, rng, cal, loss):
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
    return packed


def _oracle_grads(ovs, thetas, gps):
    out = []
    for ov, th, gp in zip(ovs, thetas, gps):
        out.append(O.value_and_grad(ov, torch.as_tensor(th).double(), gp))
    return out


def _check_theta_grad(gth, ref, K):
    v0 = 0
    for gi, (_, _, g, _) in enumerate(ref):
        n = g.shape[0]
        for name, sl in block_slices(K).items():
            e = normwise(gth[v0:v0 + n, sl], g[:, sl].numpy())
            assert e <= TOL_GRAD, (gi, name, e)
        v0 += n


def _check_group_grad(gg, ref, f, loss, cal):
    off = f.group_layout()
    for gi, (_, _, _, ggr) in enumerate(ref):
        a, b, c, d = (int(x) for x in off[4 * gi:4 * gi + 4])
        N = f.n_meas[gi]
        if loss == "nll":
            assert normwise([gg[a]], [float(ggr["sigma_log"])]) <= TOL_GRAD, ("sigma", gi)
        if cal:
            assert normwise(gg[b:b + N], ggr["alpha"].numpy()) <= TOL_GRAD, ("alpha", gi)
            assert normwise(gg[c:c + N], ggr["beta"].numpy()) <= TOL_GRAD, ("beta", gi)
            assert normwise(gg[d:d + 512], ggr["blr"].numpy().ravel()) <= TOL_GRAD, ("blr", gi)


@pytest.mark.parametrize("loss,cal", [("mse", False), ("nll", False), ("mse", True), ("nll", True)])
def test_prism_loss_matches_oracle_gradient(loss, cal):
    import paper_2604_00250_gb300 as prism
    rng = np.random.default_rng(21)
    vols = _problem(cal)
    K = 3
    inits = [(t + rng.normal(0, 0.3, t.shape)).astype(np.float32) for t in inits_for(vols, K, 4)]
    f, ovs = make_pair(vols, inits, K=K, loss=loss, calibration=cal, patch_dim=4, lam_sp=0.01, lam_dir=0.005)
    packed = _perturbed_groups(f, rng, cal, loss)
    theta = torch.as_tensor(np.concatenate(inits)).cuda().requires_grad_(True)
    groups = torch.as_tensor(packed).cuda().requires_grad_(True)
    J = prism.PrismLoss.apply(theta, groups, f)
    J.backward()
    ref = _oracle_grads(ovs, inits, split_groups(packed, f))
    Jref = sum(float(r[0]) for r in ref)
    assert abs(float(J.detach()) - Jref) <= TOL_LOSS * abs(Jref), (float(J.detach()), Jref)
    _check_theta_grad(theta.grad.cpu().numpy(), ref, K)
    _check_group_grad(groups.grad.cpu().numpy(), ref, f, loss, cal)
    # groups=None: the handle's current group parameters (now `packed`), no group gradient
    theta2 = theta.detach().clone().requires_grad_(True)
    prism.PrismLoss.apply(theta2, None, f).backward()
    _check_theta_grad(theta2.grad.cpu().numpy(), ref, K)
    f.close()


def _away_from_kinks(th, K, tau=0.15, margin=2e-3):
    """True when no WM fraction is near the sparsity gate and no fiber pair is near |d.d'| = 0,
    so that +-h steps (h = 1e-4) stay on one side of every non-smooth point."""
    _, fr, d, _ = O.transforms(th, K)
    fw = fr[:, 2:K + 2]
    if float((fw - tau).abs().min()) <= margin:
        return False
    for i in range(K):
        for j in range(i + 1, K):
            if float((d[:, i] * d[:, j]).sum(-1).abs().min()) <= margin:
                return False
    return True


@pytest.mark.parametrize("loss,cal,K", [("mse", False, 2), ("nll", True, 3), ("mse", True, 3), ("nll", False, 3)])
def test_prism_loss_against_central_differences(loss, cal, K):
    """PrismLoss's gradient vs central differences of the FP64 oracle objective, h = 1e-4,
    over all 8 x (4K + 5) raw voxel parameters and sampled group parameters of one 2x2x2
    patch with N = 12 (every prior on)."""
    import paper_2604_00250_gb300 as prism
    rng = np.random.default_rng(31 + K)
    bv, gv = P.make_scheme(2, [(1000, 5), (2500, 5)], 8)
    vol = P.random_volume((2, 2, 2), scheme=(bv, gv), seed=8, calibration=cal)
    while True:
        th = rng.normal(0, 0.7, size=(vol.n_vox, 4 * K + 5)).astype(np.float32)
        if _away_from_kinks(torch.as_tensor(th).double(), K):
            break
    kw = dict(K=K, loss=loss, calibration=cal, patch_dim=2, lam_sp=0.01, lam_dir=0.005)
    f, ovs = make_pair([vol], [th], **kw)
    ov = ovs[0]
    packed = _perturbed_groups(f, rng, cal, loss)
    theta = torch.as_tensor(th).cuda().requires_grad_(True)
    groups = torch.as_tensor(packed).cuda().requires_grad_(True)
    prism.PrismLoss.apply(theta, groups, f).backward()
    gth = theta.grad.cpu().numpy()
    gg = groups.grad.cpu().numpy()
    gp = split_groups(packed, f)[0]
    h = 1e-4
    t64 = torch.as_tensor(th).double()

    def J(t, q):
        return float(O.objective(ov, t, q)[0])

    fd = np.zeros(th.shape)
    for v in range(th.shape[0]):
        for q in range(th.shape[1]):
            tp = t64.clone(); tp[v, q] += h
            tm = t64.clone(); tm[v, q] -= h
            fd[v, q] = (J(tp, gp) - J(tm, gp)) / (2 * h)
    for name, sl in block_slices(K).items():
        e = normwise(gth[:, sl], fd[:, sl])
        assert e <= TOL_GRAD, (name, e)
    off = f.group_layout()
    a, b, c, d = (int(x) for x in off[:4])
    blocks = {}
    if loss == "nll":
        blocks["sigma_log"] = [(None, a)]
    if cal:
        blocks["alpha"] = [(i, b + i) for i in rng.choice(ov.n_meas, 5, replace=False)]
        blocks["beta"] = [(i, c + i) for i in rng.choice(ov.n_meas, 5, replace=False)]
        blocks["blr"] = [(i, d + i) for i in rng.choice(512, 8, replace=False)]
    for name, picks in blocks.items():
        got, want = [], []
        for i, pos in picks:
            qp = {k: x.clone() for k, x in gp.items()}
            qm = {k: x.clone() for k, x in gp.items()}
            if i is None:
                qp[name] = qp[name] + h
                qm[name] = qm[name] - h
            else:
                qp[name].view(-1)[i] += h
                qm[name].view(-1)[i] -= h
            want.append((J(t64, qp) - J(t64, qm)) / (2 * h))
            got.append(gg[pos])
        assert normwise(got, want) <= TOL_GRAD, (name, got, want)
    f.close()


def test_two_prism_loss_nodes_on_one_handle():
    """J = L(theta_1) + 2 L(theta_2) on one Fitter: the second node's forward overwrites the
    handle's point, so the first node's backward must evaluate again at theta_1."""
    import paper_2604_00250_gb300 as prism
    rng = np.random.default_rng(41)
    vols = _problem(False)
    K = 3
    i1 = [(t + rng.normal(0, 0.3, t.shape)).astype(np.float32) for t in inits_for(vols, K, 5)]
    i2 = [(t + rng.normal(0, 0.3, t.shape)).astype(np.float32) for t in inits_for(vols, K, 6)]
    f, ovs = make_pair(vols, i1, K=K, loss="nll", patch_dim=4, lam_sp=0.01)
    gps = split_groups(f.groups(), f)
    t1 = torch.as_tensor(np.concatenate(i1)).cuda().requires_grad_(True)
    t2 = torch.as_tensor(np.concatenate(i2)).cuda().requires_grad_(True)
    J = prism.PrismLoss.apply(t1, None, f) + 2.0 * prism.PrismLoss.apply(t2, None, f)
    J.backward()
    r1 = _oracle_grads(ovs, i1, gps)
    r2 = _oracle_grads(ovs, i2, gps)
    Jref = sum(float(r[0]) for r in r1) + 2.0 * sum(float(r[0]) for r in r2)
    assert abs(float(J.detach()) - Jref) <= TOL_LOSS * abs(Jref)
    _check_theta_grad(t1.grad.cpu().numpy(), r1, K)
    _check_theta_grad(t2.grad.cpu().numpy() / 2.0, r2, K)
    f.close()
