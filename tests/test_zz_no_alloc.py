"""The allocation-free entry point (prism_grad_noalloc) against the handle-based path and
the oracle.

Callers that cannot allocate device memory (a host framework owning the memory pool,
real-time pipelines that reserve memory at start-up) use prism_grad_noalloc; it must
give the objective and gradient that prism_forward / prism_backward give for the same
voxel-local problem, on consecutive calls that share its fixed scratch array, and those of
the FP64 oracle. A voxel whose b <= 50 mean is not positive comes back as a NaN gradient row
and a NaN loss; inputs the handle path refuses are refused here too. This file is named to
be collected last.
"""
import ctypes
import types

import numpy as np
import pytest
import torch

import phantoms as P
from oracle import prism_oracle as O
from tests.helpers import TOL_GRAD, TOL_LOSS, block_slices, normwise

pytestmark = pytest.mark.gpu


def _call(lib, sig, bvals, bvecs, theta, V, N, K, lam_rep, lam_sparse, tau, grad, loss):
    return lib.prism_grad_noalloc(ctypes.c_void_p(sig.data_ptr()), bvals.ctypes.data, bvecs.ctypes.data,
                                  ctypes.c_void_p(theta.data_ptr()), V, N, K, lam_rep, lam_sparse, tau,
                                  ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("K", [3, 2])
def test_noalloc_matches_handle_path_twice(K):
    import paper_2604_00250_gb300 as prism
    from paper_2604_00250_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(21 + K)
    vol = P.random_volume((9, 7, 6), seed=21 + K, mask_density=0.8)
    V, N = vol.n_vox, vol.n_meas
    theta0 = (P.default_init(V, K, 4) + rng.normal(0, 0.3, (V, 4 * K + 5))).astype(np.float32)
    v = types.SimpleNamespace(mask=vol.mask, signal=vol.signal, bvals=vol.bvals, bvecs=vol.bvecs, init=theta0)
    f = prism.Fitter([v], prism.options(K=K, loss="mse", calibration=0, lam_sp=0.0, lam_dir=0.0, patch_dim=4))
    loss_ref, _ = f.forward()
    g_ref, _ = f.backward()
    torch.cuda.synchronize()
    loss_ref = float(loss_ref[0])
    g_ref = g_ref.cpu().numpy()
    f.close()
    sig = torch.as_tensor(vol.signal).cuda()
    th = torch.as_tensor(theta0).cuda()
    bvals = np.ascontiguousarray(vol.bvals, dtype=np.float32)
    bvecs = np.ascontiguousarray(vol.bvecs, dtype=np.float32)
    opts = prism.options(K=K)
    for _ in range(2):
        grad = torch.full((V, 4 * K + 5), float("nan"), dtype=torch.float32, device="cuda")
        loss = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        rc = _call(lib, sig, bvals, bvecs, th, V, N, K, opts.lam_rep, opts.lam_sparse, opts.tau, grad, loss)
        assert rc == 0, lib.prism_last_error()
        torch.cuda.synchronize()
        assert abs(float(loss[0]) - loss_ref) <= TOL_LOSS * abs(loss_ref)
        assert normwise(grad.cpu().numpy(), g_ref) <= TOL_GRAD


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2604_00250_gb300 import _lib
    lib = _lib.load()
    bvals = np.zeros(4, np.float32)
    bvecs = np.zeros((4, 3), np.float32)
    dummy = torch.zeros(16, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = _call(lib, dummy, bvals, bvecs, dummy, 1_048_577, 4, 3, 0.01, 0.02, 0.15, dummy, loss)
    assert rc == 2
    assert b"1048576" in lib.prism_last_error()
    rc = _call(lib, dummy, bvals, bvecs, dummy, 16, 1025, 3, 0.01, 0.02, 0.15, dummy, loss)
    assert rc == 2


def _oracle_value_and_grad(vol, theta0, K):
    o = O.Options(K=K, loss="mse", calibration=False, lam_sp=0.0, lam_dir=0.0, patch_dim=4)
    ov = O.OracleVolume(vol.mask, vol.signal, vol.bvals, vol.bvecs, o)
    J, _, g, _ = O.value_and_grad(ov, torch.as_tensor(theta0).double(), O.group_init(ov))
    return float(J), g.numpy()


def _run(lib, vol, theta0, K, signal=None):
    V, N = vol.n_vox, vol.n_meas
    sig = torch.as_tensor(vol.signal if signal is None else signal).cuda()
    th = torch.as_tensor(theta0).cuda()
    bvals = np.ascontiguousarray(vol.bvals, dtype=np.float32)
    bvecs = np.ascontiguousarray(vol.bvecs, dtype=np.float32)
    grad = torch.full((V, 4 * K + 5), float("nan"), dtype=torch.float32, device="cuda")
    loss = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    rc = _call(lib, sig, bvals, bvecs, th, V, N, K, 0.01, 0.02, 0.15, grad, loss)
    assert rc == 0, lib.prism_last_error()
    torch.cuda.synchronize()
    return float(loss[0]), grad.cpu().numpy()


@pytest.mark.parametrize("K", [3, 5])
def test_noalloc_matches_oracle(K):
    from paper_2604_00250_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(51 + K)
    vol = P.random_volume((11, 6, 5), seed=51 + K, mask_density=0.7)
    theta0 = (P.default_init(vol.n_vox, K, 5) + rng.normal(0, 0.3, (vol.n_vox, 4 * K + 5))).astype(np.float32)
    J, g = _oracle_value_and_grad(vol, theta0, K)
    loss, grad = _run(lib, vol, theta0, K)
    assert abs(loss - J) <= TOL_LOSS * abs(J), (loss, J)
    for name, sl in block_slices(K).items():
        assert normwise(grad[:, sl], g[:, sl]) <= TOL_GRAD, name


def test_noalloc_reports_a_non_positive_b0_mean():
    """One voxel with zero signal at every b <= 50 measurement: its gradient row and the loss
    are NaN; every other row is the oracle's (each row depends only on its own voxel and on
    n_vox, which still counts the bad voxel)."""
    from paper_2604_00250_gb300 import _lib
    lib = _lib.load()
    K = 3
    rng = np.random.default_rng(61)
    vol = P.random_volume((6, 5, 4), seed=61, mask_density=0.8)
    theta0 = (P.default_init(vol.n_vox, K, 6) + rng.normal(0, 0.3, (vol.n_vox, 4 * K + 5))).astype(np.float32)
    bad = 7
    sig = np.array(vol.signal, dtype=np.float32, copy=True)
    sig[bad, vol.bvals <= 50] = 0.0
    loss, grad = _run(lib, vol, theta0, K, signal=sig)
    assert np.isnan(loss)
    assert np.isnan(grad[bad]).all()
    keep = np.ones(vol.n_vox, bool)
    keep[bad] = False
    assert np.isfinite(grad[keep]).all()
    _, g = _oracle_value_and_grad(vol, theta0, K)
    for name, sl in block_slices(K).items():
        assert normwise(grad[keep][:, sl], g[keep][:, sl]) <= TOL_GRAD, name


def test_noalloc_rejects_what_the_handle_path_rejects():
    """Non-finite b-vectors and non-unit b-vectors of b > 50 measurements: E_INVALID_ARG
    before any device work, as prism_fit_init answers."""
    from paper_2604_00250_gb300 import _lib
    lib = _lib.load()
    bvals = np.array([0.0, 1000.0, 2000.0, 5.0], np.float32)
    good = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.3, 0.0, 0.0]], np.float32)   # b = 5: any length
    dummy = torch.zeros(64, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    for bad_row, val in [(1, [np.nan, 0, 0]), (3, [np.inf, 0, 0]), (2, [0, 0.9, 0])]:
        bvecs = good.copy()
        bvecs[bad_row] = val
        rc = _call(lib, dummy, bvals, bvecs, dummy, 2, 4, 3, 0.01, 0.02, 0.15, dummy, loss)
        assert rc == 1, (bad_row, rc)
    bv = bvals.copy()
    bv[2] = np.nan
    assert _call(lib, dummy, bv, good, dummy, 2, 4, 3, 0.01, 0.02, 0.15, dummy, loss) == 1
