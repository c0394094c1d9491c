"""The allocation-free entry point (prism_grad_noalloc) against the handle-based path.

Callers that cannot allocate device memory (a host framework owning the memory pool,
real-time pipelines that reserve memory at start-up) use prism_grad_noalloc; it must
give the objective and gradient that prism_forward / prism_backward give for the same
voxel-local problem, on consecutive calls that share its fixed scratch array. This file
is named to be collected last.
"""
import ctypes
import types

import numpy as np
import pytest
import torch

import phantoms as P
from tests.helpers import TOL_GRAD, TOL_LOSS, normwise

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
