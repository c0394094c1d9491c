"""Shared helpers of the GPU parity tests (oracle <-> library on the same inputs)."""
import types

import numpy as np
import torch

import phantoms as P
from oracle import prism_oracle as O

# Tolerances: signal and objective relative
# error <= 1e-5 (signal relative to max(|y_hat|, 1e-3)); gradient normwise relative error
# <= 1e-4 per parameter block.
TOL_SIGNAL = 1e-5
TOL_LOSS = 1e-5
TOL_GRAD = 1e-4

OPT_KEYS = ("K", "loss", "calibration", "lam_rep", "lam_sparse", "tau", "lam_sp", "huber_delta", "lam_dir",
            "w_alpha", "w_beta", "w_blr", "w_tv", "tv_eps", "patch_dim", "sigma_init", "lr", "beta1",
            "beta2", "eps", "lam_orphan", "s_orphan", "lam_order", "connectivity")


def gpu_volume(vol, init=None, device_signal=False):
    sig = torch.as_tensor(vol.signal).cuda() if device_signal else vol.signal
    return types.SimpleNamespace(mask=vol.mask, signal=sig, bvals=vol.bvals, bvecs=vol.bvecs, init=init)


def oracle_opts(**kw):
    return O.Options(**{k: v for k, v in kw.items() if k in OPT_KEYS})


def make_pair(vols, inits, **kw):
    """(library Fitter, list of OracleVolume) on the same volumes and initial parameters."""
    import paper_2604_00250_gb300 as prism
    o = oracle_opts(**kw)
    ovs = [O.OracleVolume(v.mask, v.signal, v.bvals, v.bvecs, o) for v in vols]
    gv = [gpu_volume(v, init) for v, init in zip(vols, inits)]
    lib_kw = {k: v for k, v in kw.items() if k != "device_signal"}
    f = prism.Fitter(gv, prism.options(**lib_kw))
    return f, ovs


def block_slices(K):
    return {"S0": slice(0, 1), "logits": slice(1, K + 4), "dirs": slice(K + 4, 4 * K + 4),
            "fin": slice(4 * K + 4, 4 * K + 5)}


def normwise(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def signal_rel(yh_gpu, yh_ref):
    d = np.abs(np.asarray(yh_gpu, np.float64) - yh_ref)
    return float(np.max(d / np.maximum(np.abs(yh_ref), 1e-3)))


def split_groups(packed, f):
    """Packed group params -> list of dicts (sigma_log, alpha, beta, blr) in float64 tensors."""
    out = []
    for g in f.group_view(packed):
        out.append(dict(sigma_log=torch.tensor(float(g["sigma_log"]), dtype=torch.float64),
                        alpha=torch.as_tensor(np.asarray(g["alpha"], np.float64)),
                        beta=torch.as_tensor(np.asarray(g["beta"], np.float64)),
                        blr=torch.as_tensor(np.asarray(g["blr"], np.float64))))
    return out


def inits_for(vols, K, seed):
    return [P.default_init(v.n_vox, K, seed + i) for i, v in enumerate(vols)]
