"""Scoring of fitted fibers against known ground truth (the crossing-fiber benchmark,
Sec. 3 "Datasets" and "Tracking & metrics").

Fiber directions are the peaks (Sec. 3 "Configuration"); a fiber is a peak when its share
of the white-matter fraction reaches a threshold (`Fitter.fibers`). Best-match angular
error: every ground-truth fiber is matched to its closest predicted peak, and errors are
pooled over ground-truth fibers, per case label and overall. Detection: peaks and
ground-truth fibers are paired one to one, greedily by increasing angle; pairs within
`match_deg` are true positives, giving recall, precision and F1.
"""
import numpy as np


def _angles(a, b):
    """[V, P, G] sign-free angles (degrees) between a [V, P, 3] and b [V, G, 3]."""
    c = np.abs(np.einsum("vpi,vgi->vpg", a, b))
    return np.degrees(np.arccos(np.clip(c, 0.0, 1.0)))


def score(dirs, peaks, gt_dirs, gt_ffib, case, match_deg=20.0):
    """(per-case mean best-match error {label: deg}, overall error, recall, precision, F1).

    dirs [V, K, 3], peaks [V, K] bool, gt_dirs [V, F, 3], gt_ffib [V, F] (> 0: the fiber
    exists), case [V] integer labels.
    """
    d = np.asarray(dirs, np.float64)
    pk = np.asarray(peaks, bool)
    g = np.asarray(gt_dirs, np.float64)
    gv = np.asarray(gt_ffib) > 0
    case = np.asarray(case)
    ang = _angles(d, g)                                   # [V, K, F]
    big = np.where(pk[:, :, None], ang, np.inf)
    best = big.min(1)                                     # [V, F] closest peak per gt fiber
    errs = best[gv]
    labels = np.broadcast_to(case[:, None], gv.shape)[gv]
    per = {int(c): float(errs[labels == c].mean()) for c in np.unique(labels)}
    # one-to-one greedy pairing by increasing angle
    m = np.where(pk[:, :, None] & gv[:, None, :], ang, np.inf)
    V, K, F = m.shape
    tp = 0
    for _ in range(min(K, F)):
        flat = m.reshape(V, K * F)
        j = flat.argmin(1)
        a = flat[np.arange(V), j]
        hit = a <= match_deg
        tp += int(hit.sum())
        rows, cols = j // F, j % F
        idx = np.flatnonzero(hit)
        m[idx, rows[idx], :] = np.inf
        m[idx, :, cols[idx]] = np.inf
        # voxels whose closest remaining pair is already beyond the threshold are done
        m[~hit] = np.inf
    n_gt = int(gv.sum())
    n_pred = int(pk.sum())
    recall = tp / max(n_gt, 1)
    precision = tp / max(n_pred, 1)
    f1 = 2 * precision * recall / max(precision + recall, 1e-12)
    return per, float(errs.mean()), recall, precision, f1
