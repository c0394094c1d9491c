"""Peak extraction and angular comparison -- TEST INFRASTRUCTURE ONLY.

Fiber directions are used directly as peaks (Sec. 3 "Configuration"); a fiber
counts as a peak when its share of the white-matter fraction is at least
`rel_thresh` (reading R20: the paper gives no threshold; 0.15 by default). Angles are arccos|d . d'| in degrees (directions
are sign-free). Best-match angular error matches each reference fiber to its
closest predicted fiber (Sec. 3 "Tracking & metrics").
"""
import itertools

import numpy as np


def fibers(theta, K):
    """(dirs [V, K, 3] unit, WM fractions [V, K]) from raw parameters (float64 numpy)."""
    th = np.asarray(theta, dtype=np.float64)
    lg = th[:, 1:K + 4]
    e = np.exp(lg - lg.max(1, keepdims=True))
    fr = e / e.sum(1, keepdims=True)
    v = th[:, K + 4:4 * K + 4].reshape(-1, K, 3)
    d = v / np.maximum(np.linalg.norm(v, axis=2, keepdims=True), 1e-12)
    return d, fr[:, 2:K + 2]


def peak_mask(fwm, rel_thresh=0.15):
    tot = np.maximum(fwm.sum(1, keepdims=True), 1e-12)
    return fwm / tot >= rel_thresh


def angle_deg(a, b):
    c = np.clip(np.abs(np.sum(a * b, axis=-1)), 0.0, 1.0)
    return np.degrees(np.arccos(c))


def matched_deviation(theta_a, theta_b, K, rel_thresh=0.15):
    """Per voxel: the largest angle between a's peaks and b's fibers after the best
    permutation (over K! assignments, sign-free). Also returns peak counts."""
    da, fa = fibers(theta_a, K)
    db, fb = fibers(theta_b, K)
    pa = peak_mask(fa, rel_thresh)
    pb = peak_mask(fb, rel_thresh)
    V = da.shape[0]
    best = np.full(V, np.inf)
    for perm in itertools.permutations(range(K)):
        ang = angle_deg(da, db[:, list(perm)])                  # [V, K]
        dev = np.where(pa, ang, 0.0).max(1)
        best = np.minimum(best, dev)
    return best, pa.sum(1), pb.sum(1)


def best_match_error(theta, gt_dirs, gt_ffib, K, rel_thresh=0.15, match_deg=20.0):
    """Best-match angular error vs ground truth, recall and precision of peaks."""
    d, f = fibers(theta, K)
    pk = peak_mask(f, rel_thresh)
    errs = []
    hit = 0
    total_gt = 0
    fp = 0
    for v in range(d.shape[0]):
        pred = d[v][pk[v]]
        gts = gt_dirs[v][gt_ffib[v] > 0]
        total_gt += len(gts)
        used = set()
        for g in gts:
            if len(pred) == 0:
                continue
            a = angle_deg(pred, g[None, :])
            j = int(np.argmin(a))
            errs.append(a[j])
            if a[j] <= match_deg:
                hit += 1
                used.add(j)
        fp += len(pred) - len(used)
    recall = hit / max(total_gt, 1)
    precision = hit / max(hit + fp, 1)
    f1 = 2 * precision * recall / max(precision + recall, 1e-12)
    return float(np.mean(errs)) if errs else float("nan"), recall, f1


def crossing_scores(dirs, peaks, gt_dirs, gt_ffib, case, match_deg=20.0):
    """Crossing-benchmark scores (Sec. 3 "Tracking & metrics"; reading R31: best-match error
    per ground-truth fiber; detection pairs peaks and fibers one to one, greedily by angle,
    within `match_deg`).

    dirs [V, K, 3] fitted unit directions, peaks [V, K] bool (R20), gt_dirs [V, F, 3],
    gt_ffib [V, F] (a ground-truth fiber exists where > 0), case [V] integer label.
    Best-match angular error: every ground-truth fiber is matched to its closest predicted
    peak (several may share one); errors are pooled over ground-truth fibers, per case and
    overall. Detection: predicted peaks and ground-truth fibers are paired one to one,
    greedily by increasing angle, pairs within match_deg counting as true positives;
    recall = TP / ground-truth fibers, precision = TP / predicted peaks, F1 their harmonic
    mean. Returns (per_case {label: mean error}, overall error, recall, precision, F1).
    """
    per = {}
    errs_all = []
    tp = n_gt = n_pred = 0
    for v in range(dirs.shape[0]):
        pred = [dirs[v, k] for k in range(dirs.shape[1]) if peaks[v, k]]
        gts = [gt_dirs[v, j] for j in range(gt_dirs.shape[1]) if gt_ffib[v, j] > 0]
        n_gt += len(gts)
        n_pred += len(pred)
        for g in gts:
            e = min(float(angle_deg(p, g)) for p in pred)
            per.setdefault(int(case[v]), []).append(e)
            errs_all.append(e)
        pairs = sorted((float(angle_deg(p, g)), i, j) for i, p in enumerate(pred) for j, g in enumerate(gts))
        used_p, used_g = set(), set()
        for a, i, j in pairs:
            if a > match_deg:
                break
            if i in used_p or j in used_g:
                continue
            used_p.add(i)
            used_g.add(j)
            tp += 1
    recall = tp / max(n_gt, 1)
    precision = tp / max(n_pred, 1)
    f1 = 2 * precision * recall / max(precision + recall, 1e-12)
    return ({c: float(np.mean(v)) for c, v in sorted(per.items())}, float(np.mean(errs_all)), recall, precision, f1)
