"""Whole-volume fitting in overlapping slabs -- oracle, TEST INFRASTRUCTURE ONLY.

Sec. 3 "Configuration" / Sec. 2.5: the whole-brain fit runs on overlapping
30-slice slabs with a 5-slice overlap, and the slab results are stitched by
weighted averaging. The paper states no more than that; the readings below are
shared with the CUDA path by documentation only.

  R28 slabs run along the last array axis (slices): slab i covers
      [i*(S-O), i*(S-O)+S) clipped to the volume, and slabs are added until one
      reaches the last slice (S = 30, O = 5). Each slab is fitted as its own
      volume (its own sigma and calibration; neighbour priors see only its own
      voxels).
  R29 stitching: a voxel covered by one slab takes that slab's estimate. In the
      overlap of slabs i and i+1 (O slices) the weight of slab i+1 ramps
      linearly, w = (z - z0_{i+1} + 1/2) / O, slab i takes 1 - w. The K fibers
      of slab i+1 are matched to those of slab i by the permutation maximising
      sum_k |d_i,k . d_i+1,pi(k)| (first maximum in lexicographic order), each
      matched direction is flipped to the same hemisphere (d . d' >= 0), and
      then S0, every fraction, f_intra and the directions are averaged with the
      weights; averaged directions are renormalised.
"""
import itertools

import numpy as np

from .prism_oracle import transforms


def slab_ranges(nz, slab=30, overlap=5):
    """List of [z0, z1) per slab along the last axis (R28)."""
    if slab < 1 or overlap < 0 or 2 * overlap > slab:
        raise ValueError("need slab >= 1 and 0 <= overlap <= slab / 2")
    step = slab - overlap
    out = []
    z0 = 0
    while True:
        z1 = min(z0 + slab, nz)
        out.append((z0, z1))
        if z1 >= nz:
            return out
        z0 += step


def slab_weights(nz, ranges):
    """[n_slabs, nz] weight of each slab at each slice (R29): 1 where a slab is alone,
    a linear ramp across each overlap; every slice's weights sum to 1."""
    w = np.zeros((len(ranges), nz))
    for i, (z0, z1) in enumerate(ranges):
        w[i, z0:z1] = 1.0
    for i in range(len(ranges) - 1):
        a0 = ranges[i + 1][0]
        a1 = ranges[i][1]
        for z in range(a0, a1):
            t = (z - a0 + 0.5) / (a1 - a0)
            w[i + 1, z] = t
            w[i, z] = 1.0 - t
    return w


def readout(theta, K):
    """S0 [V], fractions [V, K+3], f_intra [V], unit directions [V, K, 3] (float64 numpy)
    from raw parameters, by the oracle's transforms (Sec. 2.2, Sec. 2.5)."""
    import torch
    s0, frac, d, fin = transforms(torch.as_tensor(np.asarray(theta, np.float64)), K)
    return s0.numpy(), frac.numpy(), fin.numpy(), d.numpy()


def match_fibers(da, db):
    """Permutation pi (tuple) of db's fibers maximising sum_k |da_k . db_pi(k)|, the first
    maximum in lexicographic order, and the signs aligning each matched pair (R29)."""
    K = da.shape[0]
    best, best_p = -1.0, None
    for p in itertools.permutations(range(K)):
        s = sum(abs(float(np.dot(da[k], db[p[k]]))) for k in range(K))
        if s > best:
            best, best_p = s, p
    signs = np.array([1.0 if np.dot(da[k], db[best_p[k]]) >= 0 else -1.0 for k in range(K)])
    return best_p, signs


def stitch(mask, ranges, slab_thetas, K):
    """Whole-volume maps (S0, fractions, f_intra, directions) in the volume's mask order
    (C order) from per-slab raw parameters (each in its slab's mask order), by R29."""
    nz = mask.shape[-1]
    w = slab_weights(nz, ranges)
    coords = np.argwhere(mask)                      # C order = mask order
    V = coords.shape[0]
    s0 = np.zeros(V)
    fr = np.zeros((V, K + 3))
    fin = np.zeros(V)
    dirs = np.zeros((V, K, 3))
    # per slab: readout and the voxel index of each of its mask voxels
    per = []
    for (z0, z1), th in zip(ranges, slab_thetas):
        sub = mask[..., z0:z1]
        c = np.argwhere(sub)
        c[:, -1] += z0
        per.append((readout(th, K), {tuple(x): i for i, x in enumerate(c)}))
    for v in range(V):
        key = tuple(coords[v])
        z = coords[v, -1]
        src = [(i, per[i][1][key]) for i, (z0, z1) in enumerate(ranges) if z0 <= z < z1]
        (ia, va) = src[0]
        A = [x[va] for x in per[ia][0]]
        if len(src) == 1:
            s0[v], fr[v], fin[v], dirs[v] = A
            continue
        (ib, vb) = src[1]
        B = [x[vb] for x in per[ib][0]]
        wa, wb = w[ia, z], w[ib, z]
        p, sg = match_fibers(A[3], B[3])
        s0[v] = wa * A[0] + wb * B[0]
        fin[v] = wa * A[2] + wb * B[2]
        fb = B[1].copy()
        fb[2:K + 2] = B[1][2:K + 2][list(p)]
        fr[v] = wa * A[1] + wb * fb
        dd = wa * A[3] + wb * sg[:, None] * B[3][list(p)]
        dirs[v] = dd / np.linalg.norm(dd, axis=1, keepdims=True)
    return s0, fr, fin, dirs
