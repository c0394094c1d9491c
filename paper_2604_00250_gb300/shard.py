"""Sharding of independent fits across ranks (one process per GPU).

Two units of independent work, each split across ranks with no data-path collective
(every rank fits its share on its own GPU; results are gathered once at the end):

- volumes: each carries its own sigma and calibration (Sec. 2.3) and neighbour priors never
  cross a volume, so a batch is split by whole volumes (any loss, any calibration);
- patches of one volume: the neighbour priors stay inside a patch (Sec. 2.4 with the
  same-patch neighbourhood), so without calibration and with the MSE (no volume-wide sigma)
  every patch is its own problem, coupled to the others only through the normaliser |M| of
  Eq. 8. A rank fits the volume's mask restricted to its patches with the whole volume's |M|
  (prism_volume.norm_count), and every voxel follows the whole-volume fit exactly.

Assignment is longest-processing-time first (cost = masked voxels x measurements for
volumes, masked voxels for patches), which bounds the slowest rank's work by 4/3 of the
optimum.
"""
import types

import numpy as np


def volume_cost(vol):
    return int(np.asarray(vol.mask).astype(bool).sum()) * int(np.asarray(vol.bvals).shape[0])


def assign_volumes(costs, world):
    """Rank of each volume: largest first onto the least-loaded rank (ties: lowest rank)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world
    owner = [0] * len(costs)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += costs[i]
    return owner, load


def run_sharded(volumes, fit_fn, rank=0, world=1, group=None):
    """Fits this rank's volumes with fit_fn(list_of_volumes) -> list of per-volume results
    and gathers {volume index: result} on every rank (torch.distributed, any backend)."""
    owner, _ = assign_volumes([volume_cost(v) for v in volumes], world)
    mine = [i for i in range(len(volumes)) if owner[i] == rank]
    local = dict(zip(mine, fit_fn([volumes[i] for i in mine]))) if mine else {}
    if world == 1:
        return local
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, local, group=group)
    merged = {}
    for p in parts:
        for k, v in p.items():
            if k in merged:
                raise RuntimeError(f"volume {k} fitted on two ranks")
            merged[k] = v
    if len(merged) != len(volumes):
        raise RuntimeError("some volumes were not fitted")
    return merged


def fit_volumes_on_this_gpu(opts, n_iters):
    """fit_fn for run_sharded: one library fit per rank over its volumes."""
    def fn(vols):
        from . import Fitter
        f = Fitter(list(vols), opts)
        f.step(n_iters)
        f.sync()
        theta = f.params_host()
        loss = f.loss()
        f.close()
        out, v0 = [], 0
        for g, v in enumerate(vols):
            n = int(np.asarray(v.mask).astype(bool).sum())
            out.append({"theta": theta[v0:v0 + n], "loss": float(loss[g])})
            v0 += n
        return out
    return fn


def patch_of_voxels(mask, patch_dim):
    """Patch id (C order over the patch grid) of every masked voxel, in mask order."""
    m = np.asarray(mask).astype(bool)
    coords = np.argwhere(m)
    pshape = tuple(-(-n // patch_dim) for n in m.shape)
    return np.ravel_multi_index(tuple((coords // patch_dim).T), pshape)


def assign_patches(mask, patch_dim, world):
    """(patch ids, owner rank of each, per-rank voxel load) for the non-empty patches of
    `mask`: the fullest patch first onto the least-loaded rank (ties: lowest rank)."""
    pid = patch_of_voxels(mask, patch_dim)
    ids, counts = np.unique(pid, return_counts=True)
    owner, load = assign_volumes([int(c) for c in counts], world)
    return ids, np.asarray(owner), load


def shard_volume(vol, patch_dim, rank, world):
    """This rank's part of one volume: a volume-like namespace whose mask keeps only the
    rank's patches (signal and init rows of those voxels, norm_count = the whole volume's
    masked voxels), and the mask-order positions `sel` of those voxels in the whole volume."""
    mask = np.asarray(vol.mask).astype(bool)
    pid = patch_of_voxels(mask, patch_dim)
    ids, owner, _ = assign_patches(mask, patch_dim, world)
    mine = ids[owner == rank]
    sel = np.flatnonzero(np.isin(pid, mine))
    sub = np.zeros_like(mask)
    coords = np.argwhere(mask)[sel]
    sub[tuple(coords.T)] = True
    sig = vol.signal
    if hasattr(sig, "is_cuda"):          # a torch tensor (host or device)
        import torch
        sig = sig[torch.as_tensor(sel, device=sig.device)]
    else:
        sig = np.asarray(sig)[sel]
    init = getattr(vol, "init", None)
    if init is not None:
        init = np.asarray(init)[sel]
    part = types.SimpleNamespace(mask=sub.astype(np.uint8), signal=sig, bvals=vol.bvals, bvecs=vol.bvecs, init=init,
                                 norm_count=int(mask.sum()))
    return part, sel


def run_sharded_patches(vol, fit_fn, patch_dim, rank=0, world=1, group=None):
    """Fits this rank's patches of one volume with fit_fn(part) -> [V_part, Q] parameters
    (rows in the part's mask order) and returns the whole volume's [V, Q] parameters in mask
    order on every rank (torch.distributed all_gather_object, any backend)."""
    part, sel = shard_volume(vol, patch_dim, rank, world)
    theta = np.asarray(fit_fn(part)) if sel.size else None
    n = int(np.asarray(vol.mask).astype(bool).sum())
    pieces = [(sel, theta)]
    if world > 1:
        import torch.distributed as dist
        pieces = [None] * world
        dist.all_gather_object(pieces, (sel, theta), group=group)
    out = None
    seen = np.zeros(n, dtype=bool)
    for s, th in pieces:
        if th is None:
            continue
        if out is None:
            out = np.empty((n, th.shape[1]), dtype=th.dtype)
        if seen[s].any():
            raise RuntimeError("a voxel was fitted on two ranks")
        seen[s] = True
        out[s] = th
    if not seen.all():
        raise RuntimeError("some voxels were not fitted")
    return out


def fit_patches_on_this_gpu(opts, n_iters):
    """fit_fn for run_sharded_patches: one library fit of this rank's part of the volume."""
    def fn(part):
        from . import Fitter
        f = Fitter([part], opts)
        f.step(n_iters)
        f.sync()
        theta = f.params_host()
        f.close()
        return theta
    return fn
