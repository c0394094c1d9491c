"""Sharding of independent fits across ranks (one process per GPU).

Volumes are independent optimisation problems -- each carries its own sigma and
calibration (Sec. 2.3) and neighbour priors never cross a volume -- so a batch is
split across ranks with no data-path collective: every rank fits its share on its own
GPU and the per-volume results are gathered once at the end.

Assignment is longest-processing-time first on cost = masked voxels x measurements,
which bounds the slowest rank's work by 4/3 of the optimum.
"""
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
