"""Multi-rank host logic on CPU with two gloo ranks: the sharding of volumes and of one
volume's patches, and the merge of the results, with the FP64 oracle doing each rank's fit.

- volumes: a batch split by whole volumes (each its own sigma / calibration group) and fitted
  rank by rank gives every volume's parameters of the single-rank fit, bitwise;
- patches of one volume (MSE, no calibration, neighbour priors inside patches): each rank fits
  the volume restricted to its patches with the whole volume's |M| as normaliser (Eq. 8), and
  the merged parameters equal the single-rank fit of the whole volume, bitwise.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import phantoms as P
from oracle import prism_oracle as O
from paper_2604_00250_gb300 import shard

K = 3
ITERS = 3
PATCH = 4
OPTS = dict(K=K, patch_dim=PATCH, lam_sp=0.01, lam_dir=0.005)


def _volumes():
    out = []
    for i, (shape, sch) in enumerate([((4, 4, 3), P.scheme_96(1)), ((6, 5, 4), P.make_scheme(2, [(1000, 8)], 2)),
                                      ((3, 3, 3), P.scheme_96(3)), ((5, 5, 5), P.make_scheme(3, [(2000, 12)], 4)),
                                      ((2, 4, 6), P.make_scheme(1, [(800, 6)], 5))]):
        out.append(P.random_volume(shape, scheme=sch, seed=i, mask_density=0.7))
    return out


def _oracle_fit_volumes(vols):
    """fit_fn for run_sharded: the oracle's fit of each volume (NLL with sigma per volume)."""
    o = O.Options(loss="nll", **OPTS)
    out = []
    for i, v in enumerate(vols):
        ov = O.OracleVolume(v.mask, v.signal, v.bvals, v.bvecs, o)
        th0 = P.default_init(v.n_vox, K, 100 + v.n_meas)
        res = O.fit([ov], [torch.as_tensor(th0).double()], ITERS)
        out.append(res.theta[0].numpy())
    return out


def _sharded_volume():
    return P.random_volume((11, 9, 8), seed=7, mask_density=0.7)


def _oracle_fit_part(vol):
    """fit_fn for run_sharded_patches: the oracle's fit of the patches a part keeps, with the
    whole volume's normaliser (the oracle's patch selection keeps |M| of the full mask)."""
    th0 = P.default_init(vol.n_vox, K, 3)

    def fn(part):
        ids = np.unique(shard.patch_of_voxels(part.mask, PATCH))
        ov = O.OracleVolume(vol.mask, vol.signal, vol.bvals, vol.bvecs, O.Options(**OPTS), patches=ids)
        assert ov.n_mask == part.norm_count
        res = O.fit([ov], [torch.as_tensor(th0[ov.sel]).double()], ITERS)
        return res.theta[0].numpy()
    return fn, th0


def test_assignment_is_balanced_and_complete():
    costs = [100, 90, 80, 70, 10, 5, 5]
    owner, load = shard.assign_volumes(costs, 3)
    assert sorted(set(owner)) == [0, 1, 2]
    assert sum(load) == sum(costs)
    assert max(load) <= 4 / 3 * (sum(costs) / 3) + max(costs)
    owner1, _ = shard.assign_volumes(costs, 1)
    assert owner1 == [0] * len(costs)


def test_patch_assignment_covers_every_voxel_once():
    vol = _sharded_volume()
    sels = [shard.shard_volume(vol, PATCH, r, 3)[1] for r in range(3)]
    allv = np.concatenate(sels)
    assert np.array_equal(np.sort(allv), np.arange(vol.n_vox))
    _, _, load = shard.assign_patches(vol.mask, PATCH, 3)
    assert sum(load) == vol.n_vox and max(load) - min(load) <= PATCH ** 3
    part, sel = shard.shard_volume(vol, PATCH, 1, 3)
    assert part.norm_count == vol.n_vox and int(part.mask.sum()) == sel.size
    np.testing.assert_array_equal(part.signal, vol.signal[sel])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        by_volume = shard.run_sharded(_volumes(), _oracle_fit_volumes, rank=rank, world=world)
        vol = _sharded_volume()
        fn, _ = _oracle_fit_part(vol)
        by_patch = shard.run_sharded_patches(vol, fn, PATCH, rank=rank, world=world)
        q.put((rank, by_volume, by_patch))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_single_rank():
    vols = _volumes()
    ref_vol = shard.run_sharded(vols, _oracle_fit_volumes)
    vol = _sharded_volume()
    fn, th0 = _oracle_fit_part(vol)
    ov = O.OracleVolume(vol.mask, vol.signal, vol.bvals, vol.bvecs, O.Options(**OPTS))
    ref_patch = O.fit([ov], [torch.as_tensor(th0).double()], ITERS).theta[0].numpy()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, by_volume, by_patch in got:
        assert sorted(by_volume) == list(range(len(vols)))
        for k in ref_vol:
            assert np.array_equal(by_volume[k], ref_vol[k]), (rank, k)
        assert np.array_equal(by_patch, ref_patch), (rank, float(np.abs(by_patch - ref_patch).max()))
