"""Multi-rank host logic on CPU: volume assignment and result merge with two gloo ranks.

The per-volume fit is replaced by a deterministic CPU digest, so this covers the sharding
and gathering of run_sharded (no GPU, no collective on the data path)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import phantoms as P
from paper_2604_00250_gb300 import shard


def _digest(vols):
    return [float(np.float64(v.signal).sum()) + 1e-3 * v.n_meas for v in vols]


def _volumes():
    out = []
    for i, (shape, sch) in enumerate([((4, 4, 3), P.scheme_96(1)), ((6, 5, 4), P.make_scheme(2, [(1000, 8)], 2)),
                                      ((3, 3, 3), P.scheme_96(3)), ((5, 5, 5), P.make_scheme(3, [(2000, 12)], 4)),
                                      ((2, 4, 6), P.make_scheme(1, [(800, 6)], 5))]):
        out.append(P.random_volume(shape, scheme=sch, seed=i, mask_density=0.7))
    return out


def test_assignment_is_balanced_and_complete():
    costs = [100, 90, 80, 70, 10, 5, 5]
    owner, load = shard.assign_volumes(costs, 3)
    assert sorted(set(owner)) == [0, 1, 2]
    assert sum(load) == sum(costs)
    assert max(load) <= 4 / 3 * (sum(costs) / 3) + max(costs)
    owner1, _ = shard.assign_volumes(costs, 1)
    assert owner1 == [0] * len(costs)


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
        res = shard.run_sharded(_volumes(), _digest, rank=rank, world=world)
        q.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_single_rank():
    vols = _volumes()
    ref = shard.run_sharded(vols, _digest)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, res in got:
        assert sorted(res) == list(range(len(vols)))
        for k in ref:
            assert res[k] == pytest.approx(ref[k], rel=0, abs=0)
