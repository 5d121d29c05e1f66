"""Multi-rank host logic on CPU: two gloo ranks on 127.0.0.1 (no GPU).

Checks what the multi-GPU benchmark relies on: units partition exactly over
ranks, every rank draws its own batch, the job time is the slowest rank's,
and the reported throughput counts every rank's units once.
"""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as tmp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import synth
    from paper_2606_29692_gb300 import dist as tqd
    r, w = tqd.init("gloo")
    assert (r, w) == (rank, world)
    res = {}
    res["shards"] = [tqd.shard_range(n, rank, world) for n in (0, 1, 7, 8192, 8193)]
    # each rank's own synthetic batch
    _, _, k, th = synth.t5_batch(64, 204, seed=tqd.rank_seed(synth.SEED_T5_BATCH, rank))
    res["batch"] = (k.tolist(), th.tolist())
    # slowest rank wins; counts add
    t = 0.25 + rank
    res["tmax"] = tqd.max_over_ranks(t)
    res["units"] = tqd.sum_over_ranks(100 + rank)
    res["value"] = tqd.weak_scaling_value(8192, world, 10, res["tmax"])
    tqd.barrier()
    dist.destroy_process_group()
    out.put((rank, res))


def test_two_gloo_ranks():
    pytest.importorskip("torch.distributed")
    world = 2
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for i, n in enumerate((0, 1, 7, 8192, 8193)):
        lo0, hi0 = got[0]["shards"][i]
        lo1, hi1 = got[1]["shards"][i]
        assert lo0 == 0 and hi0 == lo1 and hi1 == n          # disjoint, covering
        assert abs((hi0 - lo0) - (hi1 - lo1)) <= 1          # balanced
    assert got[0]["batch"] != got[1]["batch"]                # own units per rank
    assert got[0]["tmax"] == got[1]["tmax"] == 1.25
    assert got[0]["units"] == got[1]["units"] == 201
    assert got[0]["value"] == pytest.approx(8192 * 2 * 10 / 1.25)


def test_single_rank_defaults():
    from paper_2606_29692_gb300 import dist as tqd
    assert tqd.shard_range(10, 0, 1) == (0, 10)
    assert tqd.max_over_ranks(3.5) == 3.5
    assert tqd.weak_scaling_value(8192, 1, 20, 2.0) == 8192 * 20 / 2.0
    assert tqd.rank_seed(3, 0) == 3 and tqd.rank_seed(3, 1) != 3
