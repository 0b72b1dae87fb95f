"""The N > 1 path on CPU: two gloo ranks, one process each.

The sampler shards into independent replicas with no exchange, so what a
multi-GPU run adds is host logic: which replicas a rank owns (disjoint, keyed
by the replica index), and the whole-job rate (units of all ranks over the
slowest rank's time).  Each rank here samples its replicas with the oracle
(the CPU statement of the same trajectories the GPU ranks produce) and the
parent checks the results against a serial re-run of every replica."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from paper_1508_07077_gb300 import replicas as R
from paper_1508_07077_gb300 import workloads as W

torch = pytest.importorskip("torch")

PER_RANK = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _system():
    return W.make_system("mr", W.SPHERE, 64, 0.2, 0.2, 0.2, seed=3)


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        ws, rk, _ = R.world()
        assert (ws, rk) == (world, rank)
        s = _system()
        ids = R.replica_ids(PER_RANK, rank)
        moves = 0
        results = {}
        for rid in ids:
            pos, _, cnt, _ = O.run(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=0.1, seed=1,
                                   replica=rid, n_sweeps=3)
            results[rid] = pos
            moves += cnt["moves"]
        # ranks take different (fake) times: the job is as slow as the slowest
        seconds = 1.0 + rank
        rate = R.world_rate(moves, seconds)
        gathered = [None] * world
        dist.all_gather_object(gathered, ids)
        out.put((rank, ids, gathered, results, moves, rate, R.reduce_max([seconds])[0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_replicas(oracle):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    all_ids = got[0][2]
    # disjoint replica sets, the same view on every rank
    assert got[1][2] == all_ids
    flat = [i for ids in all_ids for i in ids]
    assert sorted(flat) == list(range(2 * PER_RANK))
    # whole-job rate: total moves over the slowest rank (2 s)
    total = sum(g[4] for g in got)
    for g in got:
        assert g[6] == 2.0
        assert g[5] == pytest.approx(total / 2.0)
    # every replica's trajectory equals a serial re-run, and replicas differ
    s = _system()
    seen = []
    for g in got:
        for rid, pos in g[3].items():
            ref, _, _, _ = oracle.run(s.pos, s.L, q=s.q, n_r=s.n_r, d_max=0.1, seed=1,
                                      replica=rid, n_sweeps=3)
            assert np.array_equal(pos, ref)
            seen.append(pos)
    for a in range(len(seen)):
        for b in range(a + 1, len(seen)):
            assert not np.array_equal(seen[a], seen[b])


def test_single_process_reductions_are_identity():
    assert R.reduce_max([3.0, 1.0]) == [3.0, 1.0]
    assert R.reduce_sum([2.0]) == [2.0]
    assert R.world_rate(10.0, 4.0) == 2.5
    assert R.replica_ids(3, 2) == [6, 7, 8]
    with pytest.raises(ValueError):
        R.replica_ids(0, 1)
