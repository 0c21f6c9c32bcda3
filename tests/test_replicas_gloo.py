"""The multi-rank path on the CPU: two gloo ranks (one process each, 127.0.0.1 rendezvous).

Checks the collectives the benchmark uses (barrier, max over ranks of a timed region,
whole-job rate), the tube sharding (disjoint, covering, balanced, identical on every rank),
and that splitting a batch of Riemann tubes between ranks changes no result: each rank
runs its shard through the oracle and the gathered tubes equal a single-process run."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1210_5246_gb300 import inputs, replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _oracle_tubes(tb, idx):
    from oracle import oracle
    out = {}
    for k in idx:
        n = int(tb.length[k])
        g = oracle.Grid((n,), (0.0,), (1.0,), ((1, 1),), tb.cfl)
        U, steps, t, rc, _ = oracle.run(g, oracle.prim_to_cons(tb.initial_tube(k)), tb.t_end)
        assert rc == 0
        out[int(k)] = (U.reshape(10, n), steps)
    return out


def _small_tubes():
    tb = inputs.tubes(ntubes=12, nmin=8, nmax=64, seed=9)
    return tb


def _worker(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    assert replicas.init("gloo") and replicas.active()
    assert replicas.dist_env() == (rank, world, rank)
    replicas.barrier()
    # max over ranks of a timed region, whole-job rate (units / slowest rank's time)
    assert replicas.max_over_ranks(1.5 + rank) == 1.5 + world - 1
    assert replicas.sum_over_ranks(rank + 1) == world * (world + 1) / 2
    assert replicas.whole_job_rate(100.0, 2.0) == 100.0 * world / 2.0
    # every rank computes the same partition
    tb = _small_tubes()
    mine = replicas.shard_tubes(tb.length, rank, world)
    parts = [None] * world
    dist.all_gather_object(parts, mine.tolist())
    for r in range(world):
        assert parts[r] == replicas.shard_tubes(tb.length, r, world).tolist()
    res = _oracle_tubes(tb, mine)
    gathered = [None] * world
    dist.all_gather_object(gathered, {k: (v[0].tolist(), v[1]) for k, v in res.items()})
    if rank == 0:
        merged = {}
        for g in gathered:
            for k, (U, s) in g.items():
                assert k not in merged
                merged[k] = (np.array(U), s)
        np.save(os.path.join(outdir, "merged.npy"), np.array([merged], dtype=object), allow_pickle=True)
    replicas.barrier()
    dist.destroy_process_group()


def test_shard_tubes_partition_and_balance():
    tb = inputs.tubes()  # 4096 tubes, 128..2048 cells
    for world in (1, 2, 3, 4, 8):
        shards = [replicas.shard_tubes(tb.length, r, world) for r in range(world)]
        allidx = np.concatenate(shards)
        assert len(allidx) == len(tb.length) and len(np.unique(allidx)) == len(tb.length)
        assert all(np.all(np.diff(s) > 0) for s in shards)
        load = np.array([replicas.tube_cost(tb.length[s]).sum() for s in shards])
        # LPT: no rank exceeds the mean by more than the largest single tube
        assert load.max() - load.mean() <= replicas.tube_cost(tb.length).max()
        assert load.max() / load.mean() < 1.01
    with pytest.raises(ValueError):
        replicas.shard_tubes(tb.length, 2, 2)


def test_single_process_is_inactive():
    assert replicas.max_over_ranks(3.0) == 3.0
    assert replicas.whole_job_rate(10.0, 2.0) == 5.0


def test_two_gloo_ranks(oracle):
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_worker, args=(world, _free_port(), d), nprocs=world, join=True,
                           start_method="spawn")
        merged = np.load(os.path.join(d, "merged.npy"), allow_pickle=True)[0]
    tb = _small_tubes()
    assert sorted(merged) == list(range(len(tb.length)))
    ref = _oracle_tubes(tb, range(len(tb.length)))
    for k, (U, s) in merged.items():
        assert s == ref[k][1]
        np.testing.assert_array_equal(U, ref[k][0])
