"""Multi-rank host logic on the CPU: two gloo ranks each run their share of the races
(with the oracle standing in for the device) and their counts equal one run over the union.
Races are independent and the stream is counter-based, so any split is exact."""
import os

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2108_02419_gb300 import workloads as W


def _base():
    return W.uneven_batch(seed=21, n_races=12, n_lo=2, n_hi=9, rollouts=150, rem_lo=100.0, rem_hi=600.0)


def _worker(rank, world, port, mode, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle

    rb = _base()
    mine = W.for_rank(rb, rank) if mode == "weak" else W.shard(rb, rank, world)
    counts, steps, st = oracle.batch_counts(mine, threads=1)
    gathered = [None] * world
    dist.all_gather_object(gathered, (mine.race_id0, mine.n_races, counts.tolist(), steps.tolist(), st))
    if rank == 0:
        out.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def _run(mode, port):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("mode,port", [("weak", 29561), ("strong", 29562)])
def test_two_rank_split_equals_union(oracle_lib, mode, port):
    res = _run(mode, port)
    rb = _base()
    if mode == "weak":
        union = W.concat([rb, rb])  # ids 0 .. 2n-1: rank 1's races are rank 0's with new ids
        assert [r[0] for r in res] == [0, rb.n_races]
    else:
        union = rb
        assert res[0][1] + res[1][1] == rb.n_races and res[1][0] == res[0][1]
    want_c, want_s, _ = oracle_lib.batch_counts(union)
    got_c = np.concatenate([np.array(r[2], np.int32) for r in res])
    got_s = np.concatenate([np.array(r[3], np.int64) for r in res])
    assert np.array_equal(got_c, want_c) and np.array_equal(got_s, want_s)
    if mode == "weak":
        n = rb.n_total
        assert not np.array_equal(got_c[:n], got_c[n:])  # distinct races per rank
