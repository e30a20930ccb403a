"""Runs the rollout paths on the checked build of the library (every computed device index
checked, a failure recorded in the batch status) and compares them with the oracle; started by
tests/test_gpu_checked_build.py with BBE_LIB naming the checked build."""
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import oracle  # noqa: E402
from paper_2108_02419_gb300 import bbe  # noqa: E402
from paper_2108_02419_gb300 import workloads as W  # noqa: E402

assert bbe.LIB_PATH == os.environ["BBE_LIB"], bbe.LIB_PATH
rng = np.random.default_rng(90)
sizes = list(range(1, 33))
nt = sum(sizes)
heavy = W.from_arrays(sizes, 300.0, 64, rng.uniform(0, 40, nt), rng.uniform(15, 17, nt), rng.uniform(0.5, 1.5, nt),
                      rng.uniform(0, 1, nt), theta=rng.uniform(1.0, 6.0, nt), seed=91)
uneven = W.uneven_batch(seed=92, n_races=30, n_lo=1, n_hi=12, rollouts=200, rem_lo=100.0, rem_hi=1200.0)
checks = 0
for rb in (heavy, uneven):
    want_c, want_s, st = oracle.batch_counts(rb)
    want_p, want_ps, _ = oracle.batch_places(rb, 3)
    for slots in (0, 1, 2, 3, 4):
        with bbe.Batch(rb) as b:
            if slots:
                b.set_cfg(slots_per_lane=slots)
            counts, steps = b.rollout()
            b.status()  # raises BBE_ERR_RANGE if an index check failed
            assert np.array_equal(counts.cpu().numpy(), want_c) and np.array_equal(steps.cpu().numpy(), want_s)
            pc, ps = b.places(3)
            b.status()
            assert np.array_equal(pc.cpu().numpy().ravel(), want_p.ravel()) and np.array_equal(ps.cpu().numpy(), want_ps)
            checks += 2
# ordered tallies and the order histogram
rb = uneven
want_o, _, _ = oracle.batch_orders(rb, 3)
want_h, _, _ = oracle.batch_order_histograms(rb, 32)
with bbe.Batch(rb) as b:
    orders, _, _ = b.orders(3)
    b.status()
    flat, pos = orders.cpu().numpy(), 0
    for r in range(rb.n_races):
        n = int(rb.race_off[r + 1] - rb.race_off[r])
        size = n ** min(3, n)
        assert np.array_equal(flat[pos:pos + size], want_o[r])
        pos += size
    keys, hc, off, _, _ = b.order_histogram(32)
    b.status()
    keys, hc = keys.cpu().numpy(), hc.cpu().numpy()
    for r in range(rb.n_races):
        n = int(rb.race_off[r + 1] - rb.race_off[r])
        k, c = keys[off[r]:off[r + 1]], hc[off[r]:off[r + 1]]
        used = k != np.uint64(2 ** 64 - 1)
        got = {tuple(int(x) for x in bbe.bbe_order_key_decode(n, 32, int(key))): int(v) for key, v in zip(k[used], c[used])}
        assert got == dict(want_h[r]), r
    checks += 2
# the time law, a single small race (one rollout per warp) and the no-allocation entry point
tl = W.with_time_law(W.uneven_batch(seed=93, n_races=12, n_lo=2, n_hi=9, rollouts=200), 30.0, 200.0)
single = W.single_race_start(rollouts=500)
for rb in (tl, single):
    want_c, want_s, _ = oracle.batch_counts(rb)
    with bbe.Batch(rb) as b:
        counts, steps = b.rollout()
        b.status()
        assert np.array_equal(counts.cpu().numpy(), want_c) and np.array_equal(steps.cpu().numpy(), want_s)
        checks += 1
rb = uneven
dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
counts = torch.empty(rb.n_total, dtype=torch.int32, device="cuda")
steps = torch.empty(rb.n_races, dtype=torch.int64, device="cuda")
bbe.bbe_rollout_noalloc(rb.n_races, rb.n_total, dev(rb.race_off), dev(rb.L), dev(rb.rollouts), dev(rb.d0), dev(rb.mu),
                        dev(rb.sigma), dev(rb.rho), dev(rb.P), dev(rb.theta), None, rb.seed, rb.dist, rb.race_id0,
                        counts, steps)
want_c, want_s, _ = oracle.batch_counts(rb)
assert np.array_equal(counts.cpu().numpy(), want_c) and np.array_equal(steps.cpu().numpy(), want_s)
checks += 1
print("checked build ok:", checks, "passes, no index check failed, all equal to the oracle")
