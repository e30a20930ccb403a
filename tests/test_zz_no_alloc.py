"""bbe_rollout_noalloc: the rollout pass for callers that cannot allocate GPU memory.

Such callers (code inside a memory pool it does not own, a latency-bound loop where an
allocation could synchronise the device, a process whose allocator another framework holds)
pass device arrays in and get win counts out; the library keeps its work list in a fixed
device array instead of allocating.  These tests call the entry point through the C ABI and
check that, on two calls in a row with different batches, its counts and step totals equal
those of the allocating path (bbe_race_init + bbe_rollout_batch), bit for bit as every
count comparison in this suite is.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2108_02419_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bbe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_02419_gb300 import bbe as B
    from paper_2108_02419_gb300 import build

    build.build()
    B.lib()
    return B


def _dev(rb):
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return {k: t(getattr(rb, k)) for k in ("race_off", "L", "rollouts", "d0", "mu", "sigma", "rho", "P", "theta",
                                            "prev0")}


def _allocating(bbe, rb):
    with bbe.Batch(rb) as b:
        counts, steps = b.rollout()
        b.status()
        torch.cuda.synchronize()
        return counts.cpu().numpy(), steps.cpu().numpy()


def _noalloc(bbe, rb, counts=None, steps=None):
    a = _dev(rb)
    counts = torch.full((rb.n_total,), -7, dtype=torch.int32, device="cuda") if counts is None else counts
    steps = torch.full((rb.n_races,), -7, dtype=torch.int64, device="cuda") if steps is None else steps
    bbe.bbe_rollout_noalloc(rb.n_races, rb.n_total, a["race_off"], a["L"], a["rollouts"], a["d0"], a["mu"],
                            a["sigma"], a["rho"], a["P"], a["theta"], a["prev0"], rb.seed, rb.dist, rb.race_id0,
                            counts, steps)
    torch.cuda.synchronize()
    return counts.cpu().numpy(), steps.cpu().numpy()


def test_two_calls_match_allocating_path(bbe):
    first = W.uneven_batch(seed=31, n_races=300, r_lo_exp=1.5, r_hi_exp=3.5)  # sizes 2..24, ragged budgets
    second = W.uniform_batch(seed=32, n_races=40, n=20, rollouts=2000)        # smaller: stale items must not leak
    for rb in (first, second):
        want_c, want_s = _allocating(bbe, rb)
        got_c, got_s = _noalloc(bbe, rb)
        assert np.array_equal(got_c, want_c)
        assert np.array_equal(got_s, want_s)
        assert np.all(np.add.reduceat(got_c, rb.race_off[:-1]) == rb.rollouts)


def test_same_batch_twice_and_prev_step(bbe):
    rb = W.uneven_batch(seed=33, n_races=64, rollouts=700)
    rb.prev0 = (rb.mu * np.float32(0.9)).astype(np.float32)
    want = _allocating(bbe, rb)
    for _ in range(2):
        got = _noalloc(bbe, rb)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_rejects_more_races_than_the_scratch_holds(bbe):
    limit = 16384
    rb = W.uniform_batch(seed=34, n_races=limit + 1, n=2, rollouts=1)
    with pytest.raises(bbe.BbeError) as ei:
        _noalloc(bbe, rb)
    assert ei.value.status == -7 and "n_races" in bbe.bbe_last_error()


def test_rejects_host_memory_and_bad_states(bbe):
    rb = W.uneven_batch(seed=35, n_races=5, rollouts=10)
    a = _dev(rb)
    counts = torch.empty(rb.n_total, dtype=torch.int32, device="cuda")
    with pytest.raises(bbe.BbeError) as ei:  # host array where device memory is required
        bbe.bbe_rollout_noalloc(rb.n_races, rb.n_total, rb.race_off, a["L"], a["rollouts"], a["d0"], a["mu"],
                                a["sigma"], a["rho"], a["P"], a["theta"], None, 0, 0, 0, counts)
    assert ei.value.status == -1
    bad = W.uneven_batch(seed=35, n_races=5, rollouts=10)
    bad.d0[3] = bad.L[0]  # a competitor already at the line
    with pytest.raises(bbe.BbeError) as ei:
        _noalloc(bbe, bad)
    assert ei.value.status == -3
    # a valid call right after a rejected one still matches the allocating path
    want = _allocating(bbe, rb)
    got = _noalloc(bbe, rb)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_scratch_edges_match_allocating_path(bbe):
    # the most races the array takes (16,384 races of 2: at most 4 items each), one race of 32
    # competitors with a large budget (its items grow to keep the list short), and a mix with
    # lone competitors
    many = W.uniform_batch(seed=36, n_races=16384, n=2, rollouts=1000)
    big = W.uniform_batch(seed=37, n_races=1, n=32, rollouts=100000)
    mix = W.concat([W.uneven_batch(seed=38, n_races=30, n_lo=1, n_hi=1, rollouts=500),
                    W.uneven_batch(seed=39, n_races=30, n_lo=2, n_hi=32, rollouts=3000)])
    for rb in (many, big, mix):
        want_c, want_s = _allocating(bbe, rb)
        got_c, got_s = _noalloc(bbe, rb)
        assert np.array_equal(got_c, want_c)
        assert np.array_equal(got_s, want_s)


def test_reports_the_lowest_invalid_race(bbe):
    rb = W.uneven_batch(seed=40, n_races=50, rollouts=10)
    rb.sigma[rb.race_off[40]] = -1.0       # race 40: BBE_ERR_ARG
    rb.d0[rb.race_off[7] + 1] = rb.L[7]    # race 7: BBE_ERR_FINISHED, the lowest
    for _ in range(3):
        with pytest.raises(bbe.BbeError) as ei:
            _noalloc(bbe, rb)
        assert ei.value.status == -3
        assert "race 7 " in bbe.bbe_last_error()
