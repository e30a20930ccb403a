"""Parity of the CUDA rollout path (through the C ABI) with the CPU oracle.

Win counts and step totals are integers and must match bit for bit; win probabilities
and odds are one binary32 division each and must match bit for bit as well.
"""
import numpy as np
import pytest

import oracle
from paper_2108_02419_gb300 import workloads as W
from tests.test_oracle_race import ENUM_CASES

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bbe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_02419_gb300 import bbe as B
    from paper_2108_02419_gb300 import build

    build.build()
    oracle.build()
    B.lib()
    return B


def run_gpu(bbe, rb, cfg=None):
    with bbe.Batch(rb) as b:
        if cfg:
            b.set_cfg(**cfg)
        counts, steps = b.rollout()
        probs, odds = b.win_probs(counts)
        b.status()
        torch.cuda.synchronize()
        return counts.cpu().numpy(), steps.cpu().numpy(), probs.cpu().numpy(), odds.cpu().numpy()


def assert_matches_oracle(rb, counts, steps, probs=None, races=None, max_steps=oracle.MAX_STEPS_DEFAULT):
    races = list(range(rb.n_races)) if races is None else list(races)
    want_c, want_s, _ = oracle.batch_counts(rb, races=races, max_steps=max_steps)
    got_c = np.concatenate([counts[rb.race_off[r]:rb.race_off[r + 1]] for r in races])
    assert np.array_equal(got_c, want_c), (got_c[:40], want_c[:40])
    assert np.array_equal(steps[races], want_s)
    if probs is not None:
        pos = 0
        for r in races:
            a, e = rb.race_off[r], rb.race_off[r + 1]
            wp, wo = oracle.win_probs(want_c[pos:pos + e - a], int(rb.rollouts[r]))
            assert np.array_equal(probs[a:e], wp)
            pos += e - a


def test_single_race_from_start(bbe):
    rb = W.single_race_start()  # 5 competitors, L 2000, 1000 rollouts, seed 0
    counts, steps, probs, odds = run_gpu(bbe, rb)
    assert counts.sum() == 1000
    assert_matches_oracle(rb, counts, steps, probs)
    assert np.all(odds[counts > 0] == np.float32(1.0) / probs[counts > 0])
    assert np.all(np.isinf(odds[counts == 0]))


def test_uniform_batch_small(bbe):
    rb = W.uniform_batch(n_races=64, rollouts=1000)
    counts, steps, probs, _ = run_gpu(bbe, rb)
    assert_matches_oracle(rb, counts, steps, probs)


def test_uneven_batch_small(bbe):
    # every competitor count 2..24, ragged rollout budgets spanning many work items
    rb = W.uneven_batch(seed=3, n_races=240, r_lo_exp=1.0, r_hi_exp=3.0)
    counts, steps, probs, _ = run_gpu(bbe, rb)
    assert_matches_oracle(rb, counts, steps, probs)


@pytest.mark.parametrize("slots", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 11, 12, 13, 16, 17, 20, 21, 22, 23, 24, 31, 32])
def test_every_segment_packing(bbe, n, slots):
    # one or two competitors per lane, every segment width and odd/even counts
    rb = W.uneven_batch(seed=100 + n, n_races=3, n_lo=n, n_hi=n, rollouts=333, rem_lo=50.0, rem_hi=900.0)
    counts, steps, probs, _ = run_gpu(bbe, rb, {"slots_per_lane": slots})
    assert_matches_oracle(rb, counts, steps, probs)


@pytest.mark.parametrize("case", range(len(ENUM_CASES)))
def test_enumerated_two_point_races(bbe, case):
    L, d0, mu, sigma, P, theta = ENUM_CASES[case]
    rb = W.from_arrays([len(d0)], L, 200000, d0, mu, sigma, [0.5] * len(d0), P=P, theta=theta, seed=11,
                       dist=W.DIST_TWO_POINT)
    rb.race_id0 = case
    counts, steps, _, _ = run_gpu(bbe, rb)
    assert_matches_oracle(rb, counts, steps)


@pytest.mark.parametrize("slots", [1, 2, 3, 4])
@pytest.mark.parametrize("dist", [W.DIST_UNIFORM, W.DIST_TWO_POINT])
def test_other_distributions(bbe, dist, slots):
    rb = W.uneven_batch(seed=7, n_races=40, rollouts=500, rem_lo=100.0, rem_hi=1500.0)
    rb.dist = dist
    counts, steps, probs, _ = run_gpu(bbe, rb, {"slots_per_lane": slots})
    assert_matches_oracle(rb, counts, steps, probs)


@pytest.mark.parametrize("slots", [1, 2, 3, 4])
def test_heavy_blocking_ties_and_given_inputs(bbe, slots):
    # start-line races (all positions equal) with large thresholds, explicit preference
    # and previous steps: the blocked branch, equal-position ties and delta_min dominate
    rng = np.random.default_rng(5)
    sizes = [4, 9, 20, 32]
    nt = sum(sizes)
    rb = W.from_arrays(sizes, [300.0, 250.0, 400.0, 200.0], [700, 500, 300, 200], np.zeros(nt),
                       rng.uniform(15, 17, nt), rng.uniform(0.5, 1.5, nt), rng.uniform(0, 1, nt),
                       P=rng.uniform(0.8, 1.0, nt), theta=rng.uniform(2.0, 8.0, nt), prev0=rng.uniform(10, 20, nt),
                       seed=99)
    counts, steps, probs, _ = run_gpu(bbe, rb, {"slots_per_lane": slots})
    assert_matches_oracle(rb, counts, steps, probs)


def test_launch_shape_does_not_change_counts(bbe):
    rb = W.uneven_batch(seed=8, n_races=60, r_lo_exp=1.5, r_hi_exp=3.0)
    ref = run_gpu(bbe, rb)
    for cfg in ({"warps_per_block": 1, "blocks_per_sm": 1, "rollouts_per_lane": 1},
                {"slots_per_lane": 1}, {"slots_per_lane": 2}, {"slots_per_lane": 3}, {"slots_per_lane": 4},
                {"warps_per_block": 16, "blocks_per_sm": 2, "rollouts_per_lane": 1000},
                {"warps_per_block": 4, "blocks_per_sm": 16, "rollouts_per_lane": 7}):
        got = run_gpu(bbe, rb, cfg)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_race_id_offset_reproduces_slices(bbe):
    rb = W.uneven_batch(seed=9, n_races=50, rollouts=400)
    whole = run_gpu(bbe, rb)
    a = run_gpu(bbe, rb.slice(0, 20))
    b = run_gpu(bbe, rb.slice(20, 50))
    assert np.array_equal(np.concatenate([a[0], b[0]]), whole[0])
    assert np.array_equal(np.concatenate([a[1], b[1]]), whole[1])


def test_graph_replay_and_new_buffers(bbe):
    rb = W.uneven_batch(seed=10, n_races=30, rollouts=300)
    with bbe.Batch(rb) as b:
        c1, s1 = b.rollout()
        c1 = c1.clone()
        b.rollout(c1.new_empty(c1.shape), s1.new_empty(s1.shape))  # new pointers: new graph
        c2, s2 = b.rollout()
        torch.cuda.synchronize()
        assert torch.equal(c1, c2) and torch.equal(s1, s2)
        c3, _ = b.rollout(steps=None, counts=torch.empty_like(c1))
        torch.cuda.synchronize()
        assert torch.equal(c1, c3)


def test_step_limit_status(bbe):
    rb = W.from_arrays([2], 1000.0, 50, [0.0, 1.0], [1.0, 1.0], [0.1, 0.1], [0.5, 0.5], seed=1)
    with bbe.Batch(rb) as b:
        b.set_cfg(max_steps=100)
        counts, steps = b.rollout()
        with pytest.raises(bbe.BbeError) as ei:
            b.status()
        assert ei.value.status == -5
        c, s = counts.cpu().numpy(), steps.cpu().numpy()
    want_c, want_s, st = oracle.batch_counts(rb, max_steps=100)
    assert st == oracle.STEP_LIMIT
    assert np.array_equal(c, want_c) and np.array_equal(s, want_s)


def test_autotune_keeps_counts(bbe):
    # the tuner picks a layout per competitor count and a launch shape; counts stay those of
    # the oracle whatever it picks
    rb = W.uneven_batch(seed=12, n_races=200, r_lo_exp=2.0, r_hi_exp=3.0)
    with bbe.Batch(rb) as b:
        scratch = torch.empty(rb.n_total, dtype=torch.int32, device="cuda")
        cfg = b.autotune(scratch, budget_ms=5000.0)
        assert 1 <= cfg["warps_per_block"] <= 16 and cfg["rollouts_per_lane"] >= 1 and cfg["slots_per_lane"] == 0
        tab = b.layout()
        assert tab[0] == 0 and np.all((tab[1:] >= 1) & (tab[1:] <= 4))
        counts, steps = b.rollout()
        b.status()
        torch.cuda.synchronize()
        assert_matches_oracle(rb, counts.cpu().numpy(), steps.cpu().numpy())


def test_mixed_layout_table(bbe):
    # every layout in one pass (one persistent launch per layout, forked in one graph), on a
    # repeated pass too (the graph replay)
    rb = W.uneven_batch(seed=14, n_races=120, n_lo=1, n_hi=32, rollouts=600)
    tab = np.zeros(33, np.int32)
    for n in range(1, 33):
        tab[n] = (1, 3, 4, 2)[n % 4]
    with bbe.Batch(rb) as b:
        b.set_layout(tab)
        ns = np.arange(1, 33)
        assert np.array_equal(b.layout()[1:], np.where(tab[1:] > ns, np.minimum(ns, 2), tab[1:]))
        assert bbe.bbe_batch_launches(b.handle) == 4
        for _ in range(2):
            counts, steps = b.rollout()
            b.status()
        torch.cuda.synchronize()
        got_c, got_s = counts.cpu().numpy(), steps.cpu().numpy()
    assert_matches_oracle(rb, got_c, got_s)


@pytest.mark.parametrize("mutate,code", [
    ("size0", -2), ("size33", -2), ("finished", -3), ("nan", -1), ("rho", -1), ("nonmono", -1), ("R0", -1),
    ("negpos", -1), ("pref0", -1), ("theta_neg", -1), ("prev0", -1), ("mu0", -1),
])
def test_validation_errors(bbe, mutate, code):
    rb = W.uneven_batch(seed=13, n_races=4, n_lo=3, n_hi=3, rollouts=10)
    off, L, R = rb.race_off.copy(), rb.L.copy(), rb.rollouts.copy()
    d0, mu, sigma, rho, P, th = rb.d0.copy(), rb.mu.copy(), rb.sigma.copy(), rb.rho.copy(), rb.P.copy(), rb.theta.copy()
    prev = None
    if mutate == "size0":
        off = np.array([0, 3, 3, 6, 9], np.int32)
    elif mutate == "size33":
        off = np.array([0, 33], np.int32)
        L = L[:1]; R = R[:1]
        d0, mu, sigma, rho, P, th = (np.resize(a, 33) for a in (d0, mu, sigma, rho, P, th))
    elif mutate == "finished":
        d0[4] = L[1]
    elif mutate == "nan":
        sigma[2] = np.nan
    elif mutate == "rho":
        rho[0] = 1.5
    elif mutate == "nonmono":
        off = np.array([0, 6, 3, 9, 12], np.int32)
    elif mutate == "R0":
        R[2] = 0
    elif mutate == "negpos":
        d0[0] = -1.0
    elif mutate == "pref0":
        P[1] = 0.0
    elif mutate == "theta_neg":
        th[1] = -0.5
    elif mutate == "prev0":
        prev = np.ones_like(mu)
        prev[5] = 0.0
    elif mutate == "mu0":
        mu[3] = 0.0
    n_races = off.size - 1
    with pytest.raises(bbe.BbeError) as ei:
        bbe.bbe_race_init(n_races, off, L, R, d0, mu, sigma, rho, P, th, prev, 0, 0, 0)
    assert ei.value.status == code
    assert bbe.bbe_last_error()


def test_device_pointers_accepted(bbe):
    rb = W.uneven_batch(seed=14, n_races=10, rollouts=200)
    dev = lambda a: None if a is None else torch.from_numpy(a).cuda()
    h = bbe.bbe_race_init(rb.n_races, dev(rb.race_off), dev(rb.L), dev(rb.rollouts), dev(rb.d0), dev(rb.mu),
                          dev(rb.sigma), dev(rb.rho), dev(rb.P), dev(rb.theta), None, rb.seed, rb.dist, 0)
    try:
        counts = torch.empty(rb.n_total, dtype=torch.int32, device="cuda")
        steps = torch.empty(rb.n_races, dtype=torch.int64, device="cuda")
        bbe.bbe_rollout_batch(h, counts, steps)
        bbe.bbe_batch_status(h)
        info = bbe.bbe_batch_info(h)
        assert info["n_races"] == 10 and info["n_competitors"] == rb.n_total
        assert info["total_rollouts"] == int(rb.rollouts.sum())
    finally:
        bbe.bbe_destroy_batch(h)
    assert_matches_oracle(rb, counts.cpu().numpy(), steps.cpu().numpy())


@pytest.mark.slow
def test_full_uniform_batch_sampled(bbe):
    # 4096 snapshots x 20 competitors x 10,000 rollouts in the benchmark's launch shape;
    # the oracle recomputes a sample of races one by one
    rb = W.uniform_batch()
    counts, steps, probs, _ = run_gpu(bbe, rb)
    sums = np.add.reduceat(counts, rb.race_off[:-1])
    assert np.all(sums == 10000)
    rng = np.random.default_rng(0)
    sample = [0, rb.n_races - 1] + list(rng.choice(rb.n_races, 4, replace=False))
    assert_matches_oracle(rb, counts, steps, probs, races=sample)


@pytest.mark.slow
def test_full_uneven_batch_sampled(bbe):
    # 10,000 snapshots, 2..24 competitors, budgets 1e3..1e5 in one persistent launch
    rb = W.uneven_batch()
    counts, steps, probs, _ = run_gpu(bbe, rb)
    sums = np.add.reduceat(counts, rb.race_off[:-1])
    assert np.all(sums == rb.rollouts)
    cheap = np.argsort(rb.rollouts * rb.sizes())[:6]
    rng = np.random.default_rng(1)
    sample = sorted(set(cheap.tolist() + rng.choice(rb.n_races, 2, replace=False).tolist()))
    assert_matches_oracle(rb, counts, steps, probs, races=sample)


def test_automatic_layout_follows_batch_size(bbe):
    # a batch too small to give every warp of the GPU an item runs one competitor per lane (its
    # steps' latency decides); a large one runs two; the counts do not depend on it
    small = W.single_race_start(seed=0)
    with bbe.Batch(small) as b:
        assert b.layout()[5] == 1
        counts, steps = b.rollout()
        b.status()
        c1, s1 = counts.cpu().numpy(), steps.cpu().numpy()
        b.set_cfg(slots_per_lane=2)
        counts, steps = b.rollout()
        b.status()
        assert np.array_equal(counts.cpu().numpy(), c1) and np.array_equal(steps.cpu().numpy(), s1)
    assert_matches_oracle(small, c1, s1)
    with bbe.Batch(W.uniform_batch(seed=0, n_races=1024, rollouts=2000)) as b:
        assert b.layout()[20] == 2
