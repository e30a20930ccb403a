"""Parity of the CUDA place-count path (bbe_place_counts through the C ABI) with the CPU
oracle's finishing-order rollouts: counts and step totals bit for bit, the first place
equal to the win counts of bbe_rollout_batch on the same stream."""
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


def run_places(bbe, rb, places, cfg=None, status=True):
    with bbe.Batch(rb) as b:
        if cfg:
            b.set_cfg(**cfg)
        counts, steps = b.places(places)
        if status:
            b.status()
        torch.cuda.synchronize()
        return counts.cpu().numpy(), steps.cpu().numpy()


def assert_places_match(rb, places, counts, steps, races=None, max_steps=oracle.MAX_STEPS_DEFAULT):
    races = list(range(rb.n_races)) if races is None else list(races)
    want_c, want_s, _ = oracle.batch_places(rb, places, races=races, max_steps=max_steps)
    got_c = np.concatenate([counts[rb.race_off[r]:rb.race_off[r + 1]] for r in races])
    assert np.array_equal(got_c, want_c), (got_c[:10], want_c[:10])
    assert np.array_equal(steps[races], want_s)


@pytest.mark.parametrize("places", [1, 3, 32])
def test_uneven_small_matches_oracle(bbe, places):
    rb = W.uneven_batch(seed=21, n_races=40, n_lo=1, n_hi=14, rollouts=300, rem_lo=100.0, rem_hi=1500.0)
    counts, steps = run_places(bbe, rb, places)
    assert counts.shape == (rb.n_total, places)
    assert_places_match(rb, places, counts, steps)


@pytest.mark.parametrize("dist", [W.DIST_UNIFORM, W.DIST_TWO_POINT])
def test_other_distributions_match_oracle(bbe, dist):
    rb = W.uneven_batch(seed=22, n_races=30, n_lo=2, n_hi=10, rollouts=300, rem_lo=100.0, rem_hi=1200.0)
    rb.dist = dist
    counts, steps = run_places(bbe, rb, 4)
    assert_places_match(rb, 4, counts, steps)


def test_every_segment_packing_and_heavy_blocking(bbe):
    # n = 1..32 covers every segment count per warp; start-line races with large thresholds,
    # given preferences and previous steps exercise blocking and equal positions
    rng = np.random.default_rng(23)
    sizes = list(range(1, 33))
    nt = sum(sizes)
    rb = W.from_arrays(sizes, 250.0, 64, np.zeros(nt), rng.uniform(15, 17, nt), rng.uniform(0.5, 1.5, nt),
                       rng.uniform(0, 1, nt), P=rng.uniform(0.8, 1.0, nt), theta=rng.uniform(2.0, 8.0, nt),
                       prev0=rng.uniform(10, 20, nt), seed=98)
    for places in (2, 32):
        counts, steps = run_places(bbe, rb, places)
        assert_places_match(rb, places, counts, steps)


def test_enumerated_two_point_races(bbe):
    rbs = []
    for i, (L, d0, mu, sigma, P, theta) in enumerate(ENUM_CASES):
        rbs.append(W.from_arrays([len(d0)], L, 4000, d0, mu, sigma, [0.5] * len(d0), P=P, theta=theta, seed=17,
                                 dist=W.DIST_TWO_POINT))
    rb = W.concat(rbs)
    counts, steps = run_places(bbe, rb, 3)
    assert_places_match(rb, 3, counts, steps)


def test_first_place_is_the_win_count(bbe):
    rb = W.uneven_batch(seed=24, n_races=1500, rollouts=2000)
    with bbe.Batch(rb) as b:
        wins, wsteps = b.rollout()
        pc, psteps = b.places(1)
        pc3, _ = b.places(3)
        b.status()
        torch.cuda.synchronize()
        wins, wsteps, pc, psteps, pc3 = (x.cpu().numpy() for x in (wins, wsteps, pc, psteps, pc3))
    assert np.array_equal(pc[:, 0], wins) and np.array_equal(psteps, wsteps)
    assert np.array_equal(pc3[:, 0], wins)
    col = np.add.reduceat(pc3, rb.race_off[:-1], axis=0)
    filled = np.arange(3)[None, :] < rb.sizes()[:, None]  # places that exist in each race
    assert np.all(np.where(filled, col == rb.rollouts[:, None], col == 0))


def test_place_probs(bbe):
    rb = W.uneven_batch(seed=25, n_races=50, n_lo=2, n_hi=12, rollouts=700)
    with bbe.Batch(rb) as b:
        counts, _ = b.places(3)
        wins, _ = b.rollout()
        wp, _ = b.win_probs(wins)
        p1 = b.place_probs(counts, 1)
        p3 = b.place_probs(counts, 3)
        with pytest.raises(bbe.BbeError):
            b.place_probs(counts, 4)
        torch.cuda.synchronize()
        counts, wp, p1, p3 = (x.cpu().numpy() for x in (counts, wp, p1, p3))
    assert np.array_equal(p1, wp)
    R = np.repeat(rb.rollouts, rb.sizes()).astype(np.float32)
    assert np.array_equal(p3, counts.sum(1).astype(np.float32) / R)


def test_step_limit_counts_for_nobody(bbe):
    rb = W.from_arrays([3], 1000.0, 40, [0.0, 1.0, 2.0], [1.0, 1.0, 9.0], [0.1, 0.1, 0.1], [0.5] * 3, seed=3)
    with bbe.Batch(rb) as b:
        b.set_cfg(max_steps=150)
        counts, steps = b.places(3)
        with pytest.raises(bbe.BbeError) as ei:
            b.status()
        assert ei.value.status == -5
        c, s = counts.cpu().numpy(), steps.cpu().numpy()
    want_c, want_s, st = oracle.batch_places(rb, 3, max_steps=150)
    assert st == oracle.STEP_LIMIT
    assert np.array_equal(c, want_c) and np.array_equal(s, want_s)
    # the fast competitor crosses within the limit, the other two do not: every rollout
    # to the third place is cut off and counts for nobody; to the first place none is
    assert c.sum() == 0 and s[0] == 40 * 150
    with bbe.Batch(rb) as b:
        b.set_cfg(max_steps=150)
        c1, _ = b.places(1)
        b.status()
        c1 = c1.cpu().numpy()
    assert c1[2, 0] == 40 and c1.sum() == 40


def test_bad_arguments(bbe):
    rb = W.uneven_batch(seed=26, n_races=3, rollouts=10)
    with bbe.Batch(rb) as b:
        out = torch.empty((rb.n_total, 33), dtype=torch.int32, device="cuda")
        for places in (0, 33):
            with pytest.raises(bbe.BbeError) as ei:
                bbe.bbe_place_counts(b.handle, places, out)
            assert ei.value.status == -1


@pytest.mark.slow
def test_full_uniform_batch_sampled(bbe):
    # 4096 snapshots x 20 competitors x 10,000 rollouts to the third finisher, launch shape
    # of the benchmark; the oracle recomputes a sample of races one by one
    rb = W.uniform_batch()
    counts, steps = run_places(bbe, rb, 3)
    col = np.add.reduceat(counts, rb.race_off[:-1], axis=0)
    assert np.all(col == 10000)
    rng = np.random.default_rng(2)
    sample = [0, rb.n_races - 1] + list(rng.choice(rb.n_races, 2, replace=False))
    assert_places_match(rb, 3, counts, steps, races=sample)


@pytest.mark.parametrize("slots", [1, 2, 3, 4])
def test_every_layout_matches_oracle(bbe, slots):
    # each competitors-per-lane layout of the place mode (races smaller than the layout take two,
    # or one for a lone competitor), to the third and to the last finisher, with heavy blocking
    rng = np.random.default_rng(24 + slots)
    sizes = [1, 2, 3, 5, 7, 11, 16, 20, 24, 32]
    nt = sum(sizes)
    rb = W.from_arrays(sizes, 300.0, 96, rng.uniform(0, 60, nt), rng.uniform(15, 17, nt), rng.uniform(0.5, 1.5, nt),
                       rng.uniform(0, 1, nt), theta=rng.uniform(1.0, 6.0, nt), seed=77)
    for places in (3, 32):
        counts, steps = run_places(bbe, rb, places, cfg={"slots_per_lane": slots})
        assert_places_match(rb, places, counts, steps)


def test_mixed_layout_table_matches_oracle(bbe):
    # a per-count layout table puts the races in four launches (one per layout) of the same pass
    rb = W.uneven_batch(seed=25, n_races=60, n_lo=1, n_hi=24, rollouts=200, rem_lo=100.0, rem_hi=1500.0)
    table = [0] + [1 + (n % 4) for n in range(1, 33)]
    with bbe.Batch(rb) as b:
        b.set_layout(table)
        counts, steps = b.places(5)
        b.status()
        counts, steps = counts.cpu().numpy(), steps.cpu().numpy()
    assert_places_match(rb, 5, counts, steps)
