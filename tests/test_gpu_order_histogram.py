"""Parity of the CUDA finishing-order histogram (bbe_order_histogram through the C ABI) with the
CPU oracle: every race's set of (order, count) pairs equal to the tally of the oracle's
dry-runs, for the full order of all finishers and for the first K places, with the place counts
and step totals of the same pass equal to bbe_place_counts's; at the full 4096 x 20 x 10^4 size,
sampled races against the oracle and the table invariants on every race.  Keys are decoded here
from their definition in include/bbe.h (a lexicographic rank), not by the library."""
import math

import numpy as np
import pytest

import oracle
from paper_2108_02419_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
EMPTY = np.uint64(2 ** 64 - 1)


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


def decode(key: int, n: int, kk: int):
    digits = []
    for j in range(kk - 1, -1, -1):
        digits.append(key % (n - j))
        key //= n - j
    left, out = list(range(n)), []
    for a in reversed(digits):
        out.append(left.pop(a))
    return tuple(out)


def histograms(rb, keys, counts, off, places, races=None):
    """Per race: {ordered tuple: count} from its hash table, after checking the table."""
    out = []
    for r in (range(rb.n_races) if races is None else races):
        n = int(rb.race_off[r + 1] - rb.race_off[r])
        kk = min(places, n)
        k = keys[off[r]:off[r + 1]]
        c = counts[off[r]:off[r + 1]]
        cap = k.size
        assert cap >= 2 and cap & (cap - 1) == 0 and cap >= 2 * min(int(rb.rollouts[r]), math.perm(n, kk))
        used = k != EMPTY
        assert np.all(c[~used] == 0) and np.all(c[used] > 0)
        ku = k[used].astype(object)
        assert len(set(ku)) == ku.size  # each order once
        assert all(int(x) < math.perm(n, kk) for x in ku)
        out.append({decode(int(x), n, kk): int(v) for x, v in zip(ku, c[used])})
    return out


def run(bbe, rb, places, with_places=False):
    with bbe.Batch(rb) as b:
        keys, counts, off, pc, steps = b.order_histogram(places, with_places=with_places)
        b.status()
        torch.cuda.synchronize()
        res = (keys.cpu().numpy(), counts.cpu().numpy(), off, None if pc is None else pc.cpu().numpy(),
               steps.cpu().numpy())
        if with_places:
            pc2, steps2 = b.places(places)
            b.status()
            res += (pc2.cpu().numpy(), steps2.cpu().numpy())
    return res


@pytest.mark.parametrize("places", [32, 4, 1])
def test_uneven_small_matches_oracle(bbe, places):
    # sizes 1..9 with ragged budgets: the full order (places >= n) and the first four places
    rb = W.uneven_batch(seed=41, n_races=40, n_lo=1, n_hi=9, rollouts=400, rem_lo=100.0, rem_hi=1500.0)
    rb.rollouts = (rb.rollouts - np.arange(rb.n_races) * 7).astype(rb.rollouts.dtype)
    keys, counts, off, pc, steps, pc2, steps2 = run(bbe, rb, places, with_places=True)
    got = histograms(rb, keys, counts, off, places)
    want, want_s, st = oracle.batch_order_histograms(rb, places)
    assert st == 0
    for r in range(rb.n_races):
        assert got[r] == dict(want[r]), r
        assert sum(got[r].values()) == int(rb.rollouts[r])
    assert np.array_equal(steps, want_s)
    assert np.array_equal(pc, pc2) and np.array_equal(steps, steps2)


def test_full_order_of_twenty_matches_oracle(bbe):
    # 20-competitor snapshots late in the race, full order (20! orders: keys up to 2.4e18)
    rb = W.uniform_batch(seed=42, n_races=6, n=20, rollouts=1500)
    rb.d0 = (rb.d0 * np.float32(0.2) + np.float32(0.75 * 5000)).astype(np.float32)
    keys, counts, off, _, steps = run(bbe, rb, 20)
    got = histograms(rb, keys, counts, off, 20)
    want, want_s, st = oracle.batch_order_histograms(rb, 20)
    assert st == 0 and np.array_equal(steps, want_s)
    for r in range(rb.n_races):
        assert got[r] == dict(want[r]), r


def test_other_distributions_and_a_second_layout(bbe):
    rb = W.uneven_batch(seed=43, n_races=20, n_lo=2, n_hi=7, rollouts=300, rem_lo=100.0, rem_hi=800.0)
    for dist in (W.DIST_UNIFORM, W.DIST_TWO_POINT):
        rb.dist = dist
        with bbe.Batch(rb) as b:
            for places in (7, 3):  # the second call lays the tables out again
                keys, counts, off, _, steps = b.order_histogram(places)
                b.status()
                got = histograms(rb, keys.cpu().numpy(), counts.cpu().numpy(), off, places)
                want, want_s, st = oracle.batch_order_histograms(rb, places)
                assert st == 0 and got == [dict(w) for w in want]
                assert np.array_equal(steps.cpu().numpy(), want_s)


def test_full_size_sampled_races(bbe):
    # the full workload (4096 x 20 x 10^4), first five places: the invariants on every race and
    # sampled races against the oracle
    rb = W.uniform_batch(seed=0)
    keys, counts, off, _, steps = run(bbe, rb, 5)
    per_race = np.add.reduceat(counts.astype(np.int64), off[:-1])
    assert np.all(per_race == 10000)
    sample = [0, 2048, 4095]
    got = histograms(rb, keys, counts, off, 5, races=sample)
    want, want_s, st = oracle.batch_order_histograms(rb, 5, races=sample)
    assert st == 0
    for i, r in enumerate(sample):
        assert got[i] == dict(want[i]), r
        assert steps[r] == want_s[i]


def test_rejects_keys_beyond_64_bits(bbe):
    rb = W.concat([W.uniform_batch(seed=44, n_races=3, n=5, rollouts=10),
                   W.uniform_batch(seed=44, n_races=1, n=21, rollouts=10)])
    with bbe.Batch(rb) as b:
        with pytest.raises(bbe.BbeError) as ei:
            b.order_histogram(21)
        assert ei.value.status == -7 and "race 3" in bbe.bbe_last_error()
        keys, counts, off, _, _ = b.order_histogram(18)  # 21! / 3! < 2^64
        b.status()
        assert int(counts.sum()) == 40



@pytest.mark.parametrize("slots", [1, 3, 4])
def test_other_layouts_match_oracle(bbe, slots):
    rb = W.uneven_batch(seed=46, n_races=24, n_lo=1, n_hi=12, rollouts=250, rem_lo=100.0, rem_hi=1200.0)
    with bbe.Batch(rb) as b:
        b.set_cfg(slots_per_lane=slots)
        keys, counts, off, _, steps = b.order_histogram(32)
        b.status()
        got = histograms(rb, keys.cpu().numpy(), counts.cpu().numpy(), off, 32)
        steps = steps.cpu().numpy()
    want, want_s, st = oracle.batch_order_histograms(rb, 32)
    assert st == 0 and got == [dict(w) for w in want]
    assert np.array_equal(steps, want_s)
