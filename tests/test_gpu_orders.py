"""Parity of the CUDA finishing-order tallies (bbe_order_counts through the C ABI) with the CPU
oracle: every race's table of ordered top-K tuples bit for bit, the place counts of the same
pass equal to bbe_place_counts's, K = 1 equal to the win counts, and a sampled check at the full
4096 x 20 x 10^4 size."""
import numpy as np
import pytest

import oracle
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
    oracle.build()
    B.lib()
    return B


def tables(rb, flat, places):
    out, pos = [], 0
    for n in rb.sizes():
        size = int(n) ** min(places, int(n))
        out.append(flat[pos:pos + size])
        pos += size
    assert pos == flat.size
    return out


@pytest.mark.parametrize("places", [1, 2, 3])
def test_uneven_small_matches_oracle(bbe, places):
    rb = W.uneven_batch(seed=31, n_races=40, n_lo=1, n_hi=14, rollouts=300, rem_lo=100.0, rem_hi=1500.0)
    with bbe.Batch(rb) as b:
        orders, pc, steps = b.orders(places, with_places=True)
        pc2, steps2 = b.places(places)
        wins, wsteps = b.rollout() if places == 1 else (None, None)
        b.status()
        torch.cuda.synchronize()
        got = tables(rb, orders.cpu().numpy(), places)
        pc, pc2, steps, steps2 = (t.cpu().numpy() for t in (pc, pc2, steps, steps2))
        assert bbe.bbe_order_table_size(b.handle, places) == sum(t.size for t in got)
        if places == 1:
            assert np.array_equal(orders.cpu().numpy(), wins.cpu().numpy())
    want, want_s, st = oracle.batch_orders(rb, places)
    assert st == 0
    for r in range(rb.n_races):
        assert np.array_equal(got[r], want[r]), r
    assert np.array_equal(steps, want_s)
    assert np.array_equal(pc, pc2) and np.array_equal(steps, steps2)


def test_distributions_and_layout_change(bbe):
    rb = W.uneven_batch(seed=32, n_races=24, n_lo=2, n_hi=9, rollouts=300, rem_lo=100.0, rem_hi=1200.0)
    for dist in (W.DIST_UNIFORM, W.DIST_TWO_POINT):
        rb.dist = dist
        with bbe.Batch(rb) as b:
            for places in (3, 2):  # the second call re-lays the tables out
                orders, _, steps = b.orders(places)
                b.status()
                got = tables(rb, orders.cpu().numpy(), places)
                want, want_s, st = oracle.batch_orders(rb, places)
                assert st == 0 and all(np.array_equal(g, w) for g, w in zip(got, want))
                assert np.array_equal(steps.cpu().numpy(), want_s)


def test_full_size_sampled_races(bbe):
    # the bench's full workload (4096 x 20 x 10^4) with K = 3: sampled races against the oracle
    rb = W.uniform_batch(seed=0)
    with bbe.Batch(rb) as b:
        orders, _, steps = b.orders(3)
        b.status()
        flat = orders.cpu().numpy()
        steps = steps.cpu().numpy()
    cells = 20 ** 3
    assert flat.size == rb.n_races * cells and int(flat.sum()) == rb.n_races * 10000
    sample = [0, 1777, 4095]
    want, want_s, st = oracle.batch_orders(rb, 3, races=sample)
    assert st == 0
    for i, r in enumerate(sample):
        assert np.array_equal(flat[r * cells:(r + 1) * cells], want[i]), r
        assert steps[r] == want_s[i]


def test_bad_arguments(bbe):
    rb = W.uneven_batch(seed=33, n_races=3, rollouts=10)
    with bbe.Batch(rb) as b:
        buf = torch.empty(10, dtype=torch.int32, device="cuda")
        for places in (0, 4):
            with pytest.raises(bbe.BbeError):
                bbe.bbe_order_counts(b.handle, places, buf)
            with pytest.raises(bbe.BbeError):
                bbe.bbe_order_table_size(b.handle, places)
