"""Parity of the time law of responsiveness on the GPU (through the C ABI): win counts and
step totals of every layout and step distribution, full-race trajectories, and the
bettors' snapshot batches (whose elapsed time grows with the snapshot's step), bit for bit
against the CPU oracle; place tallies and the surrogate refuse time-law batches."""
import numpy as np
import pytest

import oracle
from oracle import bettors as Bt
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


def timed_batch(seed, n_races, **kw):
    rb = W.uneven_batch(seed=seed, n_races=n_races, **kw)
    rng = np.random.default_rng(seed + 1)
    # elapsed 0 .. 400 steps (some past the horizon, where u is held at 1), horizons 50 .. 400
    return W.with_time_law(rb, rng.integers(0, 400, rb.n_races).astype(np.float32),
                           rng.uniform(50.0, 400.0, rb.n_races).astype(np.float32))


def run(bbe, rb, cfg=None):
    with bbe.Batch(rb) as b:
        if cfg:
            b.set_cfg(**cfg)
        counts, steps = b.rollout()
        b.rollout(counts, steps)  # the captured graph's replay
        b.status()
        torch.cuda.synchronize()
        return counts.cpu().numpy(), steps.cpu().numpy()


@pytest.mark.parametrize("slots", [1, 2, 3, 4])
@pytest.mark.parametrize("dist", [W.DIST_NORMAL, W.DIST_UNIFORM, W.DIST_TWO_POINT])
def test_counts_match_oracle(bbe, slots, dist):
    rb = timed_batch(70 + slots, 40, n_lo=1, n_hi=32, rollouts=300, rem_lo=100.0, rem_hi=1500.0)
    rb.dist = dist
    got_c, got_s = run(bbe, rb, {"slots_per_lane": slots})
    want_c, want_s, st = oracle.batch_counts(rb)
    assert st == 0
    assert np.array_equal(got_c, want_c) and np.array_equal(got_s, want_s)


def test_uniform_workload_sample(bbe):
    # the uniform workload's full budget under the time law; three races checked one by one
    rb = W.with_time_law(W.uniform_batch(seed=0, n_races=256), 0.0, 300.0)
    got_c, got_s = run(bbe, rb)
    races = [0, 101, 255]
    want_c, want_s, _ = oracle.batch_counts(rb, races=races)
    got = np.concatenate([got_c[rb.race_off[r]:rb.race_off[r + 1]] for r in races])
    assert np.array_equal(got, want_c) and np.array_equal(got_s[races], want_s)


def test_step_limit(bbe):
    rb = timed_batch(80, 12, rollouts=50, rem_lo=3000.0, rem_hi=5000.0)
    with bbe.Batch(rb) as b:
        b.set_cfg(max_steps=101)
        counts, steps = b.rollout()
        with pytest.raises(bbe.BbeError) as ei:
            b.status()
        assert ei.value.status == -5
        c, s = counts.cpu().numpy(), steps.cpu().numpy()
    want_c, want_s, st = oracle.batch_counts(rb, max_steps=101)
    assert st == oracle.STEP_LIMIT and np.array_equal(c, want_c) and np.array_equal(s, want_s)


def test_back_to_the_position_law(bbe):
    rb = timed_batch(81, 20, rollouts=200)
    plain = W.uneven_batch(seed=81, n_races=20, rollouts=200)
    with bbe.Batch(rb) as b:
        bbe.bbe_batch_set_law(b.handle, bbe.LAW_POSITION)
        counts, steps = b.rollout()
        b.status()
        c, s = counts.cpu().numpy(), steps.cpu().numpy()
    want_c, want_s, _ = oracle.batch_counts(plain)
    assert np.array_equal(c, want_c) and np.array_equal(s, want_s)


def test_trajectories_and_snapshots(bbe):
    rb = W.with_time_law(W.single_race_start(seed=2), 25.0, 140.0)
    cap, every, bettors, dry, id0, k = 400, 9, 2, 80, 500, 12345
    with bbe.Batch(rb) as b:
        pos = torch.full((rb.n_total * cap,), float("nan"), dtype=torch.float32, device="cuda")
        stp = torch.full_like(pos, float("nan"))
        ns = torch.empty(rb.n_races, dtype=torch.int32, device="cuda")
        bbe.bbe_race_trajectory(b.handle, k, cap, pos, stp, ns)
        h, n_snap = bbe.bbe_snapshot_batch(b.handle, 0, pos, stp, ns, cap, every, bettors, dry, id0)
        try:
            info = bbe.bbe_batch_info(h)
            counts = torch.empty(info["n_competitors"], dtype=torch.int32, device="cuda")
            steps = torch.empty(info["n_races"], dtype=torch.int64, device="cuda")
            bbe.bbe_rollout_batch(h, counts, steps)
            bbe.bbe_batch_status(h)
            torch.cuda.synchronize()
            counts, steps = counts.cpu().numpy(), steps.cpu().numpy()
        finally:
            bbe.bbe_destroy_batch(h)
        pos, stp, ns = (x.cpu().numpy() for x in (pos, stp, ns))
    rc = rb.race(0)
    n = rc["n"]
    wd, ws, T, st = oracle.trajectory(rc, rb.seed, 0, k, cap=cap)
    assert st == 0 and ns[0] == T
    assert np.array_equal(pos[:T * n].reshape(T, n), wd) and np.array_equal(stp[:T * n].reshape(T, n), ws)
    prev0 = (rc["mu"] * rc["P"]).astype(np.float32)
    for s, bt in [(0, 0), (1, 1), (n_snap // 2, 0), (n_snap - 1, 1)]:
        ts = s * every
        state = dict(rc, d0=Bt.state_at(rc["d0"], wd, ts), prev0=prev0 if ts == 0 else ws[ts - 1],
                     t0=float(np.float32(rc["t0"]) + np.float32(ts)))
        rr = s * bettors + bt
        want, wsteps, _ = oracle.race_counts(state, rb.seed, r=id0 + rr, R=dry)
        assert np.array_equal(counts[rr * n:(rr + 1) * n], want), (s, bt)
        assert steps[rr] == wsteps


@pytest.mark.parametrize("slots", [0, 1, 4])
def test_places_orders_and_order_histogram_follow_the_time_law(bbe, slots):
    # the place mode under the time law: place counts, dense ordered tallies and the full-order
    # histogram of one pass each, against the oracle's dry-runs of the same law
    rb = timed_batch(84, 24, n_lo=1, n_hi=9, rollouts=300, rem_lo=100.0, rem_hi=1500.0)
    with bbe.Batch(rb) as b:
        if slots:
            b.set_cfg(slots_per_lane=slots)
        pc, psteps = b.places(3)
        orders, _, osteps = b.orders(2)
        keys, hc, off, _, hsteps = b.order_histogram(32)
        b.status()
        pc, psteps, orders, osteps = (t.cpu().numpy() for t in (pc, psteps, orders, osteps))
        keys, hc, hsteps = keys.cpu().numpy(), hc.cpu().numpy(), hsteps.cpu().numpy()
    want_p, want_ps, st = oracle.batch_places(rb, 3)
    assert st == 0 and np.array_equal(pc.ravel(), want_p.ravel()) and np.array_equal(psteps, want_ps)
    want_o, want_os, st = oracle.batch_orders(rb, 2)
    pos = 0
    for r in range(rb.n_races):
        n = int(rb.race_off[r + 1] - rb.race_off[r])
        size = n ** min(2, n)
        assert np.array_equal(orders[pos:pos + size], want_o[r]), r
        pos += size
    assert np.array_equal(osteps, want_os)
    want_h, want_hs, st = oracle.batch_order_histograms(rb, 32)
    assert st == 0 and np.array_equal(hsteps, want_hs)
    for r in range(rb.n_races):
        n = int(rb.race_off[r + 1] - rb.race_off[r])
        k, c = keys[off[r]:off[r + 1]], hc[off[r]:off[r + 1]]
        used = k != np.uint64(2 ** 64 - 1)
        got = {tuple(int(x) for x in bbe.bbe_order_key_decode(n, 32, int(key))): int(v) for key, v in zip(k[used], c[used])}
        assert got == dict(want_h[r]), r
    # the law matters: the same batch under the position law places differently somewhere
    pos_rb = W.uneven_batch(seed=84, n_races=24, n_lo=1, n_hi=9, rollouts=300, rem_lo=100.0, rem_hi=1500.0)
    want_pos, _, _ = oracle.batch_places(pos_rb, 3)
    assert not np.array_equal(want_pos.ravel(), want_p.ravel())


def test_surrogate_refuses_the_time_law(bbe):
    rb = timed_batch(82, 8, rollouts=50)
    with bbe.Batch(rb) as b:
        s = bbe.bbe_surrogate_create(0)
        try:
            out = torch.empty(rb.n_total, dtype=torch.float32, device="cuda")
            with pytest.raises(bbe.BbeError) as ei:
                bbe.bbe_surrogate_forward(s, b.handle, out)
            assert ei.value.status == -2
        finally:
            bbe.bbe_surrogate_destroy(s)
    with pytest.raises(bbe.BbeError) as ei:  # the time law needs a horizon
        with bbe.Batch(W.uneven_batch(seed=83, n_races=3, rollouts=5)) as b2:
            bbe.bbe_batch_set_law(b2.handle, bbe.LAW_TIME, None, None)
    assert ei.value.status == -1
