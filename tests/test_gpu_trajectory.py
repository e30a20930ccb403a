"""Parity of the actual-race path on the GPU (through the C ABI): full-race trajectories, the
bettors' snapshot batch and its dry-runs, and the rule-based bettors' predictions, against the
CPU oracle (oracle/bbe_oracle.c, oracle/bettors.py)."""
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


def gpu_trajectory(bbe, b, rb, k, cap):
    pos = torch.full((rb.n_total * cap,), float("nan"), dtype=torch.float32, device="cuda")
    stp = torch.full_like(pos, float("nan"))
    ns = torch.empty(rb.n_races, dtype=torch.int32, device="cuda")
    bbe.bbe_race_trajectory(b.handle, k, cap, pos, stp, ns)
    return pos, stp, ns


@pytest.mark.parametrize("dist", [W.DIST_NORMAL, W.DIST_UNIFORM, W.DIST_TWO_POINT])
def test_trajectories_match_oracle(bbe, dist):
    rb = W.uneven_batch(seed=61, n_races=24, n_lo=1, n_hi=32, rollouts=10, rem_lo=100.0, rem_hi=800.0)
    rb.dist = dist
    cap = 200
    with bbe.Batch(rb) as b:
        pos, stp, ns = gpu_trajectory(bbe, b, rb, 5, cap)
        b.status()
        pos, stp, ns = (x.cpu().numpy() for x in (pos, stp, ns))
    for r in range(rb.n_races):
        n = int(rb.race_off[r + 1] - rb.race_off[r])
        wd, ws, T, st = oracle.trajectory(rb.race(r), rb.seed, r, 5, cap=cap)
        assert st == 0 and ns[r] == T
        base = int(rb.race_off[r]) * cap
        rows = min(T, cap)
        assert np.array_equal(pos[base:base + rows * n].reshape(rows, n), wd), r
        assert np.array_equal(stp[base:base + rows * n].reshape(rows, n), ws), r


def test_snapshot_batch_dry_runs_and_predictions(bbe):
    rb = W.single_race_start(seed=0)  # 5 competitors, L 2000
    cap, every, bettors, dry, id0, k = 400, 7, 3, 64, 1000, 1 << 30
    with bbe.Batch(rb) as b:
        pos, stp, ns = gpu_trajectory(bbe, b, rb, k, cap)
        h, n_snap = bbe.bbe_snapshot_batch(b.handle, 0, pos, stp, ns, cap, every, bettors, dry, id0)
        try:
            info = bbe.bbe_batch_info(h)
            counts = torch.empty(info["n_competitors"], dtype=torch.int32, device="cuda")
            steps = torch.empty(info["n_races"], dtype=torch.int64, device="cuda")
            bbe.bbe_rollout_batch(h, counts, steps)
            bbe.bbe_batch_status(h)
            pred = torch.empty(n_snap * 4, dtype=torch.int32, device="cuda")
            bbe.bbe_bettor_predictions(b.handle, 0, pos, stp, ns, cap, every, n_snap, 10, 3.0, 77, pred)
            torch.cuda.synchronize()
            counts, steps, pred = counts.cpu().numpy(), steps.cpu().numpy(), pred.cpu().numpy().reshape(n_snap, 4)
        finally:
            bbe.bbe_destroy_batch(h)
    rc = rb.race(0)
    n = rc["n"]
    wd, ws, T, st = oracle.trajectory(rc, rb.seed, 0, k, cap=cap)
    open_t = [t for t in range(0, T + 1, every) if np.all(Bt.state_at(rc["d0"], wd, t) < rc["L"])]
    open_t = open_t[:next((i for i, t in enumerate(open_t) if i * every != t), len(open_t))]
    assert n_snap == len(open_t) and info["n_races"] == n_snap * bettors
    prev0 = (rc["mu"] * rc["P"]).astype(np.float32)
    sample = [(0, 0), (0, bettors - 1), (n_snap // 2, 1), (n_snap - 1, 2)]
    for s, bt in sample:
        ts = s * every
        state = dict(rc, d0=Bt.state_at(rc["d0"], wd, ts), prev0=prev0 if ts == 0 else ws[ts - 1])
        rr = s * bettors + bt
        want, wsteps, _ = oracle.race_counts(state, rb.seed, r=id0 + rr, R=dry)
        assert np.array_equal(counts[rr * n:(rr + 1) * n], want), (s, bt)
        assert steps[rr] == wsteps
    for s in range(n_snap):
        ts = s * every
        d = Bt.state_at(rc["d0"], wd, ts)
        want = [Bt.leader(d), Bt.underdog(d, 3.0), Bt.linex(d, ws, ts, 10, rc["L"], prev0),
                Bt.zero_intelligence(n, rb.seed, s, 77)]
        assert list(pred[s]) == want, (s, list(pred[s]), want)


def test_bad_arguments(bbe):
    rb = W.single_race_start(seed=1)
    with bbe.Batch(rb) as b:
        pos, stp, ns = gpu_trajectory(bbe, b, rb, 0, 10)
        with pytest.raises(bbe.BbeError) as ei:
            bbe.bbe_snapshot_batch(b.handle, 1, pos, stp, ns, 10, 1, 1, 10, 0)
        assert ei.value.status == -1
        with pytest.raises(bbe.BbeError) as ei:
            bbe.bbe_race_trajectory(b.handle, 0, 0, pos, stp, ns)
        assert ei.value.status == -1


def test_preference_coefficients_match_oracle(bbe):
    rng = np.random.default_rng(12)
    sizes = rng.integers(1, 25, 300)
    off = np.zeros(sizes.size + 1, np.int32)
    off[1:] = np.cumsum(sizes)
    F = 6
    f = rng.uniform(0, 1, (sizes.size, F)).astype(np.float32)
    p = rng.uniform(-0.5, 1.5, (int(off[-1]), F)).astype(np.float32)
    w = rng.uniform(0, 1, F).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    P = torch.empty(int(off[-1]), dtype=torch.float32, device="cuda")
    bbe.bbe_preference_coefficients(sizes.size, dev(off), int(off[-1]), F, dev(f), dev(p), dev(w), P)
    torch.cuda.synchronize()
    assert np.array_equal(P.cpu().numpy(), oracle.preference(off, f, p, w))
    # the coefficients drive Eq. 1 through bbe_race_init's preference input
    rb = W.uneven_batch(seed=62, n_races=sizes.size, n_lo=1, n_hi=24, rollouts=200, rem_lo=100.0, rem_hi=600.0)
    rb = W.from_arrays(rb.sizes(), rb.L, rb.rollouts, rb.d0, rb.mu, rb.sigma, rb.rho, seed=5)
    off2 = rb.race_off
    f2 = rng.uniform(0, 1, (rb.n_races, F)).astype(np.float32)
    p2 = rng.uniform(0, 1, (rb.n_total, F)).astype(np.float32)
    P2 = torch.empty(rb.n_total, dtype=torch.float32, device="cuda")
    bbe.bbe_preference_coefficients(rb.n_races, dev(off2), rb.n_total, F, dev(f2), dev(p2), dev(w), P2)
    rb.P = P2.cpu().numpy()
    with bbe.Batch(rb) as b:
        counts, steps = b.rollout()
        b.status()
        counts, steps = counts.cpu().numpy(), steps.cpu().numpy()
    races = [0, 7, rb.n_races - 1]
    want_c, want_s, _ = oracle.batch_counts(rb, races=races)
    got = np.concatenate([counts[off2[r]:off2[r + 1]] for r in races])
    assert np.array_equal(got, want_c) and np.array_equal(steps[races], want_s)
