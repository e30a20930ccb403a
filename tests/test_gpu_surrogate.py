"""The surrogate network on the GPU (through the C ABI) against the float64 reference in
oracle/surrogate_ref.py, evaluated with bfloat16 rounding at the same points as the GPU,
plus training, Monte Carlo fallback and checkpoint behaviour."""
import numpy as np
import pytest

import oracle
from oracle import surrogate_ref as S
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


def ref_inputs(rb):
    L = np.repeat(rb.L.astype(np.float64), rb.sizes())
    return S.features(rb.d0, L, rb.mu, rb.sigma, rb.rho, rb.race_off)


def dirichlet_targets(rb, seed):
    rng = np.random.default_rng(seed)
    t = np.empty(rb.n_total, np.float32)
    for r in range(rb.n_races):
        a, b = rb.race_off[r], rb.race_off[r + 1]
        t[a:b] = rng.dirichlet(np.ones(b - a))
    return t


def test_param_count_matches_reference(bbe):
    assert bbe.bbe_surrogate_num_params() == S.N_PARAMS


def test_forward_matches_reference(bbe):
    rb = W.uneven_batch(seed=41, n_races=300, rollouts=10)  # 2..24 competitors, many tiles
    params = S.init_params(1).astype(np.float32)
    s = bbe.bbe_surrogate_create(0)
    try:
        bbe.bbe_surrogate_set_params(s, params)
        with bbe.Batch(rb) as b:
            probs = torch.empty(rb.n_total, dtype=torch.float32, device="cuda")
            bbe.bbe_surrogate_forward(s, b.handle, probs)
            bbe.bbe_surrogate_status(s)
            got = probs.cpu().numpy().astype(np.float64)
        assert np.allclose(bbe.bbe_surrogate_get_params(s), params)
    finally:
        bbe.bbe_surrogate_destroy(s)
    want, _ = S.forward(params.astype(np.float64), ref_inputs(rb), rb.race_off, bf16=True)
    sums = np.add.reduceat(got, rb.race_off[:-1])
    assert np.allclose(sums, 1.0, atol=1e-5)
    err = np.abs(got - want)
    assert err.max() < 5e-3 and err.mean() < 3e-4, (err.max(), err.mean())


def test_forward_persistent_blocks_match_reference(bbe):
    # more tiles than the persistent grid has tile pipelines (two per SM), full 64-race tiles
    # of two competitors, single-competitor races
    rb = W.concat([W.uniform_batch(seed=51, n_races=3000, n=20, rollouts=10),
                   W.uneven_batch(seed=52, n_races=1500, n_lo=2, n_hi=2, rollouts=10),
                   W.uneven_batch(seed=53, n_races=300, n_lo=1, n_hi=3, rollouts=10)])
    params = S.init_params(3).astype(np.float32)
    s = bbe.bbe_surrogate_create(0)
    try:
        bbe.bbe_surrogate_set_params(s, params)
        with bbe.Batch(rb) as b:
            probs = torch.full((rb.n_total,), float("nan"), dtype=torch.float32, device="cuda")
            bbe.bbe_surrogate_forward(s, b.handle, probs)
            bbe.bbe_surrogate_status(s)
            got = probs.cpu().numpy().astype(np.float64)
    finally:
        bbe.bbe_surrogate_destroy(s)
    want, _ = S.forward(params.astype(np.float64), ref_inputs(rb), rb.race_off, bf16=True)
    assert np.all(np.isfinite(got))
    err = np.abs(got - want)
    assert err.max() < 5e-3 and err.mean() < 3e-4, (err.max(), err.mean())
    single = np.flatnonzero(np.diff(rb.race_off) == 1)
    assert np.all(got[rb.race_off[single]] == 1.0)


def test_gradient_matches_reference(bbe):
    rb = W.uneven_batch(seed=42, n_races=150, rollouts=10)
    target = dirichlet_targets(rb, 3)
    params = S.init_params(2).astype(np.float32)
    s = bbe.bbe_surrogate_create(0)
    try:
        bbe.bbe_surrogate_set_params(s, params)
        with bbe.Batch(rb) as b:
            grad = torch.empty(S.N_PARAMS, dtype=torch.float32, device="cuda")
            loss = torch.empty(1, dtype=torch.float32, device="cuda")
            bbe.bbe_surrogate_grad(s, b.handle, torch.from_numpy(target).cuda(), grad, loss)
            torch.cuda.synchronize()
            g = grad.cpu().numpy().astype(np.float64)
            lv = float(loss.item())
    finally:
        bbe.bbe_surrogate_destroy(s)
    x = ref_inputs(rb)
    want = S.backward(params.astype(np.float64), x, rb.race_off, target.astype(np.float64), bf16=True)
    want_loss = S.loss(params.astype(np.float64), x, rb.race_off, target.astype(np.float64), bf16=True)
    assert abs(lv - want_loss) < 1e-3 * abs(want_loss)
    assert_gradient_close(g, want)


def assert_gradient_close(g, want):
    """Element by element: |gpu - ref| <= 3 % of the element plus 0.5 % of its block's largest
    element.  The GPU sums bfloat16-rounded du, da and pooled dz where the reference sums the
    unrounded values (bias gradients, the context's gradient): bfloat16 carries 8 significant
    bits (a relative rounding of 2^-9), so those sums differ by a few parts per thousand where
    their terms cancel, which the block-relative term absorbs."""
    for name, _ in S.SHAPES[:-1]:  # b5's gradient is ~0 (targets sum to 1)
        gu, wu = S.unpack(g)[name].ravel(), S.unpack(want)[name].ravel()
        bound = 3e-2 * np.abs(wu) + 5e-3 * np.abs(wu).max()
        worst = np.max(np.abs(gu - wu) / bound)
        assert worst <= 1.0, (name, worst, int(np.argmax(np.abs(gu - wu) / bound)))


def test_first_adam_step_follows_the_reference_gradient(bbe):
    # one training step over every race (batch = all of them) from known parameters: Adam's
    # first step is w - lr g / (|g| + eps), about lr sign(g), so every parameter must move by
    # the step the float64 reference gradient gives it (a misplaced gradient element or a
    # misrouted update moves about half of them the wrong way)
    rb = W.uneven_batch(seed=43, n_races=150, rollouts=10)
    target = dirichlet_targets(rb, 5)
    params = S.init_params(4).astype(np.float32)
    lr = 1e-3
    s = bbe.bbe_surrogate_create(0)
    try:
        bbe.bbe_surrogate_set_params(s, params)
        with bbe.Batch(rb) as b:
            bbe.bbe_surrogate_train(s, b.handle, torch.from_numpy(target).cuda(), lr=lr, batch_states=rb.n_races,
                                    steps=1)
            torch.cuda.synchronize()
        after = bbe.bbe_surrogate_get_params(s).astype(np.float64)
    finally:
        bbe.bbe_surrogate_destroy(s)
    g = S.backward(params.astype(np.float64), ref_inputs(rb), rb.race_off, target.astype(np.float64), bf16=True)
    want = -lr * g / (np.abs(g) + 1e-8)
    got = after - params.astype(np.float64)
    assert np.all(np.abs(got) <= lr * (1 + 1e-3))
    clear = np.abs(g) > 1e-4  # elements whose sign the GPU's bfloat16 gradient cannot flip
    assert clear.sum() > 0.5 * g.size
    close = np.abs(got - want) <= 2e-2 * lr
    assert close[clear].mean() > 0.99, close[clear].mean()


def test_training_reduces_loss_on_mc_targets(bbe):
    rb = W.uneven_batch(seed=43, n_races=3000, n_lo=2, n_hi=10, rollouts=2000, rem_lo=100.0, rem_hi=1500.0)
    s = bbe.bbe_surrogate_create(5)
    try:
        with bbe.Batch(rb) as b:
            counts, _ = b.rollout()
            probs, _ = b.win_probs(counts)
            log = torch.empty(300, dtype=torch.float32, device="cuda")
            bbe.bbe_surrogate_train(s, b.handle, probs, lr=2e-3, batch_states=512, steps=300, loss_log=log)
            torch.cuda.synchronize()
            losses = log.cpu().numpy()
            out = torch.empty_like(probs)
            bbe.bbe_surrogate_forward(s, b.handle, out)
            torch.cuda.synchronize()
            err = np.abs(out.cpu().numpy() - probs.cpu().numpy())
    finally:
        bbe.bbe_surrogate_destroy(s)
    assert np.all(np.isfinite(losses))
    assert losses[-20:].mean() < 0.6 * losses[:5].mean()
    assert err.mean() < 0.05


def test_infer_falls_back_to_exact_monte_carlo(bbe, tmp_path):
    train = W.uneven_batch(seed=44, n_races=400, n_lo=2, n_hi=12, rollouts=500)
    query = W.concat([W.uneven_batch(seed=45, n_races=30, n_lo=2, n_hi=12, rollouts=700),   # in range
                      W.uneven_batch(seed=46, n_races=10, n_lo=16, n_hi=20, rollouts=700),  # too many competitors
                      W.uneven_batch(seed=47, n_races=10, n_lo=3, n_hi=6, rollouts=700, rem_lo=20.0, rem_hi=90.0)])
    s = bbe.bbe_surrogate_create(6)
    try:
        with bbe.Batch(train) as tb:
            c, _ = tb.rollout()
            p, _ = tb.win_probs(c)
            bbe.bbe_surrogate_train(s, tb.handle, p, batch_states=128, steps=20)
        with bbe.Batch(query) as qb:
            probs = torch.empty(query.n_total, dtype=torch.float32, device="cuda")
            used = torch.empty(query.n_races, dtype=torch.uint8, device="cuda")
            bbe.bbe_surrogate_infer(s, qb.handle, probs, used)
            counts, _ = qb.rollout()
            mc_p, _ = qb.win_probs(counts)
            torch.cuda.synchronize()
            used = used.cpu().numpy()
            got, mc = probs.cpu().numpy(), mc_p.cpu().numpy()
        assert used[:30].sum() == 0 and used[30:].sum() == 20
        for r in range(30, 50):
            a, e = query.race_off[r], query.race_off[r + 1]
            assert np.array_equal(got[a:e], mc[a:e])  # the fallback is the Monte Carlo path itself
        sums = np.add.reduceat(got.astype(np.float64), query.race_off[:-1])
        assert np.allclose(sums, 1.0, atol=1e-5)
        # checkpoint round trip keeps parameters, ranges and outputs
        path = tmp_path / "sg.bin"
        bbe.bbe_surrogate_save(s, str(path))
        s2 = bbe.bbe_surrogate_load(str(path))
        try:
            assert np.array_equal(bbe.bbe_surrogate_get_params(s2), bbe.bbe_surrogate_get_params(s))
            with bbe.Batch(query) as qb:
                probs2 = torch.empty_like(probs)
                used2 = torch.empty(query.n_races, dtype=torch.uint8, device="cuda")
                bbe.bbe_surrogate_infer(s2, qb.handle, probs2, used2)
                torch.cuda.synchronize()
                assert np.array_equal(probs2.cpu().numpy(), got)
                assert np.array_equal(used2.cpu().numpy(), used)
        finally:
            bbe.bbe_surrogate_destroy(s2)
    finally:
        bbe.bbe_surrogate_destroy(s)


def test_confidence_gate_sends_uncertain_races_to_monte_carlo(bbe):
    rb = W.uneven_batch(seed=54, n_races=600, n_lo=2, n_hi=10, rollouts=800)
    s = bbe.bbe_surrogate_create(9)
    try:
        with bbe.Batch(rb) as b:
            c, _ = b.rollout()
            mc, _ = b.win_probs(c)
            bbe.bbe_surrogate_train(s, b.handle, mc, batch_states=128, steps=30)
            net = torch.empty_like(mc)
            bbe.bbe_surrogate_forward(s, b.handle, net)  # the training states are all in range
            out = torch.empty_like(mc)
            used = torch.empty(rb.n_races, dtype=torch.uint8, device="cuda")
            thr = 1e-3
            bbe.bbe_surrogate_set_gate(s, thr)
            bbe.bbe_surrogate_infer(s, b.handle, out, used)
            gated = used.cpu().numpy()
            bbe.bbe_surrogate_set_gate(s, 1.0)
            bbe.bbe_surrogate_infer(s, b.handle, out2 := torch.empty_like(mc), used)
            ungated = used.cpu().numpy()
            torch.cuda.synchronize()
            net, out, out2, mc = (t.cpu().numpy() for t in (net, out, out2, mc))
        with pytest.raises(bbe.BbeError):
            bbe.bbe_surrogate_set_gate(s, 1.5)
    finally:
        bbe.bbe_surrogate_destroy(s)
    assert np.all(ungated == 0) and np.array_equal(out2, net)
    assert set(np.unique(gated)) <= {0, 2} and 0 < (gated == 2).sum() < rb.n_races
    for r in range(rb.n_races):
        a, e = rb.race_off[r], rb.race_off[r + 1]
        runner_up = np.sort(net[a:e])[-2]
        assert (gated[r] == 2) == (runner_up > np.float32(thr)), r
        assert np.array_equal(out[a:e], mc[a:e] if gated[r] else net[a:e]), r


def test_two_stage_fallback_is_monte_carlo_at_the_rule_budget(bbe):
    # every query race falls back (too many competitors, or gated); each must equal the oracle's
    # Monte Carlo at the budget that the rule derives from the oracle's own pilot counts
    import dataclasses

    train = W.uneven_batch(seed=60, n_races=300, n_lo=2, n_hi=8, rollouts=300)
    query = W.concat([W.uneven_batch(seed=61, n_races=8, n_lo=10, n_hi=16, rollouts=3000),
                      W.uneven_batch(seed=62, n_races=12, n_lo=2, n_hi=8, rollouts=3000)])
    pilot, sd = 400, 0.01
    s = bbe.bbe_surrogate_create(12)
    try:
        with bbe.Batch(train) as tb:
            c, _ = tb.rollout()
            p, _ = tb.win_probs(c)
            bbe.bbe_surrogate_train(s, tb.handle, p, batch_states=64, steps=10)
        bbe.bbe_surrogate_set_gate(s, 0.0)
        bbe.bbe_surrogate_set_fallback(s, pilot, sd)
        with bbe.Batch(query) as qb:
            probs = torch.empty(query.n_total, dtype=torch.float32, device="cuda")
            used = torch.empty(query.n_races, dtype=torch.uint8, device="cuda")
            bbe.bbe_surrogate_infer(s, qb.handle, probs, used)
            torch.cuda.synchronize()
            got, used = probs.cpu().numpy(), used.cpu().numpy()
        races, rollouts = bbe.bbe_surrogate_fallback_stats(s)
        with pytest.raises(bbe.BbeError):
            bbe.bbe_surrogate_set_fallback(s, 10, 0.0)
    finally:
        bbe.bbe_surrogate_destroy(s)
    assert np.all(used[:8] == 1) and np.all(used[8:] >= 1)
    R1 = np.minimum(query.rollouts, pilot)
    c1, _, st = oracle.batch_counts(dataclasses.replace(query, rollouts=R1))
    assert st == 0
    budget = np.array([bbe.bbe_surrogate_fallback_budget(c1[query.race_off[r]:query.race_off[r + 1]], int(R1[r]),
                                                         int(query.rollouts[r]), sd) for r in range(query.n_races)])
    assert races == query.n_races and rollouts == int(budget.sum())
    assert np.any(budget > pilot) and np.any(budget < query.rollouts)  # both stages and the cap-free case occur
    c, _, st = oracle.batch_counts(dataclasses.replace(query, rollouts=budget))
    assert st == 0
    want = c.astype(np.float32) / np.repeat(budget, query.sizes()).astype(np.float32)
    assert np.array_equal(got, want)


def test_bounded_wait_reports_timeout_and_context_stays_usable(bbe):
    # a wait on an mbarrier that nothing completes gives up after 1 ms: the status call reports
    # BBE_ERR_TIMEOUT once, and the handle and context keep working
    rb = W.uneven_batch(seed=49, n_races=20, rollouts=10)
    params = S.init_params(6).astype(np.float32)
    s = bbe.bbe_surrogate_create(0)
    try:
        bbe.bbe_surrogate_set_params(s, params)
        bbe.bbe_surrogate_wait_probe(s, 1_000_000)
        with pytest.raises(bbe.BbeError) as ei:
            bbe.bbe_surrogate_status(s)
        assert ei.value.status == -6
        bbe.bbe_surrogate_status(s)  # cleared
        with bbe.Batch(rb) as b:
            probs = torch.empty(rb.n_total, dtype=torch.float32, device="cuda")
            bbe.bbe_surrogate_forward(s, b.handle, probs)
            bbe.bbe_surrogate_status(s)
            got = probs.cpu().numpy().astype(np.float64)
        with pytest.raises(bbe.BbeError):
            bbe.bbe_surrogate_wait_probe(s, -1)
    finally:
        bbe.bbe_surrogate_destroy(s)
    want, _ = S.forward(params.astype(np.float64), ref_inputs(rb), rb.race_off, bf16=True)
    assert np.abs(got - want).max() < 5e-3


def test_infer_without_training_ranges_is_refused(bbe):
    rb = W.uneven_batch(seed=48, n_races=4, rollouts=10)
    s = bbe.bbe_surrogate_create(7)
    try:
        with bbe.Batch(rb) as b:
            probs = torch.empty(rb.n_total, dtype=torch.float32, device="cuda")
            with pytest.raises(bbe.BbeError) as ei:
                bbe.bbe_surrogate_infer(s, b.handle, probs)
            assert ei.value.status == -7
    finally:
        bbe.bbe_surrogate_destroy(s)


def test_relabelling_competitors_relabels_output(bbe):
    rb = W.uneven_batch(seed=49, n_races=40, rollouts=10)
    rng = np.random.default_rng(0)
    perm = np.concatenate([rb.race_off[r] + rng.permutation(rb.race_off[r + 1] - rb.race_off[r])
                           for r in range(rb.n_races)])
    pb = W.from_arrays(rb.sizes(), rb.L, rb.rollouts, rb.d0[perm], rb.mu[perm], rb.sigma[perm], rb.rho[perm])
    s = bbe.bbe_surrogate_create(8)
    try:
        outs = []
        for batch in (rb, pb):
            with bbe.Batch(batch) as b:
                probs = torch.empty(batch.n_total, dtype=torch.float32, device="cuda")
                bbe.bbe_surrogate_forward(s, b.handle, probs)
                torch.cuda.synchronize()
                outs.append(probs.cpu().numpy())
    finally:
        bbe.bbe_surrogate_destroy(s)
    assert np.allclose(outs[1], outs[0][perm], atol=2e-3)


def test_raw_inputs_forward_matches_reference(bbe):
    # the five-input network: derived columns zero on both sides
    rb = W.uneven_batch(seed=46, n_races=200, rollouts=10)
    params = S.init_params(7).astype(np.float32)
    s = bbe.bbe_surrogate_create(0)
    try:
        bbe.bbe_surrogate_set_params(s, params)
        bbe.bbe_surrogate_set_inputs(s, bbe.SURROGATE_INPUTS_RAW)
        with bbe.Batch(rb) as b:
            probs = torch.empty(rb.n_total, dtype=torch.float32, device="cuda")
            bbe.bbe_surrogate_forward(s, b.handle, probs)
            bbe.bbe_surrogate_status(s)
            got = probs.cpu().numpy().astype(np.float64)
    finally:
        bbe.bbe_surrogate_destroy(s)
    L = np.repeat(rb.L.astype(np.float64), rb.sizes())
    want, _ = S.forward(params.astype(np.float64), S.features(rb.d0, L, rb.mu, rb.sigma, rb.rho), rb.race_off,
                        bf16=True)
    err = np.abs(got - want)
    assert err.max() < 5e-3 and err.mean() < 3e-4, (err.max(), err.mean())


def test_training_resumes_from_a_checkpoint(bbe, tmp_path):
    # save in the middle of an epoch, load into a new handle, train on: the parameters equal
    # those of the run that was never interrupted (the epoch's order is regenerated, Adam's
    # moments and step count are restored)
    rb = W.uneven_batch(seed=47, n_races=700, n_lo=2, n_hi=12, rollouts=300)
    kw = dict(lr=2e-3, batch_states=128, shuffle_seed=11)
    path = str(tmp_path / "mid.bin")
    with bbe.Batch(rb) as b:
        counts, _ = b.rollout()
        probs, _ = b.win_probs(counts)
        a = bbe.bbe_surrogate_create(3)
        try:
            bbe.bbe_surrogate_train(a, b.handle, probs, steps=9, **kw)  # 9 x 128 races: into epoch 2
            bbe.bbe_surrogate_save(a, path)
            bbe.bbe_surrogate_train(a, b.handle, probs, steps=8, **kw)
            torch.cuda.synchronize()
            want = bbe.bbe_surrogate_get_params(a)
        finally:
            bbe.bbe_surrogate_destroy(a)
        c = bbe.bbe_surrogate_load(path)
        try:
            bbe.bbe_surrogate_train(c, b.handle, probs, steps=8, **kw)
            torch.cuda.synchronize()
            got = bbe.bbe_surrogate_get_params(c)
        finally:
            bbe.bbe_surrogate_destroy(c)
    assert np.array_equal(got, want)
