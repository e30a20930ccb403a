"""Benchmark: Monte Carlo race rollouts -> win counts -> win probabilities, on GB300.

A step is one pass of the whole path over one batch: bbe_rollout_batch (every race's
rollouts, winners counted) and bbe_win_probs (probabilities and odds).  The default
workload is 4096 mid-race snapshots x 20 competitors x 10,000 rollouts (track 5000, positions
U(0, 0.9 L), mean step U(15,17), spread U(0.5,1.5), responsiveness U(0,1), seed 0).  The metric is
competitor-steps per second: one competitor advanced by one step of Eq. 1, summed over all
rollouts until each rollout's first finisher.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload uniform|uneven|single]
                  [--impl gb300|reference] [--no-cpu-baseline] [--no-e2e]

Under torchrun (N > 1) every rank runs its own batch of the same shape with a distinct
range of race ids (weak scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2108_02419_gb300 import workloads as W  # noqa: E402

METRIC = "competitor-steps/s & win-prob vectors/s, MC vs surrogate (≤0.01 max-abs err), 1 GB300"
UNIT = "competitor-steps/s"

# Algorithmic 32-bit operations per competitor-step of the rollout contract (the operations
# the contract itself names, independent of how an implementation issues them):
#   Philox4x32-10 per 4 steps: 10 rounds x (2 mul.hi + 2 mul.lo + 4 two-input xor)     = 80 -> 20
#     (the round-key schedule depends on the seed alone and is computed once per launch)
#   Box-Muller per pair (2 steps): u1 = ((w >> 8) + 1) 2^-24 (4); log: exponent and
#     mantissa (4), range test and the two adjustments (3), f = m - 1 (1), 9 Horner FMAs,
#     f g (1), int -> float of e (1), 2 FMAs (21); radius -2 log, sqrt (2); angle:
#     shift, q (2), remainder (2), int -> float, scale (7); f^2, sin (4 FMA + 1 mul) and
#     cos (5 FMA) (11); quadrant rotation (7); r cos, r sin (2)                            = 54 -> 27
#   Eq. 1: R (2 FMA), successor load and order test (2), Delta and the theta test (2),
#     free step (FMA + 2 mul), blocked step (min, mul), select, floor, advance, finish test = 15
ALG_OPS_PER_COMPETITOR_STEP = 62.0
SMS = 152
LANES_PER_SM = 128  # 4 schedulers x 32 lanes: one warp instruction per scheduler per clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="uniform", choices=["uniform", "uneven", "single"])
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU work of the oracle sample")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--races", type=int, default=0, help="use only the first N races (profiling of a small case)")
    ap.add_argument("--surrogate", default="full", choices=["full", "small", "off"],
                    help="learned-surrogate leg: full = 2e6 training states x 1e4 rollouts, 20 epochs")
    ap.add_argument("--surrogate-kernels", default="", choices=["", "forward", "train"],
                    help="profiling aid: run only the surrogate's inference (3 calls) or 4 training steps of "
                         "4096 races on the first --races uneven states (default 100000), print timings and exit")
    ap.add_argument("--place-kernels", type=int, default=0, metavar="K",
                    help="profiling aid: run place counts to the K-th finisher on the --workload batch "
                         "(first --races races), print timings and exit")
    return ap.parse_args()


def run_place_kernels(args) -> dict:
    """Place counts alone (for profiler captures): one warm-up pass, one timed pass."""
    import torch

    from paper_2108_02419_gb300 import bbe

    rb = make_workload(args.workload, 0, args.races)
    K = args.place_kernels
    with bbe.Batch(rb) as b:
        counts = torch.empty((rb.n_total, K), dtype=torch.int32, device="cuda")
        steps = torch.empty(rb.n_races, dtype=torch.int64, device="cuda")
        bbe.bbe_place_counts(b.handle, K, counts, steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bbe.bbe_place_counts(b.handle, K, counts, steps)
        e1.record()
        e1.synchronize()
        b.status()
        cs = float((rb.sizes() * steps.cpu().numpy()).sum())
    t = e0.elapsed_time(e1) / 1e3
    return {"place_kernels": K, "workload": args.workload, "races": rb.n_races, "s": t,
            "competitor_steps_per_s": cs / t}


def run_surrogate_kernels(mode: str, races: int) -> dict:
    """The surrogate's kernels alone on a small uneven workload (for profiler captures)."""
    import torch

    from paper_2108_02419_gb300 import bbe

    n = races or 100_000
    rb = W.uneven_batch(seed=400, n_races=n, rollouts=1000)
    s = bbe.bbe_surrogate_create(1)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    out = {"surrogate_kernels": mode, "races": n, "rows": rb.n_total}
    try:
        with bbe.Batch(rb) as b:
            if mode == "forward":
                p = torch.empty(rb.n_total, dtype=torch.float32, device="cuda")
                ms = []
                for _ in range(3):
                    ev[0].record()
                    bbe.bbe_surrogate_forward(s, b.handle, p)
                    ev[1].record()
                    ev[1].synchronize()
                    ms.append(ev[0].elapsed_time(ev[1]))
                out["forward_ms"] = ms
            else:
                c, _ = b.rollout()
                p, _ = b.win_probs(c)
                ev[0].record()
                bbe.bbe_surrogate_train(s, b.handle, p, batch_states=4096, steps=4)
                ev[1].record()
                ev[1].synchronize()
                out["train_ms_per_step"] = ev[0].elapsed_time(ev[1]) / 4
            bbe.bbe_surrogate_status(s)
    finally:
        bbe.bbe_surrogate_destroy(s)
    return out


def make_workload(name: str, rank: int = 0, races: int = 0) -> W.RaceBatch:
    if name == "uniform":
        rb = W.uniform_batch(seed=0)
    elif name == "uneven":
        rb = W.uneven_batch(seed=0)
    else:
        rb = W.single_race_start(seed=0)
    if races and races < rb.n_races:
        rb = rb.slice(0, races)
    # weak scaling: rank r simulates its own races, ids offset past the other ranks'
    return W.for_rank(rb, rank)


def workload_config(name: str, rb: W.RaceBatch) -> dict:
    sizes = rb.sizes()
    cfg = {
        "uniform": {"workload": "uniform mid-race snapshots", "races": rb.n_races, "competitors": int(sizes[0]),
                    "track_len": 5000, "rollouts_per_race": int(rb.rollouts[0]),
                    "positions": "U(0, 0.9 L)"},
        "uneven": {"workload": "uneven snapshots, one persistent launch", "races": rb.n_races,
                   "competitors": "U{2..24}", "track_len": 5000, "remaining": "U(100, 5000)",
                   "rollouts_per_race": "floor(10^U(3,5))"},
        "single": {"workload": "single race from the start line", "races": 1, "competitors": int(sizes[0]),
                   "track_len": 2000, "rollouts_per_race": int(rb.rollouts[0])},
    }[name]
    cfg.update({"params": "mu U(15,17), sigma U(0.5,1.5), rho U(0,1), P 1, theta 1", "seed": 0,
                "dist": "normal (Box-Muller)", "total_rollouts": int(rb.rollouts.sum()),
                "competitors_total": rb.n_total})
    return cfg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


# the sources of the win-count rollout kernel (a traffic record applies while they hash the same)
KERNEL_SOURCES = ("bbe_win.cuh", "bbe_win.cu", "bbe_rng.cuh", "bbe_internal.h")


def kernel_sources_sha16() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2108_02419_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def kernel_traffic(workload: str, races: int):
    """DRAM bytes per rollout launch from the committed ncu record, or None when the kernel
    sources changed since the counters were taken (or the workload is not the recorded one)."""
    path = os.path.join(ROOT, "profiles", "rollout_kernel_traffic.json")
    if races or not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if kernel_sources_sha16() != rec.get("kernel_sources_sha256_16"):
        return None
    w = rec.get("workloads", {}).get(workload)
    return None if w is None else w["dram_bytes_per_launch"]


def competitor_steps(rb: W.RaceBatch, steps_total: np.ndarray) -> int:
    return int((rb.sizes() * steps_total.astype(np.int64)).sum())


# ---------------------------------------------------------------------------- oracle leg

def oracle_sample(rb: W.RaceBatch, seconds: float, threads: int):
    """Time the CPU oracle (as it stands) on a leading sample of the workload's races, sized
    to about `seconds` of CPU time on `threads` threads.  Returns (comp-steps/s, description)."""
    import oracle

    oracle.build()
    # calibrate on one chunk of race 0
    probe = min(int(rb.rollouts[0]), 500)
    t0 = time.perf_counter()
    _, st, _ = oracle.race_counts(rb.race(0), rb.seed, R=probe)
    per_rollout_s = (time.perf_counter() - t0) / probe
    rollouts_target = max(1, int(seconds * threads / max(per_rollout_s, 1e-9)))
    races, tot = [], 0
    for r in range(rb.n_races):
        races.append(r)
        tot += int(rb.rollouts[r])
        if tot >= rollouts_target:
            break
    t0 = time.perf_counter()
    _, steps, _ = oracle.batch_counts(rb, races=races, threads=threads)
    dt = time.perf_counter() - t0
    cs = int((rb.sizes()[races] * steps).sum())
    desc = f"races 0..{races[-1]} of the workload ({len(races)} races, {tot} rollouts, {cs} competitor-steps), {dt:.1f} s"
    return cs / dt, desc, dt


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step a bounded sample of the same workload."""
    if rank != 0:
        return
    import oracle

    oracle.build()
    rb = make_workload(args.workload, 0, args.races)
    threads = os.cpu_count() or 1
    # size one step to ~1.5 s of CPU work on all cores
    probe = min(int(rb.rollouts[0]), 400)
    t0 = time.perf_counter()
    oracle.race_counts(rb.race(0), rb.seed, R=probe)
    per_rollout = (time.perf_counter() - t0) / probe
    target = max(1, int(1.5 * threads / max(per_rollout, 1e-9)))
    races, tot = [], 0
    for r in range(rb.n_races):
        races.append(r)
        tot += int(rb.rollouts[r])
        if tot >= target:
            break
    units, times = 0, []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, steps, _ = oracle.batch_counts(rb, races=races, threads=threads)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            units = int((rb.sizes()[races] * steps).sum())
    total = sum(times)
    value = units * len(times) / total
    sample = f"races 0..{races[-1]} ({len(races)} races, {tot} rollouts, {units} competitor-steps) per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args.workload, rb),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- surrogate leg

# algorithmic FLOPs per competitor row of the surrogate network (one forward pass):
# 2 x (5*128 + 128*128 + 128*128 + 256*128 + 128)
SURROGATE_FWD_FLOPS_PER_ROW = 2 * (5 * 128 + 2 * 128 * 128 + 256 * 128 + 128)
# Monte Carlo budget of a query: about what plain Monte Carlo needs for a 0.01 max-abs error
# over 1e4 states (4.5 sigma of a binomial proportion at p = 1/2)
QUERY_ROLLOUTS = 50000
# confidence gate of the surrogate: a race whose runner-up network probability exceeds the
# threshold goes to Monte Carlo.  The threshold is chosen in the run itself, on two held-out
# sets (seeds 300 and 301), as the largest candidate whose network-answered races stay within
# GATE_ERR of the 10^5-rollout references on both; the third set (seed 302) reports the error.
GATE_CANDIDATES = (1e-3, 2e-3, 5e-3, 1e-2, 2e-2, 3e-2, 5e-2)
GATE_ERR = 0.005
# two-stage fallback: a pilot of this many rollouts, then the budget that bounds every
# probability's standard deviation by FALLBACK_SD (0.01 / 4.5: a 0.01 max-abs error over the
# ~10^5 probabilities a run reports, at 4.5 standard deviations)
FALLBACK_PILOT = 2000
FALLBACK_SD = 0.01 / 4.5


def _race_errors(P, Q, off):
    err = np.abs(P - Q)
    kl = np.where(P > 0, P * (np.log(np.maximum(P, 1e-30)) - np.log(np.maximum(Q, 1e-30))), 0.0)
    return err, np.add.reduceat(kl, off[:-1])


def _errors(P, Q, off, mask_races=None):
    err, klr = _race_errors(P, Q, off)
    if mask_races is not None:
        err = err[np.repeat(mask_races, np.diff(off))]
        klr = klr[mask_races]
    return {"max_abs": float(err.max()), "mean_abs": float(err.mean()), "p99_abs": float(np.quantile(err, 0.99)),
            "kl_mean": float(klr.mean()), "kl_max": float(klr.max())}


def _runner_up(Q, off):
    return np.array([np.sort(Q[off[r]:off[r + 1]])[-2] if off[r + 1] - off[r] > 1 else 0.0
                     for r in range(off.size - 1)])


def run_surrogate(mode: str, dev, stream) -> dict:
    """Training-data generation, training (the 14-input network and the five-input one of the
    stated configuration), the confidence gate chosen on held-out states, the error on other
    held-out states against 10^5- and 10^6-rollout Monte Carlo, and inference throughput next
    to plain Monte Carlo on the uneven workload."""
    import torch

    from paper_2108_02419_gb300 import bbe

    full = mode == "full"
    n_train = 4_000_000 if full else 200_000
    epochs = 100 if full else 4
    B = 4096
    ev = lambda: torch.cuda.Event(enable_timing=True)
    e0, e1 = ev(), ev()
    out = {"mode": mode, "train_states": n_train, "train_rollouts": 10000, "epochs": epochs, "batch": B}

    def timed(fn):
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3

    # C3: (state, win-prob) pairs from the uneven generator at 1e4 rollouts, on the GPU
    gen = W.uneven_batch(seed=100, n_races=n_train, rollouts=10000)
    t0 = time.perf_counter()
    tb = bbe.Batch(gen, stream=stream)
    out["train_stage_s"] = time.perf_counter() - t0
    counts = torch.empty(gen.n_total, dtype=torch.int32, device=dev)
    steps_t = torch.empty(gen.n_races, dtype=torch.int64, device=dev)
    probs = torch.empty(gen.n_total, dtype=torch.float32, device=dev)
    out["gen_s"] = timed(lambda: (tb.rollout(counts, steps_t, stream=stream), tb.win_probs(counts, probs, stream=stream)))
    gcs = int((gen.sizes() * steps_t.cpu().numpy()).sum())
    out["gen_competitor_steps_per_s"] = gcs / out["gen_s"]
    nets = {}
    try:
        for inputs in (14, 5):
            s = bbe.bbe_surrogate_create(1)
            nets[inputs] = s
            bbe.bbe_surrogate_set_inputs(s, inputs)
            nsteps = int(epochs * n_train / B)
            log = torch.empty(nsteps, dtype=torch.float32, device=dev)
            lr0, chunk = 2e-3, 250

            def train():
                done = 0
                while done < nsteps:
                    k = min(chunk, nsteps - done)
                    lr = lr0 * 0.5 * (1.0 + np.cos(np.pi * done / nsteps))  # cosine decay, per chunk
                    bbe.bbe_surrogate_train(s, tb.handle, probs, lr=float(lr), batch_states=B, steps=k,
                                            loss_log=log[done:done + k], shuffle_seed=7, stream=stream)
                    done += k

            t_tr = timed(train)
            L = log.cpu().numpy()
            rows = float(gen.sizes().mean()) * B * nsteps
            # the loss curve: the mean training loss over each tenth of the run
            curve = [round(float(c.mean()), 5) for c in np.array_split(L, 10)]
            tr = {"train_steps": nsteps, "train_s": t_tr, "loss_first": float(L[:10].mean()),
                  "loss_last": float(L[-10:].mean()), "loss_curve_tenths": curve, "train_states_per_s": nsteps * B / t_tr,
                  "train_tflops": 3 * SURROGATE_FWD_FLOPS_PER_ROW * rows / t_tr / 1e12}
            if inputs == 14:
                out.update(tr)
            else:
                out["five_input"] = tr
        tb.close()

        # held-out states against 10^5-rollout Monte Carlo: seeds 300, 301 choose the gate,
        # seed 302 reports; network outputs with the gate open
        held_sets = {}
        for seed in (300, 301, 302):
            ho = W.uneven_batch(seed=seed, n_races=10000, rollouts=100000)
            with bbe.Batch(ho, stream=stream) as hb:
                hc = torch.empty(ho.n_total, dtype=torch.int32, device=dev)
                hp = torch.empty(ho.n_total, dtype=torch.float32, device=dev)
                hs = torch.empty(ho.n_races, dtype=torch.int64, device=dev)
                hb.rollout(hc, hs, stream=stream)
                hb.win_probs(hc, hp, stream=stream)
                stream.synchronize()
                P = hp.cpu().numpy().astype(np.float64)
            hq = dataclasses.replace(ho, rollouts=np.full(ho.n_races, QUERY_ROLLOUTS, np.int64), seed=seed + 1000)
            qb = bbe.Batch(hq, stream=stream)
            Qn = {}
            for inputs, s in nets.items():
                q = torch.empty(ho.n_total, dtype=torch.float32, device=dev)
                used = torch.empty(ho.n_races, dtype=torch.uint8, device=dev)
                bbe.bbe_surrogate_set_gate(s, 1.0)
                bbe.bbe_surrogate_infer(s, qb.handle, q, used, stream=stream)
                stream.synchronize()
                Qn[inputs] = q.cpu().numpy().astype(np.float64)
            held_sets[seed] = (ho, qb, P, Qn)

        def choose_gate(inputs):
            best = GATE_CANDIDATES[0]
            for thr in GATE_CANDIDATES:
                ok = True
                for seed in (300, 301):
                    ho, _, P, Qn = held_sets[seed]
                    err, _ = _race_errors(P, Qn[inputs], ho.race_off)
                    answered = _runner_up(Qn[inputs], ho.race_off) <= thr
                    ok = ok and (not answered.any() or err[np.repeat(answered, ho.sizes())].max() <= GATE_ERR)
                if ok:
                    best = thr
            return best

        gates = {inputs: choose_gate(inputs) for inputs in nets}
        out["gate"] = {"candidates": list(GATE_CANDIDATES), "max_err_on_choice_sets": GATE_ERR,
                       "chosen_14": gates[14], "chosen_5": gates[5], "choice_sets": [300, 301], "report_set": 302}
        ho, qb, P, Qn = held_sets[302]
        held = {"states": ho.n_races, "reference_rollouts": 100000, "query_rollouts": QUERY_ROLLOUTS}
        held["network"] = _errors(P, Qn[14], ho.race_off)
        ru = _runner_up(Qn[14], ho.race_off)
        held["network_answered"] = _errors(P, Qn[14], ho.race_off, ru <= gates[14])
        held["network_answered"]["races"] = int((ru <= gates[14]).sum())
        s = nets[14]
        q = torch.empty(ho.n_total, dtype=torch.float32, device=dev)
        used = torch.empty(ho.n_races, dtype=torch.uint8, device=dev)
        bbe.bbe_surrogate_set_gate(s, gates[14])
        bbe.bbe_surrogate_infer(s, qb.handle, q, used, stream=stream)
        stream.synchronize()
        Qg = q.cpu().numpy().astype(np.float64)
        held["gated"] = _errors(P, Qg, ho.race_off)
        u = used.cpu().numpy()
        held["gated"].update(runner_up_max=gates[14], gated=int((u == 2).sum()), out_of_range=int((u == 1).sum()))
        bbe.bbe_surrogate_set_fallback(s, FALLBACK_PILOT, FALLBACK_SD)
        bbe.bbe_surrogate_infer(s, qb.handle, q, used, stream=stream)
        stream.synchronize()
        Qg2 = q.cpu().numpy().astype(np.float64)
        held["gated_two_stage"] = _errors(P, Qg2, ho.race_off)
        fr, fro = bbe.bbe_surrogate_fallback_stats(s)
        held["gated_two_stage"].update(pilot=FALLBACK_PILOT, max_sd=FALLBACK_SD, fallback_races=fr,
                                       fallback_rollouts_mean=fro / max(fr, 1))
        bbe.bbe_surrogate_set_fallback(s, 0)
        mcq_c = torch.empty(ho.n_total, dtype=torch.int32, device=dev)
        mcq_p = torch.empty(ho.n_total, dtype=torch.float32, device=dev)
        qb.rollout(mcq_c, stream=stream)
        qb.win_probs(mcq_c, mcq_p, stream=stream)
        stream.synchronize()
        held["mc_at_query_rollouts"] = _errors(P, mcq_p.cpu().numpy().astype(np.float64), ho.race_off)
        # the five-input network on the same states
        ru5 = _runner_up(Qn[5], ho.race_off)
        out["five_input"].update(network=_errors(P, Qn[5], ho.race_off), gate=gates[5],
                                 answered=_errors(P, Qn[5], ho.race_off, ru5 <= gates[5]),
                                 gated_share=float((ru5 > gates[5]).mean()))
        # the first 1000 report states against 10^6-rollout Monte Carlo
        n6 = 1000
        r6 = W.uneven_batch(seed=302, n_races=10000, rollouts=1_000_000).slice(0, n6)
        with bbe.Batch(r6, stream=stream) as b6:
            c6 = torch.empty(r6.n_total, dtype=torch.int32, device=dev)
            p6 = torch.empty(r6.n_total, dtype=torch.float32, device=dev)
            b6.rollout(c6, stream=stream)
            b6.win_probs(c6, p6, stream=stream)
            stream.synchronize()
            P6 = p6.cpu().numpy().astype(np.float64)
        k6 = int(r6.race_off[-1])
        off6 = r6.race_off
        out["reference_1e6"] = {"states": n6, "rollouts": 1_000_000,
                                "reference_1e5_vs_1e6": _errors(P6, P[:k6], off6),
                                "network": _errors(P6, Qn[14][:k6], off6),
                                "gated": _errors(P6, Qg[:k6], off6),
                                "gated_two_stage": _errors(P6, Qg2[:k6], off6),
                                "mc_at_query_rollouts": _errors(P6, mcq_p.cpu().numpy()[:k6].astype(np.float64), off6),
                                "five_input_network": _errors(P6, Qn[5][:k6], off6)}
        out["heldout"] = held
        for seed in (300, 301, 302):
            held_sets[seed][1].close()

        # C4: 1e6 queries drawn as in the uneven workload, network alone and gated
        qrb = W.uneven_batch(seed=400, n_races=1_000_000 if full else 100_000, rollouts=QUERY_ROLLOUTS)
        t0 = time.perf_counter()
        qb = bbe.Batch(qrb, stream=stream)
        out["query_stage_s"] = time.perf_counter() - t0
        qp = torch.empty(qrb.n_total, dtype=torch.float32, device=dev)
        qu = torch.empty(qrb.n_races, dtype=torch.uint8, device=dev)
        qrows = float(qrb.n_total)
        bbe.bbe_surrogate_set_gate(s, 1.0)
        bbe.bbe_surrogate_infer(s, qb.handle, qp, qu, stream=stream)  # plans once per batch
        t_inf = min(timed(lambda: bbe.bbe_surrogate_infer(s, qb.handle, qp, qu, stream=stream)) for _ in range(3))
        out["infer"] = {"states": qrb.n_races, "s": t_inf, "win_prob_vectors_per_s": qrb.n_races / t_inf,
                        "used_mc": int(qu.cpu().numpy().sum()),
                        "tflops": SURROGATE_FWD_FLOPS_PER_ROW * qrows / t_inf / 1e12}
        bbe.bbe_surrogate_set_gate(s, gates[14])
        t_g = timed(lambda: bbe.bbe_surrogate_infer(s, qb.handle, qp, qu, stream=stream))
        u = qu.cpu().numpy()
        out["infer_gated"] = {"states": qrb.n_races, "s": t_g, "win_prob_vectors_per_s": qrb.n_races / t_g,
                              "runner_up_max": gates[14], "gated": int((u == 2).sum()),
                              "out_of_range": int((u == 1).sum()), "fallback_rollouts": QUERY_ROLLOUTS}
        bbe.bbe_surrogate_set_fallback(s, FALLBACK_PILOT, FALLBACK_SD)
        t_g2 = timed(lambda: bbe.bbe_surrogate_infer(s, qb.handle, qp, qu, stream=stream))
        fr, fro = bbe.bbe_surrogate_fallback_stats(s)
        ft = bbe.bbe_surrogate_fallback_times(s)
        out["infer_gated_two_stage"] = {"states": qrb.n_races, "s": t_g2, "win_prob_vectors_per_s": qrb.n_races / t_g2,
                                        "runner_up_max": gates[14], "pilot": FALLBACK_PILOT, "max_sd": FALLBACK_SD,
                                        "fallback_races": fr, "fallback_rollouts_mean": fro / max(fr, 1),
                                        "fallback_phase_s": {"stage": ft[0], "pilot": ft[1], "budget": ft[2],
                                                             "stage_topup": ft[3], "topup_and_finish": ft[4]}}
        # the same queries with 3 % of them outside the training ranges (26 to 30 competitors
        # against the trained 2 to 24), which the range check sends to Monte Carlo
        n_oor = qrb.n_races * 3 // 100
        oor = W.uneven_batch(seed=401, n_races=n_oor, n_lo=26, n_hi=30, rollouts=QUERY_ROLLOUTS)
        mixed = W.concat([qrb.slice(0, qrb.n_races - n_oor), oor])
        mb = bbe.Batch(mixed, stream=stream)
        mp = torch.empty(mixed.n_total, dtype=torch.float32, device=dev)
        mu8 = torch.empty(mixed.n_races, dtype=torch.uint8, device=dev)
        bbe.bbe_surrogate_infer(s, mb.handle, mp, mu8, stream=stream)  # plans once per batch
        t_m = timed(lambda: bbe.bbe_surrogate_infer(s, mb.handle, mp, mu8, stream=stream))
        um = mu8.cpu().numpy()
        out["infer_with_out_of_range"] = {"states": mixed.n_races, "planted_out_of_range": n_oor,
                                          "out_of_range": int((um == 1).sum()),
                                          "out_of_range_among_planted": int((um[-n_oor:] == 1).sum()),
                                          "gated": int((um == 2).sum()), "s": t_m,
                                          "win_prob_vectors_per_s": mixed.n_races / t_m}
        mb.close()
        bbe.bbe_surrogate_set_fallback(s, 0)
        qb.close()
        # plain Monte Carlo at the query budget on a 20,000-query sample of the same stream
        ms = qrb.slice(0, 20000)
        with bbe.Batch(ms, stream=stream) as mb:
            mcnt = torch.empty(ms.n_total, dtype=torch.int32, device=dev)
            mstp = torch.empty(ms.n_races, dtype=torch.int64, device=dev)
            mpr = torch.empty(ms.n_total, dtype=torch.float32, device=dev)
            t_ms = timed(lambda: (mb.rollout(mcnt, mstp, stream=stream), mb.win_probs(mcnt, mpr, stream=stream)))
            # the same two-stage rule without the network: every race through the fallback
            # (gate 0), so the comparison isolates what the network adds
            mq = torch.empty(ms.n_total, dtype=torch.float32, device=dev)
            mu_ = torch.empty(ms.n_races, dtype=torch.uint8, device=dev)
            bbe.bbe_surrogate_set_gate(s, 0.0)
            bbe.bbe_surrogate_set_fallback(s, FALLBACK_PILOT, FALLBACK_SD)
            t_m2 = timed(lambda: bbe.bbe_surrogate_infer(s, mb.handle, mq, mu_, stream=stream))
            fr, fro = bbe.bbe_surrogate_fallback_stats(s)
            bbe.bbe_surrogate_set_fallback(s, 0)
            bbe.bbe_surrogate_set_gate(s, gates[14])
        out["mc_at_query_rollouts"] = {"states": ms.n_races, "s": t_ms, "win_prob_vectors_per_s": ms.n_races / t_ms,
                                       "rollouts": QUERY_ROLLOUTS}
        out["mc_two_stage"] = {"states": ms.n_races, "s": t_m2, "win_prob_vectors_per_s": ms.n_races / t_m2,
                               "pilot": FALLBACK_PILOT, "max_sd": FALLBACK_SD, "races": fr,
                               "rollouts_mean": fro / max(fr, 1)}
        out["gain_gated_vs_mc_at_query_rollouts"] = out["infer_gated"]["win_prob_vectors_per_s"] / (ms.n_races / t_ms)
        out["gain_gated_two_stage_vs_mc_at_query_rollouts"] = (out["infer_gated_two_stage"]["win_prob_vectors_per_s"]
                                                               / (ms.n_races / t_ms))
        out["gain_gated_two_stage_vs_mc_two_stage"] = (out["infer_gated_two_stage"]["win_prob_vectors_per_s"]
                                                       / (ms.n_races / t_m2))
    finally:
        for s_ in nets.values():
            bbe.bbe_surrogate_destroy(s_)
    # plain Monte Carlo on the uneven workload (10,000 snapshots, budgets 1e3..1e5)
    u = W.uneven_batch(seed=0)
    with bbe.Batch(u, stream=stream) as ub:
        uc = torch.empty(u.n_total, dtype=torch.int32, device=dev)
        us = torch.empty(u.n_races, dtype=torch.int64, device=dev)
        up = torch.empty(u.n_total, dtype=torch.float32, device=dev)
        timed(lambda: (ub.rollout(uc, us, stream=stream), ub.win_probs(uc, up, stream=stream)))
        t_mc = min(timed(lambda: (ub.rollout(uc, us, stream=stream), ub.win_probs(uc, up, stream=stream)))
                   for _ in range(2))
    out["mc"] = {"workload": "uneven 10,000 snapshots, rollouts floor(10^U(3,5))", "win_prob_vectors_per_s": u.n_races / t_mc}
    out["gain_network_vs_mc_uneven"] = out["infer"]["win_prob_vectors_per_s"] / (u.n_races / t_mc)
    return out


# ---------------------------------------------------------------------------- place-count leg

def run_places(dev, stream) -> dict:
    """Finishing places (rollouts to the K-th finisher) on the uniform workload: K = 3 (a
    three-place market) and K = 20 (the full order), next to the win counts (K = 1)."""
    import torch

    from paper_2108_02419_gb300 import bbe

    rb = W.uniform_batch(seed=0)
    out = {"workload": "uniform 4096 x 20, L 5000, 10,000 rollouts per race", "ops_per_competitor_step": ALG_OPS_PER_COMPETITOR_STEP}
    peak = SMS * LANES_PER_SM * 2070e6
    with bbe.Batch(rb, stream=stream) as b:
        for K in (3, 20):
            counts = torch.empty((rb.n_total, K), dtype=torch.int32, device=dev)
            steps = torch.empty(rb.n_races, dtype=torch.int64, device=dev)
            bbe.bbe_place_counts(b.handle, K, counts, steps, stream)  # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bbe.bbe_place_counts(b.handle, K, counts, steps, stream)
            e1.record(stream)
            e1.synchronize()
            b.status(stream)
            t = e0.elapsed_time(e1) / 1e3
            cs = float((rb.sizes() * steps.cpu().numpy()).sum())
            rate = cs / t
            out[f"K{K}"] = {"s": t, "competitor_steps": cs, "competitor_steps_per_s": rate,
                            "steps_per_rollout": cs / float(rb.n_total) / 10000.0,
                            "alu_frac": rate * ALG_OPS_PER_COMPETITOR_STEP / peak}
        # ordered top-3 tallies (tricast) in the same pass as the place counts
        total = bbe.bbe_order_table_size(b.handle, 3)
        orders = torch.empty(total, dtype=torch.int32, device=dev)
        counts = torch.empty((rb.n_total, 3), dtype=torch.int32, device=dev)
        bbe.bbe_order_counts(b.handle, 3, orders, counts, steps, stream)  # warm-up (uploads the layout)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bbe.bbe_order_counts(b.handle, 3, orders, counts, steps, stream)
        e1.record(stream)
        e1.synchronize()
        b.status(stream)
        t = e0.elapsed_time(e1) / 1e3
        cs = float((rb.sizes() * steps.cpu().numpy()).sum())
        out["K3_orders"] = {"s": t, "table_entries": total, "competitor_steps_per_s": cs / t,
                            "tuples_counted": int(orders.sum().item())}
        del orders, counts
        # the full finishing order (K = 20 of 20: 20! possible orders) as per-race hash tables
        off = bbe.bbe_order_histogram_layout(b.handle, 20, rb.n_races)
        entries = int(off[-1])
        keys = torch.empty(entries, dtype=torch.uint64, device=dev)
        hc = torch.empty(entries, dtype=torch.int32, device=dev)
        bbe.bbe_order_histogram(b.handle, 20, keys, hc, None, steps, stream)  # warm-up (uploads the layout)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bbe.bbe_order_histogram(b.handle, 20, keys, hc, None, steps, stream)
        e1.record(stream)
        e1.synchronize()
        b.status(stream)
        t = e0.elapsed_time(e1) / 1e3
        cs = float((rb.sizes() * steps.cpu().numpy()).sum())
        out["K20_histogram"] = {"s": t, "table_entries": entries, "table_bytes": entries * 12,
                                "distinct_orders": int((hc > 0).sum().item()),
                                "orders_counted": int(hc.sum(dtype=torch.int64).item()),
                                "competitor_steps_per_s": cs / t,
                                "alu_frac": cs / t * ALG_OPS_PER_COMPETITOR_STEP / peak}
        del keys, hc
    return out


# ---------------------------------------------------------------------------- bettor-population leg

def run_population(dev, stream, bettors: int = 1000, dry_runs: int = 50) -> dict:
    """Section 6's use case on the single-race workload (5 competitors, L 2000): one actual race
    (a full trajectory), and at every step until the first competitor crosses, `bettors` RP(d)
    bettors with d = dry_runs dry-runs each on their own streams, plus the rule-based bettors'
    predictions; timed end to end on the device (trajectory, snapshot batch, dry-runs, odds,
    predictions)."""
    import torch

    from paper_2108_02419_gb300 import bbe

    rb = W.single_race_start(seed=0)
    cap, every, k_actual, id0 = 1024, 1, 1 << 30, 1 << 20
    out = {"workload": "single race, 5 competitors, L 2000; snapshots every step until the first finisher",
           "bettors": bettors, "dry_runs": dry_runs}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with bbe.Batch(rb, stream=stream) as b:
        pos = torch.empty(rb.n_total * cap, dtype=torch.float32, device=dev)
        stp = torch.empty_like(pos)
        ns = torch.empty(rb.n_races, dtype=torch.int32, device=dev)
        for rep in range(2):  # the first pass warms up
            t0 = time.perf_counter()
            ev[0].record(stream)
            bbe.bbe_race_trajectory(b.handle, k_actual, cap, pos, stp, ns, stream)
            h, n_snap = bbe.bbe_snapshot_batch(b.handle, 0, pos, stp, ns, cap, every, bettors, dry_runs, id0, stream)
            try:
                nc = n_snap * bettors * rb.n_total
                counts = torch.empty(nc, dtype=torch.int32, device=dev)
                steps = torch.empty(n_snap * bettors, dtype=torch.int64, device=dev)
                probs = torch.empty(nc, dtype=torch.float32, device=dev)
                odds = torch.empty(nc, dtype=torch.float32, device=dev)
                e2 = torch.cuda.Event(enable_timing=True)
                e3 = torch.cuda.Event(enable_timing=True)
                e2.record(stream)
                bbe.bbe_rollout_batch(h, counts, steps, stream)
                e3.record(stream)
                bbe.bbe_win_probs(h, counts, probs, odds, stream)
                pred = torch.empty(n_snap * 4, dtype=torch.int32, device=dev)
                bbe.bbe_bettor_predictions(b.handle, 0, pos, stp, ns, cap, every, n_snap, 10, 3.0, 77, pred, stream)
                ev[1].record(stream)
                ev[1].synchronize()
                wall = time.perf_counter() - t0
                bbe.bbe_batch_status(h, stream)
            finally:
                bbe.bbe_destroy_batch(h)
        t_all = ev[0].elapsed_time(ev[1]) / 1e3
        t_dry = e2.elapsed_time(e3) / 1e3
        cs = float(steps.sum().item()) * rb.n_total
        T = int(ns[0].item())
        P = pos[:T * rb.n_total].view(T, rb.n_total).cpu().numpy()
        S = stp[:T * rb.n_total].view(T, rb.n_total).cpu().numpy()
        cnt = counts.view(n_snap, bettors, rb.n_total).cpu().numpy()
        pr = pred.view(n_snap, 4).cpu().numpy()
    # the actual winner: first step across the line, then the crossing time within it
    prev = np.vstack([rb.d0[None, :], P[:-1]])
    cross = [int(np.argmax(P[:, c] >= rb.L[0])) for c in range(rb.n_total)]
    tau = [np.float32(np.float32(rb.L[0]) - prev[cross[c], c]) / S[cross[c], c] for c in range(rb.n_total)]
    winner = min(range(rb.n_total), key=lambda c: (cross[c], tau[c], c))
    rp_pick = cnt.argmax(axis=2)                  # each bettor's favourite at each snapshot
    pooled = cnt.sum(axis=1) / float(bettors * dry_runs)  # all bettors' dry-runs pooled
    out.update({
        "snapshots": n_snap, "actual_race_steps": T, "actual_winner": winner,
        "dry_runs_total": n_snap * bettors * dry_runs,
        "s_end_to_end_device": t_all, "s_wall": wall, "s_dry_runs": t_dry,
        "dry_runs_per_s": n_snap * bettors * dry_runs / t_dry,
        "competitor_steps_per_s": cs / t_dry,
        "bettor_updates_per_s_end_to_end": n_snap * bettors / t_all,
        "pick_is_winner": {"RP(d) bettor": float((rp_pick == winner).mean()),
                           "pooled dry-runs": float((pooled.argmax(axis=1) == winner).mean()),
                           "LW": float((pr[:, 0] == winner).mean()), "UD(3)": float((pr[:, 1] == winner).mean()),
                           "LinEx(10)": float((pr[:, 2] == winner).mean()), "ZI": float((pr[:, 3] == winner).mean())},
        # each rule scored against the Monte Carlo probabilities at every snapshot (all bettors'
        # dry-runs pooled, 50,000 per snapshot): the probability that its pick wins, and how often
        # it picks the Monte Carlo favourite
        "mc_prob_of_pick": {"RP(d) bettor": float(np.take_along_axis(pooled, rp_pick, axis=1).mean()),
                            **{name: float(pooled[np.arange(n_snap), pr[:, i]].mean())
                               for i, name in enumerate(("LW", "UD(3)", "LinEx(10)", "ZI"))}},
        "picks_mc_favourite": {"RP(d) bettor": float((rp_pick == pooled.argmax(axis=1)[:, None]).mean()),
                               **{name: float((pr[:, i] == pooled.argmax(axis=1)).mean())
                                  for i, name in enumerate(("LW", "UD(3)", "LinEx(10)", "ZI"))}},
    })
    # the live use (Section 6: every bettor re-evaluates at each step): one snapshot's bettors
    # alone, the race's positions at the middle snapshot, `bettors` races of `dry_runs` rollouts on
    # the bettors' own streams; device time of the rollouts and probabilities, and end to end
    # from host buffers
    s_mid = max(1, n_snap // 2)
    snap = W.from_arrays([rb.n_total] * bettors, float(rb.L[0]), dry_runs, np.tile(P[s_mid * every - 1], bettors),
                         np.tile(rb.mu, bettors), np.tile(rb.sigma, bettors), np.tile(rb.rho, bettors),
                         P=np.tile(rb.P, bettors), theta=np.tile(rb.theta, bettors), seed=rb.seed)
    snap.race_id0 = id0 + s_mid * bettors
    sc = torch.empty(snap.n_total, dtype=torch.int32, device=dev)
    ss = torch.empty(snap.n_races, dtype=torch.int64, device=dev)
    sp = torch.empty(snap.n_total, dtype=torch.float32, device=dev)
    so = torch.empty(snap.n_total, dtype=torch.float32, device=dev)
    with bbe.Batch(snap, stream=stream) as sb:
        times, _ = _device_passes(sb, snap, sc, ss, sp, stream, dev, passes=20, warmup=3)
    e2e_s, _, _ = _e2e_calls(snap, sc, sp, so, stream, dev, calls=20)
    out["one_snapshot"] = {"bettors": bettors, "dry_runs": dry_runs, "snapshot_step": s_mid * every,
                           "device_ms_median": float(np.median(times)) * 1e3, "e2e_ms_median": e2e_s * 1e3}
    return out



# ---------------------------------------------------------------------------- batching legs

def _peak_ops() -> float:
    return SMS * LANES_PER_SM * float(measured_peaks().get("sm_max_mhz", 2070.0)) * 1e6


def _device_passes(batch, rb, counts, steps_t, probs, stream, dev, passes: int, warmup: int = 2, flush=None):
    """Device time (CUDA events on the batch's stream) of `passes` rollout + probability passes,
    after `warmup` untimed ones; L2 flushed between passes when `flush` is given."""
    import torch

    for _ in range(warmup):
        batch.rollout(counts, steps_t, stream=stream)
        batch.win_probs(counts, probs, stream=stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(passes)]
    for i in range(passes):
        if flush is not None:
            flush.fill_(i)
        ev[i][0].record(stream)
        batch.rollout(counts, steps_t, stream=stream)
        batch.win_probs(counts, probs, stream=stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    batch.status(stream)
    return [a.elapsed_time(b) / 1e3 for a, b in ev], competitor_steps(rb, steps_t.cpu().numpy())


def _e2e_calls(rb, counts, probs, odds, stream, dev, calls: int, cfg=None, layout=None):
    """End to end through the public API: pinned host inputs -> bbe_race_init (H2D inside) ->
    [launch configuration] -> rollouts -> probabilities -> D2H of probabilities and counts.
    Median seconds per call, and the bytes copied each way."""
    import torch

    from paper_2108_02419_gb300 import bbe

    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    host = {k: pin(getattr(rb, k)) for k in ("race_off", "L", "rollouts", "d0", "mu", "sigma", "rho", "P", "theta")}
    h_probs = torch.empty(rb.n_total, dtype=torch.float32).pin_memory()
    h_counts = torch.empty(rb.n_total, dtype=torch.int32).pin_memory()
    times = []
    for i in range(2 + calls):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        h = bbe.bbe_race_init(rb.n_races, host["race_off"], host["L"], host["rollouts"], host["d0"], host["mu"],
                              host["sigma"], host["rho"], host["P"], host["theta"], None, rb.seed, rb.dist,
                              rb.race_id0, stream)
        if layout is not None:
            bbe.bbe_batch_set_layout(h, layout)
        if cfg is not None:
            bbe.bbe_batch_set_cfg(h, **cfg)
        bbe.bbe_rollout_batch(h, counts, None, stream)
        bbe.bbe_win_probs(h, counts, probs, odds, stream)
        h_probs.copy_(probs, non_blocking=True)
        h_counts.copy_(counts, non_blocking=True)
        stream.synchronize()
        dt = time.perf_counter() - t0
        bbe.bbe_destroy_batch(h)
        if i >= 2:
            times.append(dt)
    h2d = sum(int(t.numel() * t.element_size()) for t in host.values())
    return statistics.median(times), h2d, int(h_probs.numel() * 4 + h_counts.numel() * 4)


def run_uneven(dev, stream) -> dict:
    """The uneven batch (10^4 snapshots of 2..24 competitors, remaining distance U(100, 5000),
    budgets floor(10^U(3, 5))) in one captured graph: at the default launch, then at the launch
    the autotuner picks (a layout per competitor count, then the block shape and work-item size),
    device-timed and end to end."""
    import torch

    from paper_2108_02419_gb300 import bbe

    rb = W.uneven_batch(seed=0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    counts = torch.empty(rb.n_total, dtype=torch.int32, device=dev)
    steps_t = torch.empty(rb.n_races, dtype=torch.int64, device=dev)
    probs = torch.empty(rb.n_total, dtype=torch.float32, device=dev)
    odds = torch.empty_like(probs)
    peak = _peak_ops()
    out = {"workload": "uneven 10,000 snapshots, n U{2..24}, L 5000, L - d U(100, 5000), rollouts floor(10^U(3,5))",
           "l2": "flushed between timed passes"}
    with bbe.Batch(rb, stream=stream) as b:
        def leg(tag):
            t, cs = _device_passes(b, rb, counts, steps_t, probs, stream, dev, passes=5, flush=flush)
            m = statistics.mean(t)
            out[tag] = {"value": cs / m, "unit": UNIT, "ms_per_pass": 1e3 * m, "win_prob_vectors_per_s": rb.n_races / m,
                        "alu_frac": ALG_OPS_PER_COMPETITOR_STEP * cs / m / peak, "launches_per_pass":
                        bbe.bbe_batch_launches(b.handle), "cfg": b.cfg(), "layout": b.layout()[1:25].tolist()}
        leg("default")
        t0 = time.perf_counter()
        cfg = b.autotune(counts, budget_ms=20000.0, stream=stream)
        out["autotune_wall_s"] = time.perf_counter() - t0
        leg("autotuned")
        layout = b.layout()
    out["gain_autotuned_vs_default"] = out["autotuned"]["value"] / out["default"]["value"]
    cfg = {k: cfg[k] for k in ("warps_per_block", "blocks_per_sm", "rollouts_per_lane", "max_steps", "slots_per_lane")}
    e, h2d, d2h = _e2e_calls(rb, counts, probs, odds, stream, dev, calls=3, cfg=cfg, layout=layout)
    cs = out["autotuned"]["value"] * out["autotuned"]["ms_per_pass"] / 1e3
    out["e2e"] = {"value": cs / e, "unit": UNIT, "seconds_per_call": e, "h2d_bytes_per_step": h2d,
                  "d2h_bytes_per_step": d2h, "launch": "the autotuned configuration, set on each new batch"}
    return out


def run_single(dev, stream) -> dict:
    """The single start-line race (5 competitors, L 2000, 10^3 rollouts): latency per pass on
    the device (graph replay) and per call end to end."""
    import torch

    from paper_2108_02419_gb300 import bbe

    rb = W.single_race_start()
    counts = torch.empty(rb.n_total, dtype=torch.int32, device=dev)
    steps_t = torch.empty(rb.n_races, dtype=torch.int64, device=dev)
    probs = torch.empty(rb.n_total, dtype=torch.float32, device=dev)
    odds = torch.empty_like(probs)
    with bbe.Batch(rb, stream=stream) as b:
        t, cs = _device_passes(b, rb, counts, steps_t, probs, stream, dev, passes=50, warmup=5)
    e, h2d, d2h = _e2e_calls(rb, counts, probs, odds, stream, dev, calls=20)
    return {"workload": "1 race, 5 competitors from the start line, L 2000, 1000 rollouts",
            "device_ms_per_pass_median": 1e3 * statistics.median(t), "device_ms_per_pass_min": 1e3 * min(t),
            "competitor_steps_per_pass": cs, "e2e_ms_per_call_median": 1e3 * e,
            "e2e_h2d_bytes": h2d, "e2e_d2h_bytes": d2h}


def run_sweep(dev, stream, repeats: int = 10) -> dict:
    """Competitor count against throughput (the analogue of the paper's runtime-against-
    competitors figures, Section 6): 1024 mid-race snapshots of n competitors, L 5000, positions
    U(0, 0.9 L), 2000 rollouts each, n = 2..32; `repeats` timed passes per n, with the
    coefficient of variation of the pass times."""
    import torch

    from paper_2108_02419_gb300 import bbe

    rows = []
    for n in range(2, 33):
        rb = W.uniform_batch(seed=600 + n, n_races=1024, n=n, rollouts=2000)
        counts = torch.empty(rb.n_total, dtype=torch.int32, device=dev)
        steps_t = torch.empty(rb.n_races, dtype=torch.int64, device=dev)
        probs = torch.empty(rb.n_total, dtype=torch.float32, device=dev)
        with bbe.Batch(rb, stream=stream) as b:
            t, cs = _device_passes(b, rb, counts, steps_t, probs, stream, dev, passes=repeats, warmup=2)
        m = statistics.mean(t)
        rows.append({"n": n, "ms_per_pass": 1e3 * m, "cov": statistics.pstdev(t) / m,
                     "competitor_steps_per_s": cs / m, "rollouts_per_s": rb.n_races * 2000 / m})
    return {"workload": "1024 snapshots x n competitors, L 5000, d U(0, 0.9 L), 2000 rollouts, n = 2..32",
            "repeats": repeats, "rows": rows}


def run_oracle_timings(threads: int) -> dict:
    """The CPU oracle as it stands, on one host thread and on all of them: the single race in
    full, and leading samples of the uniform and uneven batches."""
    import oracle

    oracle.build()
    out = {"threads_all": threads}
    rb = W.single_race_start()
    for tag, th in (("single_1thread", 1), ("single_all", threads)):
        t0 = time.perf_counter()
        _, steps, _ = oracle.batch_counts(rb, threads=th)
        dt = time.perf_counter() - t0
        out[tag] = {"value": int((rb.sizes() * steps).sum()) / dt, "unit": UNIT, "s": dt, "sample": "the whole race"}
    for name, wb in (("uniform", W.uniform_batch(seed=0)), ("uneven", W.uneven_batch(seed=0))):
        for tag, th, sec in (("1thread", 1, 4.0), ("all", threads, 4.0)):
            v, desc, _ = oracle_sample(wb, sec, th)
            out[f"{name}_{tag}"] = {"value": v, "unit": UNIT, "cores": th, "sample": desc}
    return out


# ---------------------------------------------------------------------------- GPU leg

def run_gpu(args, rank, world, dist):
    import torch

    from paper_2108_02419_gb300 import bbe

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rb = make_workload(args.workload, rank, args.races)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    batch = bbe.Batch(rb, stream=stream)
    counts = torch.empty(rb.n_total, dtype=torch.int32, device=dev)
    steps_t = torch.empty(rb.n_races, dtype=torch.int64, device=dev)
    probs = torch.empty(rb.n_total, dtype=torch.float32, device=dev)
    odds = torch.empty_like(probs)
    if args.autotune:
        batch.autotune(counts, budget_ms=5000.0, stream=stream)
    l2_flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)  # 256 MB > 129 MB L2

    def one_step():
        batch.rollout(counts, steps_t, stream=stream)
        batch.win_probs(counts, probs, odds, stream=stream)

    for _ in range(args.warmup):
        one_step()
    stream.synchronize()
    batch.status(stream)
    units_per_step = competitor_steps(rb, steps_t.cpu().numpy())
    rollouts_per_step = int(rb.rollouts.sum())
    # kernels of one step: the rollout pass's persistent launches plus the win-probability kernel
    launches_per_step = bbe.bbe_batch_launches(batch.handle) + 1

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        l2_flush.fill_(i)  # flush L2 between timed steps (outside the events)
        ev[i][0].record(stream)
        batch.rollout(counts, steps_t, stream=stream)
        ev[i][1].record(stream)
        batch.win_probs(counts, probs, odds, stream=stream)
        ev[i][2].record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    roll_ms = [a.elapsed_time(b) for a, b, c in ev]
    batch.status(stream)
    t_local = sum(step_ms) / 1e3
    t_max = t_local
    if dist:
        tt = torch.tensor([t_local], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    value = units_per_step * world * args.steps / t_max

    # end to end through the public API: pinned host inputs -> bbe_race_init (H2D) ->
    # rollouts -> probabilities -> D2H of probabilities and counts
    e2e = None
    if not args.no_e2e:
        pin = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        host = {k: pin(getattr(rb, k)) for k in ("race_off", "L", "rollouts", "d0", "mu", "sigma", "rho", "P", "theta")}
        h_probs = torch.empty(rb.n_total, dtype=torch.float32).pin_memory()
        h_counts = torch.empty(rb.n_total, dtype=torch.int32).pin_memory()
        h2d = sum(int(t.numel() * t.element_size()) for t in host.values())
        d2h = int(h_probs.numel() * 4 + h_counts.numel() * 4)
        e_times = []
        for i in range(2 + max(1, min(args.steps, 5))):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            h = bbe.bbe_race_init(rb.n_races, host["race_off"], host["L"], host["rollouts"], host["d0"], host["mu"],
                                  host["sigma"], host["rho"], host["P"], host["theta"], None, rb.seed, rb.dist,
                                  rb.race_id0, stream)
            bbe.bbe_rollout_batch(h, counts, None, stream)
            bbe.bbe_win_probs(h, counts, probs, odds, stream)
            h_probs.copy_(probs, non_blocking=True)
            h_counts.copy_(counts, non_blocking=True)
            stream.synchronize()
            dt = time.perf_counter() - t0
            bbe.bbe_destroy_batch(h)
            if i >= 2:
                e_times.append(dt)
        e_local = statistics.median(e_times)
        if dist:
            tt = torch.tensor([e_local], dtype=torch.float64, device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e_local = float(tt.item())
        e2e = {"value": units_per_step * world / e_local, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "seconds_per_step": e_local}

    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = SMS * LANES_PER_SM * sm_max * 1e6  # lane-operations per second at the maximum SM clock
    roll_s = statistics.mean(roll_ms) / 1e3
    achieved = ALG_OPS_PER_COMPETITOR_STEP * units_per_step / roll_s
    roofline = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak_ops / 1e9, "unit": "Gop/s",
                "frac": achieved / peak_ops, "traffic": kernel_traffic(args.workload, args.races),
                "kernel": "win_rollout_kernel", "ops_per_competitor_step": ALG_OPS_PER_COMPETITOR_STEP,
                "peak_basis": f"{SMS} SMs x {LANES_PER_SM} lanes x {sm_max:.0f} MHz (maximum SM clock)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        v, desc, _ = oracle_sample(rb, args.cpu_seconds, threads)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc}

    batch_cfg = batch.cfg()
    batch.close()
    sur = None
    if rank == 0 and args.surrogate != "off" and not args.races:
        sur = run_surrogate(args.surrogate, dev, stream)
    legs_on = rank == 0 and not args.races and args.workload == "uniform"
    places = run_places(dev, stream) if legs_on else None
    population = run_population(dev, stream) if rank == 0 and not args.races else None
    uneven = run_uneven(dev, stream) if legs_on else None
    single = run_single(dev, stream) if legs_on else None
    sweep = run_sweep(dev, stream) if legs_on else None
    oracle_t = run_oracle_timings(os.cpu_count() or 1) if legs_on and not args.no_cpu_baseline else None

    cfg = workload_config(args.workload, rb)
    cfg.update({"l2": "flushed between timed steps (256 MB write)", "launch": batch_cfg,
                "rollouts_per_step_per_gpu": rollouts_per_step, "competitor_steps_per_step_per_gpu": units_per_step,
                "parallelism": f"races x{world} (weak)"})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "win_prob_vectors_per_s": rb.n_races * world * args.steps / t_max,
            "rollout_kernel_ms": 1e3 * roll_s, "wall_s": wall,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches_per_step * args.steps, "surrogate": sur, "places": places,
            "population": population, "uneven": uneven, "single": single, "sweep": sweep, "cpu_oracle": oracle_t}
    # the numbers the results table quotes, last on the line (a reader of its tail sees them)
    line["summary"] = make_summary(line)
    line["surrogate_summary"] = surrogate_summary(sur)
    if rank == 0:
        print(json.dumps(line), flush=True)



def make_summary(line: dict) -> dict:
    r = lambda x, k=4: None if x is None else float(f"{x:.{k}g}")
    out = {"uniform": {"value": r(line["value"]), "alu_frac": r(line["roofline"]["frac"], 3),
                       "e2e": r((line.get("e2e") or {}).get("value")),
                       "oracle_all_cores": r((line.get("cpu_baseline") or {}).get("value"))}}
    u, si, sw, co = line.get("uneven"), line.get("single"), line.get("sweep"), line.get("cpu_oracle")
    if u:
        out["uneven"] = {"default": r(u["default"]["value"]), "autotuned": r(u["autotuned"]["value"]),
                         "gain": r(u["gain_autotuned_vs_default"], 3), "alu_frac": r(u["autotuned"]["alu_frac"], 3),
                         "vectors_per_s": r(u["autotuned"]["win_prob_vectors_per_s"]), "e2e": r(u["e2e"]["value"])}
    if si:
        out["single"] = {"device_ms": r(si["device_ms_per_pass_median"], 3), "e2e_ms": r(si["e2e_ms_per_call_median"], 3)}
    if sw:
        rows = sw["rows"]
        out["sweep"] = {"cov_max": r(max(x["cov"] for x in rows), 3),
                        "rate_n": {str(x["n"]): r(x["competitor_steps_per_s"], 3) for x in rows if x["n"] in (2, 5, 10, 20, 24, 32)}}
    if co:
        out["oracle"] = {k: r(v["value"], 3) for k, v in co.items() if isinstance(v, dict)}
    pop = (line.get("population") or {}).get("one_snapshot")
    if pop:
        out["one_snapshot_bettors"] = {"bettors": pop["bettors"], "dry_runs": pop["dry_runs"],
                                       "device_ms": r(pop["device_ms_median"], 3), "e2e_ms": r(pop["e2e_ms_median"], 3)}
    return out


def surrogate_summary(sur):
    if not sur:
        return None
    r = lambda x, k=4: None if x is None else float(f"{x:.{k}g}")
    h = sur.get("heldout", {})
    err = lambda d: {"max_abs": r(d.get("max_abs"), 3), "kl_mean": r(d.get("kl_mean"), 3)}
    ref6 = sur.get("reference_1e6", {})
    five = sur.get("five_input", {})
    return {"train": {"states_per_s": r(sur.get("train_states_per_s")), "tflops": r(sur.get("train_tflops"), 3),
                      "loss_last": r(sur.get("loss_last"), 3), "loss_curve_tenths": sur.get("loss_curve_tenths"),
                      "epochs": sur.get("epochs"), "states": sur.get("train_states")},
            "gate": sur.get("gate", {}).get("chosen_14"),
            "network": dict(err(h.get("network", {})), vectors_per_s=r(sur.get("infer", {}).get("win_prob_vectors_per_s"))),
            "gated": dict(err(h.get("gated", {})), gated=h.get("gated", {}).get("gated"),
                          vectors_per_s=r(sur.get("infer_gated", {}).get("win_prob_vectors_per_s"))),
            "gated_two_stage": dict(err(h.get("gated_two_stage", {})),
                                    vectors_per_s=r(sur.get("infer_gated_two_stage", {}).get("win_prob_vectors_per_s")),
                                    fallback_phase_s={k: r(v, 3) for k, v in sur.get("infer_gated_two_stage", {})
                                                      .get("fallback_phase_s", {}).items()}),
            "mc_at_query_rollouts": dict(err(h.get("mc_at_query_rollouts", {})),
                                         vectors_per_s=r(sur.get("mc_at_query_rollouts", {}).get("win_prob_vectors_per_s"))),
            "gain_gated_two_stage_vs_mc": r(sur.get("gain_gated_two_stage_vs_mc_at_query_rollouts"), 3),
            "with_3pct_out_of_range": {k: (r(v) if isinstance(v, float) else v) for k, v in
                                       sur.get("infer_with_out_of_range", {}).items()
                                       if k in ("out_of_range", "planted_out_of_range", "win_prob_vectors_per_s")},
            "vs_1e6_rollouts": {k: r(v.get("max_abs"), 3) for k, v in ref6.items() if isinstance(v, dict)},
            "five_input": {"network": err(five.get("network", {})), "answered": err(five.get("answered", {})),
                           "gate": five.get("gate"), "gated_share": r(five.get("gated_share"), 3)}}


def main():
    args = parse()
    if args.surrogate_kernels:
        print(json.dumps(run_surrogate_kernels(args.surrogate_kernels, args.races)))
        return
    if args.place_kernels:
        print(json.dumps(run_place_kernels(args)))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as D

        backend = "nccl" if args.impl == "gb300" else "gloo"
        if backend == "nccl":
            import torch

            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        D.init_process_group(backend)
        dist = D
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_gpu(args, rank, world, dist)
    finally:
        if dist:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
