"""The benchmark's reference arm (the CPU oracle timed on the host cores) prints one JSON line
with the contract's keys, alone and under torchrun with two ranks (rank 0 prints, rank 1 exits
without work).  CPU only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def check(line, gpus):
    assert KEYS <= set(line), KEYS - set(line)
    assert line["impl"] == "reference" and line["n_gpus"] == gpus and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_reference_arm_single_process():
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "single", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = json_lines(res.stdout)
    assert len(lines) == 1
    check(lines[0], 1)


def test_reference_arm_under_torchrun_two_ranks():
    pytest.importorskip("torch")
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    res = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
                          "--gpus", "2", "--workload", "single", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-3000:]
    lines = json_lines(res.stdout)
    assert len(lines) == 1
    check(lines[0], 2)
