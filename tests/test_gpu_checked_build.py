"""The checked build of the library (build.build(checked=True): every computed device index of
the rollout kernels tested, a failure recorded in the batch status as BBE_ERR_RANGE instead of an
access out of range; the stand-in for a memory checker).  The rollout paths run on it in a
child process (the binding loads the library named by BBE_LIB) and must report no failed check
and equal the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_rollout_paths_pass_every_index_check():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_02419_gb300 import build

    so = build.build(checked=True)
    env = dict(os.environ, BBE_LIB=so)
    res = subprocess.run([sys.executable, os.path.join(HERE, "checked_build_run.py")], env=env, capture_output=True,
                         text=True, timeout=900)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    assert "checked build ok" in res.stdout
