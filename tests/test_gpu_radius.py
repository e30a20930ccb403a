"""The Box-Muller radius sqrt(-2 log u1) of the CUDA generator, for every u1 it can produce
(u1 = (m + 1) 2^-24, m = 0 .. 2^24 - 1): its square root (a Markstein sequence on the hardware
reciprocal-square-root estimate) must be the correctly rounded one, i.e. equal bit for bit to
the IEEE square root on the GPU and to the CPU oracle's radius (the oracle's own log, then a
binary32 multiply by -2 and the IEEE square root)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
N = 1 << 24


@pytest.fixture(scope="module")
def radii(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    so = str(tmp_path_factory.mktemp("radius") / "libbm_radius.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "--fmad=false",
                    "-shared", "-Xcompiler", "-fPIC", os.path.join(HERE, "native", "bm_radius.cu"), "-o", so],
                   check=True)
    lib = ctypes.CDLL(so)
    lib.bm_radii.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.bm_radii.restype = ctypes.c_int
    ours = np.empty(N, np.float32)
    ieee = np.empty(N, np.float32)
    assert lib.bm_radii(ours.ctypes.data, ieee.ctypes.data) == 0
    return ours, ieee


def test_radius_equals_the_ieee_square_root_for_every_input(radii):
    ours, ieee = radii
    bad = np.flatnonzero(ours.view(np.uint32) != ieee.view(np.uint32))
    assert bad.size == 0, (bad[:10], ours[bad[:10]], ieee[bad[:10]])


def test_radius_equals_the_oracle_for_every_input(radii):
    ours, _ = radii
    u1 = ((np.arange(N, dtype=np.float64) + 1.0) * 2.0 ** -24).astype(np.float32)  # exact
    m2l = np.float32(-2.0) * oracle.log_f32(u1)
    want = np.sqrt(m2l)  # binary32, correctly rounded
    bad = np.flatnonzero(ours.view(np.uint32) != want.view(np.uint32))
    assert bad.size == 0, (bad[:10], ours[bad[:10]], want[bad[:10]])
    assert np.signbit(ours[N - 1]) and ours[N - 1] == 0.0  # u1 = 1: sqrt(-0) = -0
