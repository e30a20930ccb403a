"""The oracle's Philox4x32-10 against NVIDIA's (cuRAND's curand_Philox4x32_10, run on the GPU)
on 65,536 random (counter, key) pairs and on the counters the method uses (k, t >> 2, c, r):
a second, independent implementation besides the published known-answer vectors."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    so = str(tmp_path_factory.mktemp("curand") / "libcurand_philox.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    os.path.join(HERE, "native", "curand_philox.cu"), "-o", so], check=True)
    lib = ctypes.CDLL(so)
    lib.curand_philox_blocks.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int]
    lib.curand_philox_blocks.restype = ctypes.c_int
    return lib


def nvidia_philox(lib, ctr, key):
    ctr = np.ascontiguousarray(ctr, np.uint32)
    key = np.ascontiguousarray(key, np.uint32)
    out = np.zeros_like(ctr)
    assert lib.curand_philox_blocks(ctr.ctypes.data, key.ctypes.data, out.ctypes.data, ctr.shape[0]) == 0
    return out


def test_random_counters_and_keys(curand_lib):
    rng = np.random.default_rng(2108)
    ctr = rng.integers(0, 2**32, (65536, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, (65536, 2), dtype=np.uint64).astype(np.uint32)
    got = nvidia_philox(curand_lib, ctr, key)
    idx = rng.choice(65536, 4096, replace=False)
    for i in idx:
        assert np.array_equal(oracle.philox4x32_10(ctr[i], key[i]), got[i]), i


def test_method_counters(curand_lib):
    # counter (k, t >> 2, c, r), key (seed lo, seed hi), around word boundaries
    seed = 0x0123456789ABCDEF
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    ks = [0, 1, 9999, 2**31 - 2]
    rows = [(k, tb, c, r) for k in ks for tb in (0, 1, 250) for c in (0, 19, 31) for r in (0, 4095, 2**31 - 1)]
    ctr = np.array(rows, np.uint32)
    got = nvidia_philox(curand_lib, ctr, np.tile(key, (len(rows), 1)))
    for i, row in enumerate(rows):
        assert np.array_equal(oracle.philox4x32_10(row, key), got[i]), row
