"""The C-ABI library loads without a GPU and exports every entry point include/*.h declares;
the Python binding has a function of the same name for each."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        text = open(h).read()
        names += re.findall(r"^BBE_API\s+[\w\s\*]+?\b(bbe_\w+)\s*\(", text, flags=re.M)
    return names


@pytest.fixture(scope="module")
def built_lib():
    from paper_2108_02419_gb300 import build

    return build.build()


def test_headers_declare_entry_points():
    names = declared_symbols()
    for required in ("bbe_race_init", "bbe_rollout_batch", "bbe_win_probs", "bbe_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_has_same_names(built_lib):
    from paper_2108_02419_gb300 import bbe

    missing = [n for n in declared_symbols() if not callable(getattr(bbe, n, None))]
    assert not missing, missing


def test_binding_refuses_without_library(tmp_path, monkeypatch):
    from paper_2108_02419_gb300 import bbe

    monkeypatch.setattr(bbe, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(bbe, "_lib", None)
    with pytest.raises(ImportError):
        bbe.lib()


def test_checked_build_compiles_and_exports_every_declared_symbol():
    # the checked build (every device index of the rollout kernels tested) compiles here without
    # a GPU and offers the same entry points; its GPU run is tests/test_gpu_checked_build.py
    from paper_2108_02419_gb300 import build

    so = build.build(checked=True)
    assert os.path.dirname(so).endswith(os.path.join("_lib", "checked"))
    lib = ctypes.CDLL(so)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
