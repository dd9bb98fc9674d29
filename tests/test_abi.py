"""CPU checks of the C ABI: the library loads, exports every function declared in
include/jtfs.h, and rejects bad configurations on the host (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2204_08269_gb300 import build, jtfs
    build.build()
    return jtfs.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "jtfs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(jtfs_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    from paper_2204_08269_gb300 import jtfs
    declared = _declared()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(L, name), name
    assert sorted(jtfs.exported_symbols()) == sorted(
        n for n in declared if n in jtfs.exported_symbols())
    assert set(declared) <= set(jtfs.exported_symbols())


def test_status_strings(L):
    for s in range(7):
        assert L.jtfs_status_string(s)


@pytest.mark.parametrize("field,value", [("J", 0), ("Q", 0), ("T", 3), ("F", 0),
                                         ("average_fr", 2), ("oversampling", -1),
                                         ("precision", 9), ("out_3d", 2), ("branches", 1),
                                         ("branches", 2), ("branches", 16 | 3)])
def test_invalid_config_rejected_on_host(L, field, value):
    from paper_2204_08269_gb300 import jtfs
    cfg = jtfs._Config(J=6, Q=8, Q2=1, J_fr=3, Q_fr=1, T=64, F=8, average_fr=1, out_3d=1)
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    st = L.jtfs_plan_create(ctypes.byref(cfg), 4096, ctypes.byref(h))
    assert st == 1  # JTFS_ERR_INVALID_ARG, before any CUDA call
    assert h.value is None
    assert L.jtfs_last_error()


def test_invalid_length_rejected(L):
    from paper_2204_08269_gb300 import jtfs
    cfg = jtfs._Config(J=6, Q=8, Q2=1, J_fr=3, Q_fr=1, T=64, F=8, average_fr=1)
    h = ctypes.c_void_p()
    assert L.jtfs_plan_create(ctypes.byref(cfg), 3000, ctypes.byref(h)) == 1
    assert L.jtfs_plan_create(ctypes.byref(cfg), 4096, None) == 1


def test_null_plan_calls(L):
    n = ctypes.c_size_t()
    assert L.jtfs_workspace_bytes(None, 1, 0, ctypes.byref(n)) == 1
    assert L.jtfs_forward(None, None, 1, None, None, None, None, None, 0, None) == 1
    assert L.jtfs_backward(None, None, None, 1, None, None, None, None, None, 0, None) == 1


def test_varlen_padded_length_rule():
    """max(2^ceil(log2 len), 2^(J+3)), computed on the host without a GPU."""
    from paper_2204_08269_gb300 import jtfs
    for J in (4, 6, 12):
        for n in (1, 2, 3, 100, 511, 512, 513, 4096, 70000):
            want = max(1 << int(np.ceil(np.log2(n))) if n > 1 else 1, 1 << (J + 3))
            assert jtfs.varlen_padded_length(n, J=J) == want
    assert jtfs.varlen_padded_length(0, J=4) == 0


def test_failure_detection_calls_reject_bad_arguments_on_host(L):
    """NULL plans are refused before any CUDA call."""
    assert L.jtfs_plan_set_wait_budget(None, 1_000_000) == 1
    assert L.jtfs_plan_set_check_finite(None, 1) == 1
    assert L.jtfs_diagnose_wait_timeout(None, 100_000, None) == 1
    assert L.jtfs_sync_status(None, None) == 1
