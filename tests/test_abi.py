"""CPU checks of the C-ABI boundary: the library loads, exports every entry
point include/mhc.h declares, and rejects bad arguments without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2102_03691_gb300 import mhc

HEADER = os.path.join(os.path.dirname(__file__), "..", "include", "mhc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mhc_[a-z_]+)\s*\(", src)))


def test_header_lists_match_binding():
    assert declared_functions() == sorted(mhc.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = mhc.load()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_default_params_and_status_strings():
    L = mhc.load()
    p = mhc.MhcParams()
    L.mhc_default_params(ctypes.byref(p))
    assert p.k_max == 256 and p.precision == 1 and p.ortho_probe == -1
    assert abs(p.F_e[0] - 1e-5) < 1e-20 and p.dt_ps == 0.01 and p.T_K == 300.0
    assert L.mhc_status_string(0) == b"ok"
    assert L.mhc_status_string(100) == b"basis not orthonormal"


@pytest.mark.parametrize("field,value", [("k_max", 0), ("k_max", 5000), ("n_lags", -1),
                                         ("precision", 7), ("tile_config", 9), ("dt_ps", 0.0)])
def test_create_rejects_bad_params(field, value):
    L = mhc.load()
    p = mhc.MhcParams()
    L.mhc_default_params(ctypes.byref(p))
    setattr(p, field, value)
    h = ctypes.c_void_p()
    assert L.mhc_create(ctypes.byref(h), ctypes.byref(p)) == 1
    assert h.value is None
    assert len(L.mhc_last_error(None)) > 0


def test_gkma_requires_lags():
    L = mhc.load()
    p = mhc.MhcParams()
    L.mhc_default_params(ctypes.byref(p))
    p.flags = mhc.FLAG_GKMA
    p.n_lags = 0
    h = ctypes.c_void_p()
    assert L.mhc_create(ctypes.byref(h), ctypes.byref(p)) == 1


def test_null_handle_calls_are_rejected():
    L = mhc.load()
    assert L.mhc_push(None, None, None, 1, 0) == 1
    assert L.mhc_sync(None) == 1
    assert L.mhc_reset(None) == 1
    L.mhc_destroy(None)   # no-op


def test_structs_match_header_sizes():
    # mhc_params: 6 int32 + pointer (8, aligned) + 2 int32 + 6 doubles
    assert ctypes.sizeof(mhc.MhcParams) == 4 + 4 + 8 + 4 * 6 + 8 * 6
    assert ctypes.sizeof(mhc.MhcInfo) % 8 == 0
