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
    return sorted(set(re.findall(r"\b(mhc_[a-z0-9_]+)\s*\(", src)))


def test_header_lists_match_binding():
    assert declared_functions() == sorted(mhc.EXPORTS)


def header_constants():
    """Every `MHC_X = v` enumerator and `#define MHC_X v` integer of the header."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    vals = {n: int(v, 0) for n, v in re.findall(r"\b(MHC_[A-Z0-9_]+)\s*=\s*(-?(?:0x)?[0-9a-fA-F]+)\b", src)}
    vals.update({n: int(v, 0) for n, v in re.findall(r"#define\s+(MHC_[A-Z0-9_]+)\s+(0x[0-9a-fA-F]+|\d+)\s*$",
                                                      src, flags=re.M)})
    return vals


def test_binding_constants_match_header():
    c = header_constants()
    pairs = {"MHC_MEM_HOST": mhc.MEM_HOST, "MHC_MEM_DEVICE": mhc.MEM_DEVICE,
             "MHC_MEM_HOST_ASYNC": mhc.MEM_HOST_ASYNC, "MHC_F32": mhc.F32, "MHC_F64": mhc.F64,
             "MHC_DOF_MAJOR": mhc.DOF_MAJOR, "MHC_MODE_MAJOR": mhc.MODE_MAJOR,
             "MHC_FLAG_GKMA": mhc.FLAG_GKMA, "MHC_FLAG_NO_GRAPH": mhc.FLAG_NO_GRAPH,
             "MHC_FLAG_PROFILE": mhc.FLAG_PROFILE, "MHC_FLAG_TEST_STALL": mhc.FLAG_TEST_STALL,
             "MHC_FLAG_DIRECTION": mhc.FLAG_DIRECTION, "MHC_FLAG_XCORR": mhc.FLAG_XCORR,
             "MHC_OK": mhc.MHC_OK, "MHC_WARN_NOT_ORTHONORMAL": mhc.MHC_WARN_NOT_ORTHONORMAL,
             "MHC_PREC_FP32": mhc.PRECISIONS["fp32"], "MHC_PREC_BF16X3": mhc.PRECISIONS["bf16x3"],
             "MHC_PREC_FP16X3": mhc.PRECISIONS["fp16x3"]}
    missing = [n for n in pairs if n not in c]
    assert not missing, missing
    assert {n: c[n] for n in pairs} == pairs


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
                                         ("precision", 7), ("tile_config", 9), ("dt_ps", 0.0),
                                         ("split_d", -2), ("split_d", 17)])
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


@pytest.mark.parametrize("split_d", [2, -1])
def test_direction_split_takes_no_d_axis_split(split_d):
    L = mhc.load()
    p = mhc.MhcParams()
    L.mhc_default_params(ctypes.byref(p))
    p.flags = mhc.FLAG_DIRECTION
    p.split_d = split_d          # a uniform or the balanced split
    h = ctypes.c_void_p()
    assert L.mhc_create(ctypes.byref(h), ctypes.byref(p)) == 1
    assert b"split" in L.mhc_last_error(None)


def test_null_handle_calls_are_rejected():
    L = mhc.load()
    assert L.mhc_push(None, None, None, 1, 0) == 1
    assert L.mhc_sync(None) == 1
    assert L.mhc_reset(None) == 1
    best = ctypes.c_int32()
    assert L.mhc_autotune_k(None, None, 0, ctypes.byref(best), None) == 1
    L.mhc_destroy(None)   # no-op


def test_structs_match_header_sizes():
    # mhc_params: int32 + pointer (8, aligned) + 6 int32 + 6 doubles + int32 (padded to 8)
    assert ctypes.sizeof(mhc.MhcParams) == 4 + 4 + 8 + 4 * 6 + 8 * 6 + 8
    assert ctypes.sizeof(mhc.MhcInfo) % 8 == 0


def test_struct_layouts_match_the_c_compiler(tmp_path):
    # the binding's ctypes structures against what a C compiler makes of include/mhc.h
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    fields_p = [f for f, _ in mhc.MhcParams._fields_]
    fields_i = [f for f, _ in mhc.MhcInfo._fields_]
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "mhc.h"', "int main(void) {",
           'printf("%zu %zu\\n", sizeof(mhc_params), sizeof(mhc_info));']
    src += [f'printf("%zu\\n", offsetof(mhc_params, {f}));' for f in fields_p]
    src += [f'printf("%zu\\n", offsetof(mhc_info, {f}));' for f in fields_i]
    src += ["return 0; }"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(c), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    vals = [int(x) for x in out]
    assert vals[0] == ctypes.sizeof(mhc.MhcParams) and vals[1] == ctypes.sizeof(mhc.MhcInfo)
    offs = vals[2:]
    want = [getattr(mhc.MhcParams, f).offset for f in fields_p] + \
        [getattr(mhc.MhcInfo, f).offset for f in fields_i]
    assert offs == want
