"""The C ABI library: builds for sm_103a, loads, exports every declared symbol, and rejects bad
arguments on the host before touching a device (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1711_11407_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fpssft.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fpssft_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    lib = _lib.load()
    names = declared_functions()
    assert len(names) >= 14
    raw = ctypes.CDLL(_lib.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), f"{n} declared in include/fpssft.h but not exported"
    assert set(names) == set(_lib.SIGNATURES), "binding signatures must cover exactly the declared functions"
    assert lib.fpssft_version().startswith(b"fpssft")


def _plan(D, batch, dims, **kw):
    lib = _lib.load()
    p = _lib.CParams(kw.get("T", 10), kw.get("k_cap", 64), kw.get("theta0", 1e-3), 1e-3, 0.05, 1,
                     kw.get("peel_mode", 0), kw.get("threads", 0), 0, 0, kw.get("gather_mode", 0), kw.get("fft_path", 0), 0,
                     kw.get("radix_plan", 0), kw.get("host_cubes", 0), kw.get("cluster_set", 0))
    h = ctypes.c_void_p()
    d = np.ascontiguousarray(np.asarray(dims, np.int64).reshape(-1))
    st = lib.fpssft_plan_create(ctypes.byref(h), D, batch, d.ctypes.data_as(ctypes.c_void_p) if d.size else None,
                                ctypes.byref(p))
    return st, lib.fpssft_last_error().decode()


@pytest.mark.parametrize("D,batch,dims,kw,expect", [
    (0, 1, [4], {}, _lib.ERR_INVALID),
    (5, 1, [2, 2, 2, 2, 2], {}, _lib.ERR_INVALID),
    (2, -1, [], {}, _lib.ERR_INVALID),
    (2, 1, [0, 4], {}, _lib.ERR_INVALID),
    (2, 1, [8, 8], {"k_cap": 0}, _lib.ERR_INVALID),
    (2, 1, [8, 8], {"T": -1}, _lib.ERR_INVALID),
    (2, 1, [8, 8], {"theta0": -1.0}, _lib.ERR_INVALID),
    (2, 1, [8, 8], {"threads": 48}, _lib.ERR_INVALID),
    (2, 1, [8, 8], {"threads": 2048}, _lib.ERR_INVALID),
    (2, 1, [8, 8], {"peel_mode": 1}, _lib.ERR_UNSUPPORTED),
    (2, 1, [8, 8], {"gather_mode": 6}, _lib.ERR_INVALID),
    (2, 1, [8, 8], {"fft_path": 4}, _lib.ERR_INVALID),
    (2, 1, [8, 8], {"radix_plan": -1}, _lib.ERR_INVALID),
    (2, 1, [8, 8], {"radix_plan": 4}, _lib.ERR_INVALID),
    (2, 1, [8, 8], {"host_cubes": 2}, _lib.ERR_INVALID),
    (2, 1, [8, 8], {"cluster_set": 3}, _lib.ERR_INVALID),
    (2, 1, [8, 8], {"cluster_set": -1}, _lib.ERR_INVALID),
    (2, 1, [1 << 20, 3], {}, _lib.ERR_UNSUPPORTED),         # D L max N_d >= 2^31
    (2, 1, [65536, 65536], {}, _lib.ERR_UNSUPPORTED),       # N >= 2^31
])
def test_plan_validation_on_host(D, batch, dims, kw, expect):
    st, msg = _plan(D, batch, dims, **kw)
    assert st == expect, msg
    assert msg, "a failing call leaves a message"


def test_null_plan_rejected():
    lib = _lib.load()
    assert lib.fpssft_recover(None, *([None] * 11)) == _lib.ERR_INVALID
    assert lib.fpssft_project(None, None, None, None, None, 1, None, None) == _lib.ERR_INVALID
    assert lib.fpssft_adjoint(None, 0, None, None, None, None, 1, None, None, None, None) == _lib.ERR_INVALID
    assert b"null plan" in lib.fpssft_last_error()


def test_phase_read_is_unsupported_in_the_default_build():
    lib = _lib.load()
    buf = (ctypes.c_int64 * 11)()
    assert lib.fpssft_phase_read(buf) == _lib.ERR_UNSUPPORTED
    assert b"FPSSFT_PHASE_TIMERS" in lib.fpssft_last_error()


def test_every_call_rejects_a_null_plan_or_pointer_on_the_host():
    """The error contract without a device: a null plan (or null params / buffer) is
    FPSSFT_ERR_INVALID with a message, before any CUDA call; destroying a null plan is a no-op."""
    lib = _lib.load()
    Z = None
    cases = {
        "fpssft_plan_get_info": (Z, Z),
        "fpssft_plan_get_lengths": (Z, Z, Z),
        "fpssft_project": (Z, Z, Z, Z, Z, 1, Z, Z),
        "fpssft_lines": (Z, Z, Z, Z, Z, 1, Z, Z),
        "fpssft_recover": (Z,) * 12,
        "fpssft_recover_host": (Z,) * 12,
        "fpssft_synth": (Z, Z, Z, 1, Z, Z, Z, 0, Z, Z),
        "fpssft_decode": (Z,) * 11,
        "fpssft_finalize": (Z,) * 5,
        "fpssft_adjoint": (Z, 0, Z, Z, Z, Z, 1, Z, Z, Z, Z),
        "fpssft_probe_gather": (Z, 1024, 1, 256, 0, 0, Z, Z),
        "fpssft_recover_noalloc": (2, 1, Z, Z) + (Z,) * 11,
        "fpssft_refine": (Z, Z, Z, Z, 1, Z, Z, Z, 1, 1e-7, Z, 0, Z, Z),
        "fpssft_refine_workspace_size": (Z, Z),
    }
    for name, args in cases.items():
        assert getattr(lib, name)(*args) == _lib.ERR_INVALID, name
        assert lib.fpssft_last_error() != b"", name
    lib.fpssft_plan_destroy(None)


def test_a_missing_library_fails_loudly_instead_of_falling_back(tmp_path):
    """No CPU fallback: with the CUDA library absent, loading it (the first step of every call)
    raises FpssftError in a fresh process."""
    import subprocess
    import sys
    code = ("from paper_1711_11407_gb300 import _lib\n"
            f"_lib.use_library({str(tmp_path / 'missing.so')!r})\n"
            "try:\n"
            "    _lib.load()\n"
            "except _lib.FpssftError as e:\n"
            "    print('raised', e.status)\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == f"raised {_lib.ERR_UNSUPPORTED}"


@pytest.mark.parametrize("plan", [0, 1, 2, 3])
def test_fft_stage_sequences_multiply_to_L_in_the_plan_order(plan):
    """fpssft_fft_stages (host only): every radix plan is a factorisation of L; plan 1 has no
    radix 8, plan 2 puts the odd factors first, plan 3 has no radix 2 unless L's power of two is 2,
    plan 0 has at most one radix-4 or radix-2 stage."""
    lib = _lib.load()
    out = (ctypes.c_int32 * 24)()
    n = ctypes.c_int32(0)
    for L in [1, 2, 3, 4, 7, 12, 64, 96, 128, 240, 256, 360, 512, 576, 1024, 2048, 3840, 4608, 7919, 2 * 7919,
              (1 << 23) * 2]:
        if L > (1 << 24):
            assert lib.fpssft_fft_stages(L, plan, out, ctypes.byref(n)) == _lib.ERR_INVALID
            continue
        assert lib.fpssft_fft_stages(L, plan, out, ctypes.byref(n)) == _lib.OK
        r = [out[i] for i in range(n.value)]
        assert int(np.prod(r, dtype=np.int64)) == L, (L, plan, r)
        e = (L & -L).bit_length() - 1
        twos = [v for v in r if v in (2, 4, 8)]
        odd = [v for v in r if v not in (2, 4, 8)]
        assert odd == sorted(odd)
        if plan == 1:
            assert 8 not in r
        if plan == 2:
            assert r == odd + twos
        else:
            assert r == twos + odd
        if plan == 3 and e >= 2:
            assert 2 not in r
        if plan == 0:
            assert sum(v in (2, 4) for v in r) <= 1
    assert lib.fpssft_fft_stages(64, 5, out, ctypes.byref(n)) == _lib.ERR_INVALID


def _header_fields(struct_name):
    """(type, name) of every member of `typedef struct { ... } struct_name;` in include/fpssft.h."""
    text = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fpssft.h")).read()
    end = text.index("} " + struct_name + ";")
    start = text.rindex("typedef struct {", 0, end)
    body = re.sub(r"/\*.*?\*/", "", text[start:end], flags=re.S)
    return re.findall(r"^\s*(int|float)\s+(\w+)\s*;", body, flags=re.M)


@pytest.mark.parametrize("struct_name,cls", [("fpssft_params", "CParams"), ("fpssft_plan_info", "PlanInfo")])
def test_ctypes_structs_match_the_header(struct_name, cls, tmp_path):
    """The binding's ctypes structs declare the header's members in the header's order and types,
    and a C compiler lays the header's struct out at the same offsets and size."""
    import shutil
    import subprocess
    klass = getattr(_lib, cls)
    fields = _header_fields(struct_name)
    ctype = {"int": ctypes.c_int, "float": ctypes.c_float}
    assert [(n, ctype[t]) for t, n in fields] == [(n, t) for n, t in klass._fields_]
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "fpssft.h"\nint main(void) {\n'
                   + f'  printf("%zu\\n", sizeof({struct_name}));\n'
                   + "".join(f'  printf("%zu\\n", offsetof({struct_name}, {n}));\n' for _, n in fields)
                   + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True, capture_output=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got[0] == ctypes.sizeof(klass)
    assert got[1:] == [getattr(klass, n).offset for _, n in fields]


def test_binding_signatures_take_as_many_arguments_as_the_header_prototypes():
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "fpssft.h")).read(), flags=re.S)
    protos = dict(re.findall(r"\b(fpssft_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S))
    assert set(protos) == set(_lib.SIGNATURES)
    for name, params in protos.items():
        params = " ".join(params.split())
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert n == len(_lib.SIGNATURES[name][1]), f"{name}: header takes {n} arguments"
