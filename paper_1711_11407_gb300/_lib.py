"""ctypes binding of the FPS-SFT C ABI (include/fpssft.h).

Argument marshalling only: every step of the recovery runs in the CUDA library.  The library is
built in-tree (``build()``); if it is missing or fails to load, every call raises -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
LIB_PATH = os.path.join(_HERE, "libfpssft.so")
SOURCES = [os.path.join(_HERE, "csrc", "fpssft.cu")]
DEPENDS = SOURCES + [os.path.join(_HERE, "csrc", f) for f in ("fpssft_device.cuh", "recover_common.cuh",
                                                                "recover_shared.cuh", "recover_warp.cuh",
                                                                "recover_cluster.cuh", "aux_kernels.cuh", "refine.cuh",
                                                                "phase_timers.cuh")] + \
    [os.path.join(_ROOT, "include", "fpssft.h")]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "--expt-relaxed-constexpr", "-shared", "-Xcompiler", "-fPIC"]

OK, ERR_INVALID, ERR_CUDA, ERR_ALLOC, ERR_CAPACITY, ERR_TIMEOUT, ERR_UNSUPPORTED = range(7)
ADJ_PROJECT, ADJ_SYNTH = 0, 1

_lock = threading.Lock()
_lib = None
_variant = None   # path of a build variant loaded instead of LIB_PATH (see use_library)


class FpssftError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"fpssft status {status}: {msg}")
        self.status = status


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def needs_build(path=LIB_PATH):
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    return any(os.path.getmtime(p) > t for p in DEPENDS)


def build(force=False, verbose=False, out=LIB_PATH, defines=()):
    """Compile the library for sm_103a next to this file (atomic rename).  `out` and `defines`
    (preprocessor macros, e.g. FPSSFT_PHASE_TIMERS) build a variant under another name."""
    if not force and not needs_build(out):
        return out
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = [_nvcc(), *NVCC_FLAGS, *(f"-D{d}" for d in defines), "-I", os.path.join(_ROOT, "include"), "-o", tmp,
           *SOURCES]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose:
            print(r.stdout + r.stderr)
        os.replace(tmp, out)
    finally:
        if os.path.exists(tmp):
            os.unlink(tmp)
    return out


class PlanInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("D", "batch", "L_max", "T_max", "k_cap", "hash_cap", "n_shapes",
                                            "threads", "grid", "smem_bytes", "twiddles_in_smem", "prefetch", "fft_path",
                                            "global_workspace")]


class CParams(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int), ("k_cap", ctypes.c_int), ("theta0", ctypes.c_float), ("rho", ctypes.c_float),
                ("eta", ctypes.c_float), ("early_stop", ctypes.c_int), ("peel_mode", ctypes.c_int),
                ("threads", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("fp64_decisions", ctypes.c_int), ("gather_mode", ctypes.c_int), ("fft_path", ctypes.c_int),
                ("amp_average", ctypes.c_int), ("radix_plan", ctypes.c_int),
                ("host_cubes", ctypes.c_int), ("cluster_set", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int

SIGNATURES = {
    "fpssft_plan_create": (_I, [ctypes.POINTER(_P), _I, _I, _P, ctypes.POINTER(CParams)]),
    "fpssft_plan": (_I, [ctypes.POINTER(_P), _I, _I, _P, ctypes.POINTER(CParams)]),
    "fpssft_plan_destroy": (None, [_P]),
    "fpssft_plan_get_info": (_I, [_P, ctypes.POINTER(PlanInfo)]),
    "fpssft_plan_get_lengths": (_I, [_P, _P, _P]),
    "fpssft_project": (_I, [_P, _P, _P, _P, _P, _I, _P, _P]),
    "fpssft_lines": (_I, [_P, _P, _P, _P, _P, _I, _P, _P]),
    "fpssft_recover": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "fpssft_recover_host": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "fpssft_synth": (_I, [_P, _P, _P, _I, _P, _P, _P, _I, _P, _P]),
    "fpssft_decode": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "fpssft_finalize": (_I, [_P, _P, _P, _P, _P]),
    "fpssft_adjoint": (_I, [_P, _I, _P, _P, _P, _P, _I, _P, _P, _P, _P]),
    "fpssft_refine_workspace_size": (_I, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "fpssft_refine": (_I, [_P, _P, _P, _P, _I, _P, _P, _P, _I, ctypes.c_float, _P, ctypes.c_size_t, _P, _P]),
    "fpssft_probe_gather": (_I, [_P, ctypes.c_int64, _I, _I, _I, _I, _P, _P]),
    "fpssft_l2_fetch_granularity": (_I, [_I, ctypes.POINTER(ctypes.c_int)]),
    "fpssft_phase_read": (_I, [_P]),
    "fpssft_recover_noalloc": (_I, [_I, _I, _P, ctypes.POINTER(CParams), _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "fpssft_fft_stages": (_I, [_I, _I, _P, _P]),
    "fpssft_last_error": (ctypes.c_char_p, []),
    "fpssft_version": (ctypes.c_char_p, []),
}


def use_library(path):
    """Load `path`, an in-tree build variant of the same sources (the phase-timer build), in place of
    libfpssft.so.  Only before the first load() of the process."""
    global _variant
    with _lock:
        if _lib is not None:
            raise RuntimeError("the CUDA library is already loaded in this process")
        _variant = path


def load(auto_build=True):
    """Load (building first when needed) and return the ctypes library handle."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _variant or LIB_PATH
        if _variant is None and auto_build and needs_build():
            build()
        if not os.path.exists(path):
            raise FpssftError(ERR_UNSUPPORTED, f"CUDA library not built: {path} (run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(status):
    if status != OK:
        msg = load().fpssft_last_error().decode(errors="replace")
        raise FpssftError(status, msg)
