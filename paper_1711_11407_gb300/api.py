"""PyTorch-facing wrapper of the FPS-SFT C ABI: device memory and streams come from torch, every
computation happens in the CUDA library (see include/fpssft.h for the exact semantics)."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib

__all__ = ["Params", "Plan", "RecoverOutput"]


@dataclass
class Params:
    """Recovery parameters (fpssft_params).  T = 0 selects the per-signal budget N / ((D+1) L)."""

    T: int = 10
    k_cap: int = 1024
    theta0: float = 1e-3
    rho: float = 1e-3
    eta: float = 0.05
    early_stop: int = 1          # 0 none, 1 stop when no line-0 bin passes T0, 2 also when all were decoded
    peel_mode: int = 0
    threads: int = 0
    ctas_per_sm: int = 0
    fp64_decisions: bool = False
    gather_mode: int = 0
    fft_path: int = 0
    amp_average: bool = False
    radix_plan: int = 0
    host_cubes: int = 0
    cluster_set: int = 0         # path 3: 0 library choice, 1 shared memory when it fits, 2 global workspace

    def c(self):
        return _lib.CParams(int(self.T), int(self.k_cap), float(self.theta0), float(self.rho), float(self.eta),
                            int(self.early_stop), int(self.peel_mode), int(self.threads), int(self.ctas_per_sm),
                            int(bool(self.fp64_decisions)), int(self.gather_mode), int(self.fft_path),
                            int(bool(self.amp_average)), int(self.radix_plan), int(self.host_cubes),
                            int(self.cluster_set))


@dataclass
class RecoverOutput:
    k: torch.Tensor        # int32 [batch][k_cap][D]
    a: torch.Tensor        # complex64 [batch][k_cap]
    count: torch.Tensor    # int32 [batch]
    iters: torch.Tensor    # int32 [batch]
    status: torch.Tensor   # int32 [batch]

    def signal(self, b):
        """(k [n][D] int64 numpy, a [n] complex128 numpy) of signal b (synchronises)."""
        n = int(self.count[b])
        return (self.k[b, :n].cpu().numpy().astype(np.int64), self.a[b, :n].cpu().numpy().astype(np.complex128))


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need(t, dtype, name, device=True):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if device and not t.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


class Plan:
    """A plan for a batch of cubes with shapes dims[b] (array-like int [batch][D])."""

    def __init__(self, dims, params: Params | None = None):
        self.lib = _lib.load()
        dims = np.ascontiguousarray(np.asarray(dims, dtype=np.int64))
        if dims.ndim != 2:
            raise ValueError("dims must be [batch][D]")
        self.dims = dims
        self.params = params or Params()
        self.batch, self.D = int(dims.shape[0]), int(dims.shape[1])
        h = ctypes.c_void_p()
        cp = self.params.c()
        _lib.check(self.lib.fpssft_plan_create(ctypes.byref(h), self.D, self.batch,
                                               dims.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cp)))
        self.handle = h
        info = _lib.PlanInfo()
        _lib.check(self.lib.fpssft_plan_get_info(self.handle, ctypes.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in _lib.PlanInfo._fields_}
        self.L_max, self.T_max, self.k_cap = info.L_max, info.T_max, info.k_cap
        Ls = np.zeros(max(1, self.batch), np.int32)
        Ts = np.zeros(max(1, self.batch), np.int32)
        _lib.check(self.lib.fpssft_plan_get_lengths(self.handle, Ls.ctypes.data_as(ctypes.c_void_p),
                                                    Ts.ctypes.data_as(ctypes.c_void_p)))
        self.L = Ls[: self.batch]
        self.T = Ts[: self.batch]
        self.N = np.prod(dims, axis=1).astype(np.int64) if self.batch else np.zeros(0, np.int64)
        self._validated = set()

    def close(self):
        if getattr(self, "handle", None):
            self.lib.fpssft_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- checks ----------------------------------------------------------------------------------
    def _sched(self, alpha, tau, rows=None):
        _need(alpha, torch.int32, "alpha")
        _need(tau, torch.int32, "tau")
        if alpha.shape != tau.shape or alpha.dim() != 3 or alpha.shape[0] != self.batch or alpha.shape[2] != self.D:
            raise ValueError(f"alpha/tau must be int32 [batch={self.batch}][n_sched][D={self.D}]")
        if rows is not None and alpha.shape[1] != rows:
            raise ValueError(f"schedule must have {rows} rows per signal")
        return alpha.shape[1]

    def _check_extent(self, cubes, offsets):
        """Every cube must lie inside `cubes`: offsets[b] >= 0 and offsets[b] + N_b <= cubes.numel().
        The kernels trust the offsets, so they are checked here (one device-to-host read) for every
        new (cubes, offsets) pair; during CUDA-graph capture the check is skipped -- capture a pair
        that has been used once outside capture."""
        key = (cubes.data_ptr(), cubes.numel(), offsets.data_ptr(), offsets.numel())
        if key in self._validated or self.batch == 0:
            return
        if torch.cuda.is_available() and torch.cuda.is_current_stream_capturing():
            return
        if offsets.numel() != self.batch:
            raise ValueError(f"offsets must have {self.batch} entries")
        off = offsets.detach().cpu().numpy()
        if np.any(off < 0) or np.any(off + self.N > cubes.numel()):
            raise ValueError("offsets place a cube outside the cubes buffer")
        if len(self._validated) > 256:
            self._validated.clear()
        self._validated.add(key)

    def _bins_shape(self, n_sched):
        return (self.batch, n_sched, self.D + 1, self.L_max)

    # ---- calls -----------------------------------------------------------------------------------
    def project(self, cubes, offsets, alpha, tau, out=None, stream=None, raw_lines=False):
        """Line DFTs (or raw line samples) [batch][n_sched][D+1][L_max] complex64."""
        _need(cubes, torch.complex64, "cubes")
        _need(offsets, torch.int64, "offsets")
        S = self._sched(alpha, tau)
        self._check_extent(cubes, offsets)
        if out is None:
            out = torch.empty(self._bins_shape(S), dtype=torch.complex64, device=cubes.device)
        _need(out, torch.complex64, "out")
        fn = self.lib.fpssft_lines if raw_lines else self.lib.fpssft_project
        _lib.check(fn(self.handle, _ptr(cubes), _ptr(offsets), _ptr(alpha), _ptr(tau), S, _ptr(out), _stream(stream)))
        return out

    def lines(self, cubes, offsets, alpha, tau, out=None, stream=None):
        return self.project(cubes, offsets, alpha, tau, out, stream, raw_lines=True)

    def alloc_output(self, device="cuda"):
        return RecoverOutput(torch.zeros((self.batch, self.k_cap, self.D), dtype=torch.int32, device=device),
                             torch.zeros((self.batch, self.k_cap), dtype=torch.complex64, device=device),
                             torch.zeros(self.batch, dtype=torch.int32, device=device),
                             torch.zeros(self.batch, dtype=torch.int32, device=device),
                             torch.zeros(self.batch, dtype=torch.int32, device=device))

    def recover(self, cubes, offsets, alpha, tau, out: RecoverOutput | None = None, init_count=None, stream=None):
        """The fused persistent recovery over the batch; schedule [batch][T_max][D]."""
        _need(cubes, torch.complex64, "cubes")
        _need(offsets, torch.int64, "offsets")
        self._sched(alpha, tau, rows=self.T_max)
        self._check_extent(cubes, offsets)
        if out is None:
            out = self.alloc_output(cubes.device)
        if init_count is not None:
            _need(init_count, torch.int32, "init_count")
        _lib.check(self.lib.fpssft_recover(self.handle, _ptr(cubes), _ptr(offsets), _ptr(alpha), _ptr(tau),
                                           _ptr(init_count), _ptr(out.k), _ptr(out.a), _ptr(out.count),
                                           _ptr(out.iters), _ptr(out.status), _stream(stream)))
        return out

    def recover_mapped(self, host_cubes, offsets, alpha, tau, out: RecoverOutput | None = None, init_count=None,
                       stream=None):
        """fpssft_recover with the cubes left in pinned host memory: the gather reads the samples it
        needs over the host link (no copy of the cubes); offsets, schedule and outputs are on the
        device.  host_cubes must be a contiguous pinned CPU complex64 tensor."""
        if not isinstance(host_cubes, torch.Tensor) or host_cubes.is_cuda or host_cubes.dtype != torch.complex64 \
                or not host_cubes.is_contiguous() or not host_cubes.is_pinned():
            raise ValueError("host_cubes must be a contiguous pinned CPU complex64 tensor")
        _need(offsets, torch.int64, "offsets")
        self._sched(alpha, tau, rows=self.T_max)
        self._check_extent(host_cubes, offsets)
        if out is None:
            out = self.alloc_output(offsets.device)
        _lib.check(self.lib.fpssft_recover(self.handle, _ptr(host_cubes), _ptr(offsets), _ptr(alpha), _ptr(tau),
                                           _ptr(init_count), _ptr(out.k), _ptr(out.a), _ptr(out.count),
                                           _ptr(out.iters), _ptr(out.status), _stream(stream)))
        return out

    def recover_host(self, cubes, offsets, alpha, tau, out=None, init_count=None, stream=None):
        """fpssft_recover_host on host arrays (numpy or pinned CPU tensors); returns host outputs."""
        def host(t, dtype):
            if isinstance(t, torch.Tensor):
                if t.is_cuda or t.dtype != dtype or not t.is_contiguous():
                    raise ValueError("host tensors must be contiguous CPU tensors of the right dtype")
                return t
            return torch.from_numpy(np.ascontiguousarray(t)).to(dtype)
        cubes = host(cubes, torch.complex64)
        offsets = host(offsets, torch.int64)
        self._check_extent(cubes, offsets)
        alpha = host(alpha, torch.int32)
        tau = host(tau, torch.int32)
        if out is None:
            out = self.alloc_output("cpu")
        _lib.check(self.lib.fpssft_recover_host(self.handle, _ptr(cubes), _ptr(offsets), _ptr(alpha), _ptr(tau),
                                                _ptr(init_count), _ptr(out.k), _ptr(out.a), _ptr(out.count),
                                                _ptr(out.iters), _ptr(out.status), _stream(stream)))
        return out

    def synth(self, alpha, tau, k, a, count, accumulate=0, bins=None, stream=None):
        """Bins of the sparse spectrum (k, a) on the schedule lines (accumulate: 0 set, +1 add, -1 subtract)."""
        S = self._sched(alpha, tau)
        self._check_set(k, a, count)
        if bins is None:
            bins = torch.empty(self._bins_shape(S), dtype=torch.complex64, device=a.device)
            accumulate = 0
        _need(bins, torch.complex64, "bins")
        _lib.check(self.lib.fpssft_synth(self.handle, _ptr(alpha), _ptr(tau), S, _ptr(k), _ptr(a), _ptr(count),
                                         int(accumulate), _ptr(bins), _stream(stream)))
        return bins

    def decode(self, bins, alpha, tau, k, a, count, t0_count, status, accepted=None, stream=None):
        self._sched(alpha, tau, rows=1)
        _need(bins, torch.complex64, "bins")
        self._check_set(k, a, count)
        _need(t0_count, torch.int32, "t0_count")
        _need(status, torch.int32, "status")
        if accepted is not None:
            _need(accepted, torch.int32, "accepted")
        _lib.check(self.lib.fpssft_decode(self.handle, _ptr(bins), _ptr(alpha), _ptr(tau), _ptr(k), _ptr(a),
                                          _ptr(count), _ptr(t0_count), _ptr(accepted), _ptr(status), _stream(stream)))

    def _check_set(self, k, a, count):
        _need(k, torch.int32, "k")
        _need(a, torch.complex64, "a")
        _need(count, torch.int32, "count")
        if tuple(k.shape) != (self.batch, self.k_cap, self.D) or tuple(a.shape) != (self.batch, self.k_cap) \
                or count.numel() != self.batch:
            raise ValueError(f"k, a, count must be [{self.batch}][{self.k_cap}][{self.D}], [{self.batch}][{self.k_cap}], [{self.batch}]")

    def finalize(self, k, a, count, stream=None):
        self._check_set(k, a, count)
        _lib.check(self.lib.fpssft_finalize(self.handle, _ptr(k), _ptr(a), _ptr(count), _stream(stream)))

    def adjoint_project(self, grad_bins, offsets, alpha, tau, grad_cubes, stream=None):
        """grad_cubes += P^H grad_bins (cube layout at offsets)."""
        S = self._sched(alpha, tau)
        _need(grad_bins, torch.complex64, "grad_bins")
        _need(grad_cubes, torch.complex64, "grad_cubes")
        _need(offsets, torch.int64, "offsets")
        self._check_extent(grad_cubes, offsets)
        _lib.check(self.lib.fpssft_adjoint(self.handle, _lib.ADJ_PROJECT, _ptr(grad_bins), _ptr(offsets),
                                           _ptr(alpha), _ptr(tau), S, None, None, _ptr(grad_cubes), _stream(stream)))
        return grad_cubes

    def adjoint_synth(self, grad_bins, alpha, tau, k, count, grad_a=None, stream=None):
        """grad_a = S^H grad_bins for the set (k, count); entries i >= count[b] are left untouched."""
        S = self._sched(alpha, tau)
        _need(grad_bins, torch.complex64, "grad_bins")
        if grad_a is None:
            grad_a = torch.zeros((self.batch, self.k_cap), dtype=torch.complex64, device=grad_bins.device)
        _lib.check(self.lib.fpssft_adjoint(self.handle, _lib.ADJ_SYNTH, _ptr(grad_bins), None, _ptr(alpha),
                                           _ptr(tau), S, _ptr(k), _ptr(count), _ptr(grad_a), _stream(stream)))
        return grad_a

    def refine_workspace_bytes(self):
        n = ctypes.c_size_t(0)
        _lib.check(self.lib.fpssft_refine_workspace_size(self.handle, ctypes.byref(n)))
        return int(n.value)

    def refine(self, bins, alpha, tau, k, a, count, iters=25, tol=1e-7, workspace=None, resid=None, stream=None):
        """Least-squares amplitudes on the support (k, count) over the rows alpha/tau, from the line
        DFTs `bins` of those rows (fpssft_refine); `a` is refined in place.  Returns (a, resid)."""
        S = self._sched(alpha, tau)
        _need(bins, torch.complex64, "bins")
        self._check_set(k, a, count)
        if tuple(bins.shape) != self._bins_shape(S):
            raise ValueError(f"bins must be {self._bins_shape(S)}")
        nbytes = self.refine_workspace_bytes()
        if workspace is None:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device=bins.device)
        _need(workspace, torch.uint8, "workspace")
        if resid is None:
            resid = torch.empty(self.batch, dtype=torch.float32, device=bins.device)
        _need(resid, torch.float32, "resid")
        _lib.check(self.lib.fpssft_refine(self.handle, _ptr(bins), _ptr(alpha), _ptr(tau), S, _ptr(k), _ptr(count),
                                          _ptr(a), int(iters), float(tol), _ptr(workspace),
                                          workspace.numel(), _ptr(resid), _stream(stream)))
        return a, resid


def probe_gather(buf, reads_per_thread=64, threads_total=152 * 8 * 256, load_mode=0, pair=0, stream=None):
    """Random 8-byte gathers over `buf` (complex64 CUDA tensor, power-of-two length); returns the
    output tensor (one complex64 per thread).  Time it with CUDA events around the call."""
    lib = _lib.load()
    _need(buf, torch.complex64, "buf")
    out = torch.empty(threads_total, dtype=torch.complex64, device=buf.device)
    _lib.check(lib.fpssft_probe_gather(_ptr(buf), buf.numel(), int(reads_per_thread), int(threads_total),
                                       int(load_mode), int(pair), _ptr(out), _stream(stream)))
    return out


def l2_fetch_granularity(nbytes=-1):
    """Set the process's L2 fetch-granularity hint (0/32/64/128 bytes; < 0 only queries); returns
    the previous value."""
    lib = _lib.load()
    prev = ctypes.c_int(0)
    _lib.check(lib.fpssft_l2_fetch_granularity(int(nbytes), ctypes.byref(prev)))
    return prev.value
