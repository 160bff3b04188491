"""The unfused, per-signal form of the recovery loop: the comparison baseline for the batched
persistent kernel.

One signal at a time and, per iteration, separate launches: the line gather (fpssft_lines), an
L-point FFT from torch.fft (cuFFT) divided by L, the peel (fpssft_synth with accumulate = -1), the
classify/decode/merge (fpssft_decode), and a host read of the T0 count for the early stop.  Same
schedule and thresholds as the fused path, so it recovers the same sets; it differs only in how
the work is launched.
"""
from __future__ import annotations

import numpy as np
import torch

from .api import Params, Plan


class PlainRecoverer:
    def __init__(self, params: Params, device="cuda"):
        self.params = params
        self.device = torch.device(device)
        self.plans = {}

    def _plan(self, dims):
        key = tuple(int(v) for v in dims)
        if key not in self.plans:
            self.plans[key] = Plan([key], Params(**{**self.params.__dict__, "T": max(1, self.params.T)}))
        return self.plans[key]

    def recover_one(self, cube, alpha, tau, T):
        """cube: complex64 device tensor (flat); alpha, tau: int32 device [T][D]."""
        D = alpha.shape[1]
        dims = tuple(int(v) for v in self._dims)
        plan = self._plan(dims)
        L = int(plan.L[0])
        dev = self.device
        k = torch.zeros((1, plan.k_cap, D), dtype=torch.int32, device=dev)
        a = torch.zeros((1, plan.k_cap), dtype=torch.complex64, device=dev)
        count = torch.zeros(1, dtype=torch.int32, device=dev)
        t0 = torch.zeros(1, dtype=torch.int32, device=dev)
        acc = torch.zeros(1, dtype=torch.int32, device=dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        off = torch.zeros(1, dtype=torch.int64, device=dev)
        iters = 0
        nvtx = torch.cuda.nvtx   # one range per step of the iteration (visible to ncu --nvtx)
        for t in range(T):
            al = alpha[t:t + 1].reshape(1, 1, D)
            ta = tau[t:t + 1].reshape(1, 1, D)
            with nvtx.range("gather"):
                lines = plan.lines(cube, off, al, ta)
            with nvtx.range("line_dft"):
                bins = (torch.fft.fft(lines[..., :L], dim=-1) / L).contiguous()
            with nvtx.range("peel"):
                plan.synth(al, ta, k, a, count, accumulate=-1, bins=bins)
            with nvtx.range("decode_merge"):
                plan.decode(bins, al, ta, k, a, count, t0, status, accepted=acc)
            iters = t + 1
            n_t0 = int(t0.item())
            if (self.params.early_stop and n_t0 == 0) or int(status.item()) != 0 or \
                    (self.params.early_stop == 2 and int(acc.item()) == n_t0):
                break
        plan.finalize(k, a, count)
        n = int(count.item())
        return (k[0, :n].cpu().numpy().astype(np.int64), a[0, :n].cpu().numpy().astype(np.complex128), iters,
                int(status.item()))

    def recover(self, wl, cubes_d, alpha_d, tau_d, signals):
        """Recover the listed signals of a workload whose cubes/schedules are already on the device."""
        out = []
        for b in signals:
            self._dims = wl.dims[b]
            n = int(np.prod(wl.dims[b]))
            o = int(wl.offsets[b])
            T = int(wl.T[b]) if self.params.T == 0 else self.params.T
            out.append(self.recover_one(cubes_d[o:o + n], alpha_d[b], tau_d[b], T))
        return out
