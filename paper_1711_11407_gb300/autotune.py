"""Autotuner for the recovery launch: picks the kernel configuration of fpssft_recover for a batch.

Candidates are the valid combinations of
  fft_path     1 (one CTA per signal, shared-memory mixed-radix FFT), 2 (one warp per line,
               register FFT; only when every line length is 32, 64, 128 or 256) or 3 (one CTA per
               line, a cluster of D+1 CTAs per signal; only for lines of 512 points or more),
  gather_mode  1 (synchronous through L1), 2 (L2 only), 3 (asynchronous prefetch: cp.async into
               shared memory; on path 2 it replaces the register prefetch) or, on path 2, 4 (no
               prefetch of the next iteration: throughput over latency) or 5 (4 with the next
               iteration's samples hinted into L2),
  threads      CTA size for paths 1 and 3 (path 2 is fixed at 32 (D+1)),
  cluster_set  on path 3, the recovered set in shared memory (1) or in global workspace (2; smaller
               CTAs, more of them resident),
  radix_plan   the order of the shared-memory FFT's mixed-radix stages (paths 1 and 3): tried for
               the fastest of the candidates above, each plan whose stage sequence differs from
               the default for some line length of the batch (fpssft_fft_stages).
Each candidate is timed on the caller's own inputs with CUDA events (warm-up first, a buffer larger
than L2 written between timed launches); the fastest wins.  Results are cached in a JSON file keyed
by GPU name, D, the sorted set of shapes, k_cap, T and the stop rule, so a batch with the same
layout is not re-tuned.  Tuning never changes what is computed, only how it is launched.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import replace

import numpy as np
import torch

from ._lib import ERR_UNSUPPORTED, FpssftError
from .api import Params, Plan

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "fpssft_autotune.json")


def cache_key(dims, params: Params, gpu_name: str):
    dims = np.asarray(dims, np.int64)
    shapes = sorted({tuple(int(v) for v in d) for d in dims})
    return json.dumps({"gpu": gpu_name, "D": int(dims.shape[1]), "shapes": shapes, "k_cap": int(params.k_cap),
                       "T": int(params.T), "early_stop": int(params.early_stop)}, sort_keys=True)


def candidates(dims, params: Params):
    """The launch configurations worth timing for this batch (host logic only)."""
    dims = np.asarray(dims, np.int64)
    Ls = {math.lcm(*[int(v) for v in d]) for d in dims}
    warp_ok = all(L % 32 == 0 and L // 32 in (1, 2, 4, 8) for L in Ls)
    L_max = max(Ls) if Ls else 1
    out = []
    if warp_ok:
        for gm in (1, 3, 4, 5):
            out.append(replace(params, fft_path=2, gather_mode=gm, threads=0))
    for th in (128, 256, 512, 1024):
        if th > 4 * max(32, L_max) or (th == 1024 and L_max < 512):
            continue
        for gm in (1, 3):
            out.append(replace(params, fft_path=1, gather_mode=gm, threads=th))
    if L_max >= 512:
        for th in (256, 512, 1024):
            if th > L_max // 2:
                continue
            for gm in (1, 3):
                for cs in (1, 2):
                    out.append(replace(params, fft_path=3, gather_mode=gm, threads=th, cluster_set=cs))
    return out


def fft_stages(L, radix_plan):
    """Radices of the L-point FFT's stages under a radix plan (host-only library call)."""
    import ctypes

    from . import _lib
    lib = _lib.load()
    out = (ctypes.c_int32 * 24)()
    n = ctypes.c_int32(0)
    _lib.check(lib.fpssft_fft_stages(int(L), int(radix_plan), out, ctypes.byref(n)))
    return [int(out[i]) for i in range(n.value)]


def radix_candidates(dims, params: Params):
    """The radix plans other than the default that change some line length's stage sequence, for
    the shared-memory FFT paths (host logic only)."""
    if params.fft_path not in (1, 3):
        return []
    dims = np.asarray(dims, np.int64)
    Ls = sorted({math.lcm(*[int(v) for v in d]) for d in dims})
    base = [fft_stages(L, 0) for L in Ls]
    out = []
    for rp in (1, 2, 3):
        if any(fft_stages(L, rp) != b for L, b in zip(Ls, base)):
            out.append(replace(params, radix_plan=rp))
    return out


def _time(plan, args, reps, flush):
    """Mean launch time over at least `reps` launches; short launches get more of them (about 4 ms
    of timed work, at most 50), so that candidates a few microseconds apart are told apart."""
    stream = torch.cuda.current_stream()
    plan.recover(*args)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.recover(*args)
    e1.record(stream)
    e1.synchronize()
    first = max(e0.elapsed_time(e1), 1e-3)
    reps = max(reps, min(50, int(math.ceil(4.0 / first))))
    total = 0.0
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.recover(*args)
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    return total / reps


def tune(dims, params: Params, cubes, offsets, alpha, tau, reps=5, cache_path=DEFAULT_CACHE, use_cache=True):
    """Return (best Params, {description: ms}) for recovering this batch."""
    gpu = torch.cuda.get_device_name(cubes.device)
    key = cache_key(dims, params, gpu)
    cache = {}
    if use_cache and cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except Exception:
            cache = {}
    if use_cache and key in cache:
        return replace(params, **cache[key]["choice"]), cache[key]["timings"]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=cubes.device)
    timings = {}
    best, best_ms = None, float("inf")

    def run(cands):
        nonlocal best, best_ms
        for cand in cands:
            try:
                plan = Plan(dims, cand)
            except FpssftError as e:
                if e.status == ERR_UNSUPPORTED:
                    continue
                raise
            out = plan.alloc_output(cubes.device)
            ms = _time(plan, (cubes, offsets, alpha, tau, out), reps, flush)
            desc = f"path={cand.fft_path} gather={cand.gather_mode} threads={plan.info['threads']}"
            if cand.fft_path == 3:
                desc += " set=global" if plan.info["global_workspace"] else " set=shared"
            if cand.radix_plan:
                desc += f" radix_plan={cand.radix_plan}"
            timings[desc] = ms
            if ms < best_ms:
                best, best_ms = cand, ms
            plan.close()

    run(candidates(dims, params))
    if best is None:
        return params, timings
    run(radix_candidates(dims, best))
    choice = {"fft_path": best.fft_path, "gather_mode": best.gather_mode, "threads": best.threads,
              "radix_plan": best.radix_plan, "cluster_set": best.cluster_set}
    if cache_path:
        cache[key] = {"choice": choice, "timings": timings}
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return best, timings
