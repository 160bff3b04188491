"""Per-phase timing of the recovery kernels (tracing; no counterpart in the paper).

Builds the library variant compiled with FPSSFT_PHASE_TIMERS (libfpssft_phases.so, next to
libfpssft.so), recovers a synthetic workload with it and reports, from the SM cycle counters that
variant keeps (fpssft_phase_read in include/fpssft.h), how long each phase of the recovery loop
took: setup, gather, FFT, peel, decode (classify and merge), exchange (the cluster barriers of the
cluster path) and output, per CTA and per iteration.  Cycles are converted to microseconds with the
cycles-per-nanosecond ratio the same CTAs measured, so the figures hold at whatever clock the
launch ran.  The phase barriers make the timed launch slower than a plain one (`event_ms` is the
timed launch); its results are the same.

    python -m paper_1711_11407_gb300.phases --workload single_240x256 [--batch B] [--fft-path P]

The variant replaces libfpssft.so in the process that runs this, so run it in a process of its
own.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os

from . import _lib

PHASES = ("setup", "gather", "fft", "peel", "decode", "exchange", "output")
VARIANT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libfpssft_phases.so")


def build_variant(force=False):
    """Compile the phase-timer variant of the library (only when a source is newer)."""
    return _lib.build(force=force, out=VARIANT_PATH, defines=("FPSSFT_PHASE_TIMERS",))


def read(lib):
    """Raw counters of the launches since the last read (and clear them)."""
    buf = (ctypes.c_int64 * (len(PHASES) + 4))()
    _lib.check(lib.fpssft_phase_read(buf))
    return [int(v) for v in buf]


def summarize(raw):
    """Per-CTA and per-iteration microseconds of each phase from the raw counters."""
    n = len(PHASES)
    cycles = raw[:n]
    ctas, iters, total, ns = raw[n:n + 4]
    if ctas <= 0 or ns <= 0:
        raise ValueError("no timed CTA in the counters")
    per_ns = total / ns                              # cycles per nanosecond of these CTAs
    us = lambda c, by: c / by / per_ns / 1e3         # noqa: E731
    other = total - sum(cycles)
    return {
        "ctas": ctas,
        "iterations_per_cta": iters / ctas,
        "sm_clock_mhz": per_ns * 1e3,
        "cta_us": us(total, ctas),
        "phase_us_per_cta": {p: us(c, ctas) for p, c in zip(PHASES, cycles)} | {"unmarked": us(other, ctas)},
        "phase_us_per_iteration": ({p: us(c, iters) for p, c in zip(PHASES, cycles)} if iters > 0 else None),
    }


def run(workload, batch=None, reps=10, snr_db="default", dump=None, **plan_over):
    """Recover `workload` reps times with the variant loaded and summarise the phase counters."""
    import numpy as np
    import torch

    from . import configs, synth
    from .api import Plan

    lib = _lib.load()
    wl = synth.make_workload(workload, batch=batch, snr_db=snr_db)
    plan = Plan(wl.dims, configs.params_for(wl, **plan_over))
    dev = torch.device("cuda")
    args = [torch.from_numpy(v).to(dev) for v in (wl.cubes, wl.offsets, wl.alpha, wl.tau)]
    out = plan.recover(*args)
    torch.cuda.synchronize()
    read(lib)                                        # drop the first launch
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    times = []
    for _ in range(reps):
        flush.zero_()                                # L2 cold, as in the benchmark
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.recover(*args, out=out)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    res = summarize(read(lib))
    res.update(workload=workload, batch=len(wl.offsets), reps=reps, event_ms=float(np.median(times)),
               plan={k: plan.info[k] for k in ("fft_path", "threads", "grid", "smem_bytes")})
    if dump:
        np.savez(dump, k=out.k.cpu().numpy(), a=out.a.cpu().numpy(), count=out.count.cpu().numpy(),
                 iters=out.iters.cpu().numpy(), status=out.status.cpu().numpy())
    plan.close()
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="single_240x256")
    ap.add_argument("--batch", type=int, default=None)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--noiseless", action="store_true", help="drop the workload's noise")
    ap.add_argument("--fft-path", type=int, default=None)
    ap.add_argument("--threads", type=int, default=None)
    ap.add_argument("--gather-mode", type=int, default=None)
    ap.add_argument("--cluster-set", type=int, default=None)
    ap.add_argument("--dump", default=None, help="save the last launch's output (.npz)")
    a = ap.parse_args(argv)
    _lib.use_library(build_variant())
    over = {k: v for k, v in (("fft_path", a.fft_path), ("threads", a.threads), ("gather_mode", a.gather_mode),
                              ("cluster_set", a.cluster_set)) if v is not None}
    res = run(a.workload, batch=a.batch, reps=a.reps, snr_db=None if a.noiseless else "default", dump=a.dump, **over)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
