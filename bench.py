#!/usr/bin/env python3
"""Throughput of the batched FPS-SFT recovery loop on GB300.

Workload (default): the uneven 2-D batch -- 4096 noiseless signals with shapes drawn uniformly
from {64x64, 128x128, 128x256, 256x256}, K = ceil(N/200) unit-magnitude sinusoids each, line
budget T = N / (3L) per signal, early stop.  One step = one fpssft_recover launch (captured in a
CUDA graph) over the whole batch with inputs resident in HBM; between timed steps a 256 MiB buffer
is written to flush L2.  The line prints signals/s, the roofline of the recovery kernel, the
end-to-end rate through fpssft_recover_host (host buffers, copies included), the unfused
per-signal GPU form on a sample, and the FP64 oracle on host cores on a bounded sample.

Multi-GPU (torchrun): every rank recovers its own batch of the same recipe (independent seeds);
there is no collective on the data path (weak scaling); a barrier and a max-reduce of the timed
region are the only communication.

--impl reference times the FP64 oracle (the reference implementation of this method) on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "signals/s batched FPS-SFT vs plain per-signal GPU at exact support; HBM GB/s"
UNIT = "signals/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fpssft", choices=["fpssft", "reference"])
    ap.add_argument("--workload", default="uneven_2d")
    ap.add_argument("--batch", type=int, default=None, help="override the signal count (smaller captures)")
    ap.add_argument("--plain-sample", type=int, default=32)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--quick", action="store_true", help="only the timed device loop (for profiler runs)")
    ap.add_argument("--ceiling", action="store_true", help="with --quick, still measure the gather ceiling")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--gather-mode", type=int, default=0)
    ap.add_argument("--fft-path", type=int, default=0)
    ap.add_argument("--cluster-set", type=int, default=0, help="path 3: 1 set in shared memory, 2 in global workspace")
    ap.add_argument("--early-stop", type=int, default=None,
                    help="stop rule (0 none, 1 after an iteration with no line-0 bin passing T0, 2 also after "
                         "an iteration whose line-0 bins passing T0 were all decoded); default: the workload's")
    ap.add_argument("--no-autotune", action="store_true", help="use the library's default launch configuration")
    ap.add_argument("--l2-fetch", type=int, default=-1, help="L2 fetch granularity hint in bytes (-1: leave)")
    ap.add_argument("--refine-rows", type=int, default=0,
                    help="after the timed recovery: least-squares amplitude refinement over this many schedule "
                         "rows, on the recovered and on the planted support, timed, with its errors (0: off)")
    ap.add_argument("--refine-iters", type=int, default=30)
    ap.add_argument("--refine-oracle", type=int, default=2, help="signals checked against FP64 least squares")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(x, world, device):
    """The largest x over all ranks (the slowest rank's time is the job's); x itself when alone."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms_per_step):
    """Whole-job throughput: what every rank processed in a step over the slowest rank's step time."""
    return units_per_rank * world / (ms_per_step / 1000.0)


def stratified(wl, n, seed=0):
    """n signal indices spread evenly over the distinct shapes of the workload."""
    rng = np.random.default_rng(seed)
    keys = [tuple(int(v) for v in d) for d in wl.dims]
    groups = {}
    for i, k in enumerate(keys):
        groups.setdefault(k, []).append(i)
    out = []
    per = max(1, n // len(groups))
    for k in sorted(groups):
        g = groups[k]
        out.extend(int(i) for i in rng.choice(g, min(per, len(g)), replace=False))
    return out[:max(n, len(groups))]


def same_sets(ref, other, amp_tol=1e-4):
    """True when two RecoverOutputs hold the same recovered sets: count, iterations and status
    equal, and per signal the first count rows of k equal and of a within amp_tol relative."""
    import torch
    r = {f: getattr(ref, f).cpu() for f in ("k", "a", "count", "iters", "status")}
    o = {f: getattr(other, f).cpu() for f in ("k", "a", "count", "iters", "status")}
    if not all(torch.equal(r[f], o[f]) for f in ("count", "iters", "status")):
        return False
    rows = torch.arange(r["k"].shape[1])[None, :] < r["count"][:, None].long()
    if not torch.equal(r["k"][rows], o["k"][rows]):
        return False
    ra, oa = r["a"][rows], o["a"][rows]
    return bool(torch.all(torch.abs(ra - oa) <= amp_tol * torch.abs(ra)))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def strip_comments(src):
    """C/C++ source without comments and with whitespace runs collapsed (string and character
    literals kept), so that a comment-only edit leaves the kernel's hash unchanged."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def source_hash():
    """Hash of the kernel sources' code (every file under csrc/, comments and whitespace excluded)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1711_11407_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, name), encoding="utf-8") as f:
                h.update(name.encode())
                h.update(strip_comments(f.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(workload, batch):
    """DRAM bytes per launch of the recovery kernel from the committed ncu summary, when it was
    taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"k_recover_{workload}.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None, None
    if d.get("source_hash") != source_hash():
        return None, path
    per_signal = d["dram_bytes_per_launch"] / d["batch"]
    return per_signal * batch, path


def probe_dram_bytes():
    """DRAM bytes per isolated random access at the probe's ceiling (committed ncu record), or None."""
    try:
        with open(os.path.join(ROOT, "profiles", "probe_gather_random_access.json")) as f:
            return json.load(f)
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region: the sampler starts before it
    (and its first line is awaited), every line is time-stamped on arrival, and the summary keeps
    the lines that arrived between begin() and end()."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid, period_ms=50):
        import threading
        self.uuid = uuid
        self.lines = []
        self.t0 = self.t1 = None
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", str(period_ms)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        deadline = time.monotonic() + 5.0
        while not self.lines and time.monotonic() < deadline and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line))

    def begin(self):
        self.t0 = time.monotonic()

    def end(self):
        self.t1 = time.monotonic()
        time.sleep(0.12)     # let the sample that covers the end of the region arrive
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for t, line in self.lines:
            if self.t0 is None or not (self.t0 <= t <= self.t1 + 0.1):
                continue
            r = [c.strip() for c in next(csv.reader([line]))]
            if len(r) < 10 or (self.uuid and self.uuid not in r[1]):
                continue
            rows.append(r)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no sample inside the timed region"], "samples": 0}
        num = lambda v: float(v) if v.replace(".", "", 1).isdigit() else None
        sm = [num(r[2]) for r in rows if num(r[2]) is not None]
        mx = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[6:10]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---- the FP64 oracle on every host core: one spawned process per core, signals spread over them --
_ORACLE = {}


def _oracle_init(shm_name, n_elems, dims, offsets, alpha, tau, T, pd):
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=shm_name)
    _ORACLE.update(shm=shm, cubes=np.ndarray((n_elems,), np.complex64, buffer=shm.buf), dims=dims,
                   offsets=offsets, alpha=alpha, tau=tau, T=T, pd=pd)


def _oracle_many(indices):
    """Recover the given signals with the oracle as it stands; returns (count, seconds)."""
    from oracle import fpssft_oracle as O
    c = _ORACLE
    t0 = time.perf_counter()
    for b in indices:
        dims = tuple(int(v) for v in c["dims"][b])
        n = int(np.prod(dims))
        o = int(c["offsets"][b])
        x = c["cubes"][o:o + n].reshape(dims).astype(np.complex128)
        T = int(c["T"][b]) if c["pd"]["T"] == 0 else int(c["pd"]["T"])
        pd = dict(c["pd"], T=T)
        O.recover(x, c["alpha"][b, :T], c["tau"][b, :T], O.Params(**pd))
    return len(indices), time.perf_counter() - t0


class OraclePool:
    """A spawn-started pool with one worker per available host core; the cubes are shared with the
    workers through one shared-memory block (no per-call copies)."""

    def __init__(self, wl, params, cores=None):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        self.cores = int(cores or len(os.sched_getaffinity(0)))
        self.shm = shared_memory.SharedMemory(create=True, size=max(8, wl.cubes.nbytes))
        np.ndarray(wl.cubes.shape, np.complex64, buffer=self.shm.buf)[:] = wl.cubes
        pd = dict(T=int(params.T), k_cap=int(params.k_cap), theta0=float(params.theta0), rho=float(params.rho),
                  eta=float(params.eta), early_stop=int(params.early_stop))
        self.pool = mp.get_context("spawn").Pool(
            self.cores, initializer=_oracle_init,
            initargs=(self.shm.name, int(wl.cubes.size), wl.dims, wl.offsets, wl.alpha, wl.tau, wl.T, pd))
        self.pool.map(_oracle_many, [[] for _ in range(self.cores)])     # workers started and attached

    def run(self, indices):
        """Recover `indices` spread over the workers; returns wall seconds."""
        return self.run_chunks([indices[i::self.cores] for i in range(self.cores)])

    def run_chunks(self, chunks):
        """Recover each list of `chunks` on a worker of its own; returns wall seconds."""
        t0 = time.perf_counter()
        self.pool.map(_oracle_many, [c for c in chunks if c])
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()
        self.shm.close()
        self.shm.unlink()


def oracle_rate(wl, params, seconds, order):
    """FP64 oracle on all host cores: signals/s over a bounded sample (signals taken in `order`,
    rounds of 4 signals per core until `seconds` of CPU work have been spent).  A workload with
    fewer signals than cores keeps one core per signal busy: each of those cores recovers its
    signal over and over (doubling the repeats) until the round takes a second, so that process
    start-up and hand-over do not dominate a few milliseconds of work."""
    op = OraclePool(wl, params)
    try:
        if len(order) < op.cores:
            reps = 1
            while True:
                wall = op.run_chunks([[b] * reps for b in order])
                if wall >= 1.0 or reps >= 1 << 16:
                    return len(order) * reps / wall, len(order) * reps, wall, len(order)
                reps *= 2
        wall, n, pos = 0.0, 0, 0
        rnd = 4 * op.cores
        while pos < len(order) and (wall * op.cores < seconds or n < op.cores):
            idx = order[pos:pos + rnd]
            pos += rnd
            wall += op.run(idx)
            n += len(idx)
        return n / wall, n, wall, op.cores
    finally:
        op.close()


def run_reference(args):
    """Reference arm: the FP64 oracle on host cores, each step a bounded sample of the workload."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    from paper_1711_11407_gb300 import configs, synth
    wl = synth.make_workload(args.workload, batch=args.batch)
    p = configs.params_for(wl)
    op = OraclePool(wl, p)
    per_step = 4 * op.cores
    order = stratified(wl, per_step * (args.steps + args.warmup) + per_step, seed=1)
    times = []
    n_done = 0
    try:
        for s in range(args.warmup + args.steps):
            idx = order[(s * per_step) % len(order):][:per_step] or order[:per_step]
            dt = op.run(idx)
            if s >= args.warmup:
                times.append(dt)
                n_done += len(idx)
    finally:
        op.close()
    total = sum(times)
    value = n_done / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "batch": int(wl.batch), "signals_per_step": per_step,
                       "note": "each step recovers a stratified sample of the workload's signals"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": op.cores, "kind": "oracle",
                             "sample": f"{n_done} signals over {args.steps} steps (stratified by shape), "
                                       f"numpy FP64, one spawned process per core"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def other_stop_rule(wl, p, cubes, offs, alpha, tau, stream, flush, world, dev, steps=200):
    """The same launch timed with the other early-stop reading (1 <-> 2), for comparison: 1 stops
    after an iteration in which no line-0 bin passes T0, 2 already after an iteration whose line-0
    bins passing T0 were all decoded."""
    import torch
    from dataclasses import replace

    from oracle import fpssft_oracle as O
    from paper_1711_11407_gb300.api import Plan
    rule = 1 if p.early_stop == 2 else 2
    plan = Plan(wl.dims, replace(p, early_stop=rule))
    out = plan.alloc_output(dev)
    with torch.cuda.stream(stream):
        plan.recover(cubes, offs, alpha, tau, out=out)
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            plan.recover(cubes, offs, alpha, tau, out=out)
        for _ in range(3):
            g.replay()
        stream.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.replay()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    step = max_over_ranks(sum(ms), world, dev) / steps
    ks, cnt, iters = out.k.cpu().numpy(), out.count.cpu().numpy(), out.iters.cpu().numpy()
    ok = sum(int(np.array_equal(O.linear_index(ks[b, :cnt[b]].astype(np.int64), tuple(int(v) for v in wl.dims[b])),
                                np.sort(O.linear_index(wl.k_true[b], tuple(int(v) for v in wl.dims[b])))))
             for b in range(wl.batch))
    plan.close()
    return {"early_stop": rule, "ms_per_step": step, "value": job_rate(wl.batch, world, step), "steps": steps,
            "mean_iterations": float(np.mean(iters)), "exact_support_success": ok / wl.batch}


def refine_leg(args, wl, plan, cubes, offs, alpha, tau, out, stream):
    """Least-squares amplitude refinement (fpssft_refine) after the recovery, over the first R
    schedule rows: timed on the device (projection of the rows plus the CG loop, per batch), and
    its amplitude errors against the planted amplitudes and against the oracle's FP64 least squares
    on a few signals.  Run on the recovered support and on the planted support."""
    import torch

    from oracle import fpssft_oracle as O
    R = min(args.refine_rows, int(alpha.shape[1]))
    ra, rt = alpha[:, :R].contiguous(), tau[:, :R].contiguous()
    dev = cubes.device
    kp = torch.zeros_like(out.k)
    cp = torch.zeros_like(out.count)
    for b in range(wl.batch):
        n = len(wl.k_true[b])
        kp[b, :n] = torch.from_numpy(wl.k_true[b].astype(np.int32))
        cp[b] = n
    supports = {"recovered": (out.k, out.a.clone(), out.count), "planted": (kp, torch.zeros_like(out.a), cp)}
    ws = torch.empty(plan.refine_workspace_bytes(), dtype=torch.uint8, device=dev)
    resid = torch.empty(wl.batch, dtype=torch.float32, device=dev)
    y = torch.empty((wl.batch, R, wl.D + 1, plan.L_max), dtype=torch.complex64, device=dev)
    rec = {"rows": R, "cg_iterations": args.refine_iters,
           "samples_fraction_of_cube": float(np.mean(R * (wl.D + 1) * plan.L / np.prod(wl.dims.astype(np.float64), axis=1)))}
    for label, (k, a0, cnt) in supports.items():
        a = torch.empty_like(a0)
        with torch.cuda.stream(stream):
            def run():
                a.copy_(a0)
                plan.project(cubes, offs, ra, rt, out=y, stream=stream)
                plan.refine(y, ra, rt, k, a, cnt, iters=args.refine_iters, workspace=ws, resid=resid, stream=stream)
            run()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 10
            e0.record(stream)
            for _ in range(reps):
                run()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            # the same work replayed from a CUDA graph (the refinement waits on nothing on the host)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                run()
            g.replay()
            stream.synchronize()
            e0.record(stream)
            for _ in range(reps):
                g.replay()
            e1.record(stream)
            e1.synchronize()
            ms_graph = e0.elapsed_time(e1) / reps
        ah = a.cpu().numpy()
        a0h = a0.cpu().numpy()
        kh = k.cpu().numpy()
        ch = cnt.cpu().numpy()
        rel_ref, rel_dec, n_common, n_total = [], [], 0, 0
        for b in range(wl.batch):
            truth = dict(zip(map(tuple, wl.k_true[b].tolist()), wl.a_true[b]))
            n = int(ch[b])
            n_total += n
            for i in range(n):
                t = truth.get(tuple(int(v) for v in kh[b, i]))
                if t is None:
                    continue
                n_common += 1
                rel_ref.append(abs(ah[b, i] - t) / abs(t))
                if label == "recovered":
                    rel_dec.append(abs(a0h[b, i] - t) / abs(t))
        vs_oracle = []
        for b in [b for b in range(wl.batch) if ch[b] > 0][:args.refine_oracle]:
            n = int(ch[b])
            ref = O.refine_lstsq(wl.cube(b), wl.alpha[b, :R], wl.tau[b, :R], kh[b, :n].astype(np.int64))
            vs_oracle.append(float(np.linalg.norm(ah[b, :n] - ref) / np.linalg.norm(ref)))
        med = lambda v: float(np.median(v)) if v else None
        rec[label] = {"ms_per_batch": ms, "ms_per_batch_graph": ms_graph,
                      "signals_per_s": wl.batch / (ms / 1000.0), "entries": n_total,
                      "entries_in_planted_support": n_common,
                      "refined_rel_error_vs_planted_median": med(rel_ref),
                      "refined_rel_error_vs_planted_p90": float(np.percentile(rel_ref, 90)) if rel_ref else None,
                      "rel_l2_vs_fp64_least_squares": vs_oracle}
        if label == "recovered":
            rec[label]["decoded_rel_error_vs_planted_median"] = med(rel_dec)
    return rec


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    from oracle import fpssft_oracle as O
    from paper_1711_11407_gb300 import configs, synth
    from paper_1711_11407_gb300.api import Plan

    rank, local_rank, world = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    # ---- workload (each rank its own independent batch of the same recipe) ----------------------
    seed = 1234 + 4 + 1000 * rank if args.workload == "uneven_2d" else None
    if seed is None:
        seed = 1234 + {v: k for k, v in synth.WORKLOAD_IDS.items()}[args.workload] + 1000 * rank
    wl = synth.make_workload(args.workload, seed=seed, batch=args.batch)
    over = {} if args.early_stop is None else {"early_stop": args.early_stop}
    p = configs.params_for(wl, **over, threads=args.threads, ctas_per_sm=args.ctas_per_sm, gather_mode=args.gather_mode,
                           fft_path=args.fft_path, cluster_set=args.cluster_set)
    from paper_1711_11407_gb300.api import l2_fetch_granularity
    l2_prev = l2_fetch_granularity(args.l2_fetch)
    cubes = torch.from_numpy(wl.cubes).to(dev)
    offs = torch.from_numpy(wl.offsets).to(dev)
    alpha = torch.from_numpy(wl.alpha).to(dev)
    tau = torch.from_numpy(wl.tau).to(dev)
    tuning = None
    if not args.no_autotune and args.threads == 0 and args.fft_path == 0 and args.gather_mode == 0 \
            and args.cluster_set == 0:
        from paper_1711_11407_gb300 import autotune
        p, tuning = autotune.tune(wl.dims, p, cubes, offs, alpha, tau, reps=3, cache_path=None)
    plan = Plan(wl.dims, p)
    out = plan.alloc_output(dev)
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        plan.recover(cubes, offs, alpha, tau, out=out)

    with torch.cuda.stream(stream):
        step()                       # first call outside capture (validates and warms the module)
        stream.synchronize()
        graph = None
        if not args.no_graph:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                step()
        run = graph.replay if graph is not None else step
        for _ in range(max(3, args.warmup)):
            run()
        stream.synchronize()

        # ---- timed device loop ---------------------------------------------------------------
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        uuid = None
        try:
            uuid = str(torch.cuda.get_device_properties(dev).uuid)
        except Exception:
            pass
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(uuid)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk.begin()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            run()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        clk.end()
        if world > 1:
            dist.barrier()
        step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ms_per_step = total_ms / args.steps
    value = job_rate(wl.batch, world, ms_per_step)

    # ---- correctness of what was timed: exact support vs the planted spectra ---------------------
    torch.cuda.synchronize()
    ks, cnt, iters = out.k.cpu().numpy(), out.count.cpu().numpy(), out.iters.cpu().numpy()
    ok = 0
    for b in range(wl.batch):
        dims = tuple(int(v) for v in wl.dims[b])
        truth = np.sort(O.linear_index(wl.k_true[b], dims))
        ok += int(np.array_equal(O.linear_index(ks[b, :cnt[b]].astype(np.int64), dims), truth))
    success = ok / wl.batch

    # ---- roofline of the recovery kernel ---------------------------------------------------------
    L = plan.L.astype(np.int64)
    it64 = iters.astype(np.int64)
    useful = float(np.sum(it64 * (wl.D + 1) * L * 8))           # gathered sample bytes (algorithmic)
    peaks, peak_src = measured_peaks()
    achieved = useful / (ms_per_step / 1000.0) / 1e9
    traffic, _ = profiled_traffic(args.workload, wl.batch)
    path = plan.info.get("fft_path")
    kname = {2: f"k_recover_w<{wl.D}>", 3: f"k_recover_c<{wl.D}>"}.get(path, f"k_recover<{wl.D}>")
    kdesc = {2: "persistent; one warp per line", 3: "one CTA per line, a cluster of D+1 CTAs per signal"}.get(
        path, "persistent; one CTA per signal")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                "frac": achieved / float(peaks["hbm_gbs"]), "traffic": traffic,
                "peak_source": f"{peak_src} (hbm_gbs, copy bandwidth; kernel timed alone: burst figure)",
                "algorithmic_bytes_per_launch": useful,
                "kernel": f"{kname} ({kdesc}; one launch per step, CUDA events on the launching stream)"}
    if traffic is not None:      # DRAM bytes actually moved per second (sectors, not useful samples)
        roofline["traffic_gbs"] = traffic / (ms_per_step / 1000.0) / 1e9
        roofline["traffic_frac"] = roofline["traffic_gbs"] / float(peaks["hbm_gbs"])
    # second view: the gather against the measured random-access ceiling of this GPU.  Each line
    # position reads one adjacent pair (lines tau and tau + e_{D-1}) and D - 1 isolated samples.
    if not args.quick or args.ceiling:
        from paper_1711_11407_gb300.api import probe_gather
        probe_buf = torch.zeros(1 << 29, dtype=torch.complex64, device=dev)          # 4 GiB >> L2
        rates = {}
        nthr = 152 * 16 * 256
        for pair in (0, 1):
            probe_gather(probe_buf, 64, nthr, 0, pair)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                probe_gather(probe_buf, 64, nthr, 0, pair)
            e1.record()
            torch.cuda.synchronize()
            rates[pair] = nthr * 64 / (e0.elapsed_time(e1) / 5 / 1000.0)
        del probe_buf
        pairs = float(np.sum(it64 * L))
        singles = float(np.sum(it64 * L * (wl.D - 1)))
        t_ceiling = pairs / rates[1] + singles / rates[0]
        roofline["gather_ceiling"] = {"pair_accesses_per_s": rates[1], "single_accesses_per_s": rates[0],
                                      "pairs_per_launch": pairs, "singles_per_launch": singles,
                                      "ceiling_ms": 1000.0 * t_ceiling, "frac": 1000.0 * t_ceiling / ms_per_step,
                                      "probe": "fpssft_probe_gather, 4 GiB buffer, 9.7M threads x 64 random reads"}
        # the same ceiling in DRAM bytes: the probe moves a whole line per isolated access, while the
        # kernel hits L2 for part of its samples, so compare the DRAM bytes each moves per second
        probe_bytes = probe_dram_bytes()
        if traffic is not None and probe_bytes is not None:
            probe_gbs = (pairs * probe_bytes["dram_bytes_per_pair_access"]
                         + singles * probe_bytes["dram_bytes_per_single_access"]) / t_ceiling / 1e9
            kern_gbs = traffic / (ms_per_step / 1000.0) / 1e9
            roofline["gather_ceiling"]["dram_view"] = {
                "kernel_dram_gbs": kern_gbs, "probe_dram_gbs": probe_gbs, "frac": kern_gbs / probe_gbs,
                "note": "kernel DRAM bytes per launch (roofline.traffic) per step time, against the DRAM bytes "
                        "per second the probe moves for the same mix of single and pair accesses"}

    refine_rec = refine_leg(args, wl, plan, cubes, offs, alpha, tau, out, stream) if args.refine_rows > 0 else None
    other_stop = other_stop_rule(wl, p, cubes, offs, alpha, tau, stream, flush, world, dev) \
        if p.early_stop in (1, 2) and not args.quick else None

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "batch_per_gpu": int(wl.batch), "global_batch": int(wl.batch * world),
                       "shapes": sorted({"x".join(str(int(v)) for v in d) for d in wl.dims}),
                       "K": "ceil(N/200)" if args.workload == "uneven_2d" else "per workload",
                       "T": "N/(3L) per signal, early stop", "l2": "256 MiB written between timed steps",
                       "cuda_graph": graph is not None, "parallelism": f"batch sharded over {world} GPU(s), no collective",
                       "threads": plan.info["threads"], "grid": plan.info["grid"], "smem_bytes": plan.info["smem_bytes"],
                       "fft_path": plan.info["fft_path"], "gather_mode": p.gather_mode,
                       "global_workspace": plan.info["global_workspace"],
                       "autotune_ms": tuning},
            "roofline": roofline, "gpu_launches": args.steps, "exact_support_success": success,
            "mean_iterations": float(np.mean(iters)),
            # samples read per signal as a fraction of its cube: iterations (D+1) L / N (Sec. 3's measure)
            "mean_sample_fraction": float(np.mean(it64 * (wl.D + 1) * L / np.prod(wl.dims.astype(np.float64), axis=1))),
            "clocks": clk.summary()}
    if refine_rec is not None:
        line["refine"] = refine_rec
    line["config"]["early_stop"] = int(p.early_stop)
    if other_stop is not None:
        line["other_stop_rule"] = other_stop

    if not args.quick:
        # ---- end to end through the host-buffer call ------------------------------------------
        # fpssft_recover_host in both host modes: every cube copied to the device (host_cubes 0), or
        # pinned cubes read in place over the host link, only offsets, schedules and results
        # copied (host_cubes 1).  Both are timed; `e2e` is the faster one, both are reported.
        from dataclasses import replace as _replace

        from paper_1711_11407_gb300.api import Plan as _Plan
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        h_cubes, h_offs, h_alpha, h_tau = pin(wl.cubes), pin(wl.offsets), pin(wl.alpha), pin(wl.tau)
        small = sum(int(x.numel() * x.element_size()) for x in (h_offs, h_alpha, h_tau))
        modes = {}
        for hc in (0, 1):
            hplan = _Plan(wl.dims, _replace(p, host_cubes=hc))
            h_out = hplan.alloc_output("cpu")
            for f in ("k", "a", "count", "iters", "status"):
                setattr(h_out, f, getattr(h_out, f).pin_memory())
            with torch.cuda.stream(stream):
                hplan.recover_host(h_cubes, h_offs, h_alpha, h_tau, out=h_out, stream=stream)
                if world > 1:
                    dist.barrier()
                e2e_ms = []
                for _ in range(args.steps):
                    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a0.record(stream)
                    hplan.recover_host(h_cubes, h_offs, h_alpha, h_tau, out=h_out, stream=stream)
                    a1.record(stream)
                    a1.synchronize()
                    e2e_ms.append(a0.elapsed_time(a1))
            e2e_step = max_over_ranks(sum(e2e_ms), world, dev) / args.steps
            d2h = sum(int(getattr(h_out, f).numel() * getattr(h_out, f).element_size())
                      for f in ("k", "a", "count", "iters", "status"))
            rec = {"value": job_rate(wl.batch, world, e2e_step), "unit": UNIT, "ms_per_step": e2e_step,
                   "h2d_bytes_per_step": small + (h_cubes.numel() * h_cubes.element_size() if hc == 0 else 0),
                   "d2h_bytes_per_step": d2h, "call": "fpssft_recover_host", "host_cubes": hc,
                   # the last run of this mode against the timed device run: whole sets compared
                   "matches_device_run": same_sets(out, h_out)}
            if hc == 1:
                rec["h2d_bytes_read_in_place_algorithmic"] = useful
                rec["note"] = ("pinned cubes read in place over NVLink-C2C: the gather fetches only the samples "
                               "the iterations use; h2d_bytes_per_step counts the copied offsets and schedules")
            modes["copy" if hc == 0 else "in_place"] = rec
            hplan.close()
        best = min(modes.values(), key=lambda r: r["ms_per_step"])
        line["e2e"] = dict(best)
        line["e2e_modes"] = {k: {kk: v[kk] for kk in ("value", "ms_per_step", "h2d_bytes_per_step", "matches_device_run")}
                             for k, v in modes.items()}

        # ---- plain per-signal GPU form on a sample ---------------------------------------------
        from paper_1711_11407_gb300._lib import ERR_UNSUPPORTED, FpssftError
        from paper_1711_11407_gb300.plain import PlainRecoverer
        sample = stratified(wl, args.plain_sample, seed=2)
        pr = PlainRecoverer(p, dev)
        try:
            pr.recover(wl, cubes, alpha, tau, sample[:4])       # warm-up (plans, cuFFT)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = pr.recover(wl, cubes, alpha, tau, sample)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            agree = all(np.array_equal(k, ks[b, :cnt[b]]) for (k, _, _, _), b in zip(res, sample))
            plain_rate = len(sample) / dt
            line["plain_gpu"] = {"value": plain_rate, "unit": UNIT,
                                 "sample": f"{len(sample)} signals stratified by shape",
                                 "same_support_as_batched": agree, "batched_over_plain": value / world / plain_rate}
        except FpssftError as e:
            if e.status != ERR_UNSUPPORTED:
                raise
            line["plain_gpu"] = {"unavailable": f"the unfused per-signal form cannot run this workload: {e}"}

        # ---- FP64 oracle on the host cores (rank 0) --------------------------------------------
        if rank == 0:
            order = stratified(wl, wl.batch, seed=3)
            rate, n, dt, cores = oracle_rate(wl, p, args.cpu_seconds, order)
            rep = " (the workload's signals repeated, one core each)" if wl.batch < len(os.sched_getaffinity(0)) else ""
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": f"{n} signals stratified by shape{rep}, {dt:.1f} s wall on {cores} cores "
                                              "(numpy FP64, one spawned process per core)",
                                    "host_cores_available": len(os.sched_getaffinity(0))}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
