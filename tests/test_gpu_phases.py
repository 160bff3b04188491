"""The phase-timer build (tracing): on each recovery kernel it recovers the same sets as the plain
library and accounts for every CTA, iteration and cycle of the timed launches."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_1711_11407_gb300 import configs, synth
from paper_1711_11407_gb300.api import Plan

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu


def _plain(workload, batch, fft_path):
    wl = synth.make_workload(workload, batch=batch)
    plan = Plan(wl.dims, configs.params_for(wl, fft_path=fft_path))
    dev = torch.device("cuda")
    out = plan.recover(*(torch.from_numpy(v).to(dev) for v in (wl.cubes, wl.offsets, wl.alpha, wl.tau)))
    torch.cuda.synchronize()
    res = {f: getattr(out, f).cpu().numpy() for f in ("k", "a", "count", "iters", "status")}
    grid = plan.info["grid"]
    plan.close()
    return res, grid


@pytest.mark.parametrize("workload,batch,fft_path", [
    ("uneven_2d", 64, 2),           # register path, persistent CTAs over 64 signals
    ("single_128x128", None, 1),    # one CTA per signal
    ("single_240x256", None, 3),    # cluster path: three CTAs exchange bins
])
def test_phase_timer_build_matches_plain_and_accounts_for_the_launch(tmp_path, workload, batch, fft_path):
    reps = 3
    dump = str(tmp_path / "out.npz")
    cmd = [sys.executable, "-m", "paper_1711_11407_gb300.phases", "--workload", workload, "--reps", str(reps),
           "--fft-path", str(fft_path), "--dump", dump]
    if batch is not None:
        cmd += ["--batch", str(batch)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    s = json.loads(r.stdout.strip().splitlines()[-1])
    plain, grid = _plain(workload, batch, fft_path)
    timed = np.load(dump)
    for f in ("count", "iters", "status"):
        assert np.array_equal(timed[f], plain[f]), f
    # identical support; amplitudes within FP32 rounding: the peel subtracts the contributions of
    # entries that share a bin with shared-memory atomics, in an order the timing decides
    for b in range(len(plain["count"])):
        n = int(plain["count"][b])
        assert np.array_equal(timed["k"][b, :n], plain["k"][b, :n])
        assert np.allclose(timed["a"][b, :n], plain["a"][b, :n], rtol=1e-5, atol=1e-6)
    assert s["plan"]["fft_path"] == fft_path
    assert s["ctas"] == reps * grid
    # every CTA of the cluster path runs the signal's iterations; the other paths sum over signals
    per_launch_iters = s["iterations_per_cta"] * grid
    expect = plain["iters"].sum() * (3 if fft_path == 3 else 1)
    assert per_launch_iters == pytest.approx(expect)
    ph = s["phase_us_per_cta"]
    assert all(v >= 0 for k, v in ph.items() if k != "unmarked")
    assert ph["unmarked"] >= -1e-6 and sum(ph.values()) == pytest.approx(s["cta_us"])
    assert ph["fft"] > 0 and ph["decode"] > 0 and ph["output"] > 0
    assert (ph["exchange"] > 0) == (fft_path == 3)
    assert 500 < s["sm_clock_mhz"] < 3000
