"""Fig. 2 of the paper (FPS-SFT half) on the GPU: perfect-recovery probability and percentage of
samples used versus the number of sinusoids K, on a 256 x 256 grid, for uniformly distributed
frequencies and for clusters of 9 and 25 frequencies, T_max = N / (3L) = 85, 100 trials per point.

Each point's trials are one batched fpssft_recover launch.  A trial succeeds when the recovered
support equals the planted one exactly and every amplitude is within 1e-3 of the planted value.
Samples are counted up to the iteration that completed the set: with the early stop, the last
iteration only confirms that nothing is left, so (iterations - 1) * 3L / N.

    python -m paper_1711_11407_gb300.fig2 [trials]
"""
from __future__ import annotations

import json
import sys
import time

import numpy as np
import torch

from . import synth
from .api import Params, Plan

N0 = 256
T_MAX = (N0 * N0) // (3 * N0)


def run_point(K, block=0, trials=100, seed=0, device="cuda"):
    dims = (N0, N0)
    pieces, ks, as_, al, ta = [], [], [], [], []
    for t in range(trials):
        k, a, x, _, alpha, tau = synth.make_signal(np.random.SeedSequence([seed, K, block, t]), dims, K, T_MAX,
                                                   block=block)
        pieces.append(x.reshape(-1).astype(np.complex64))
        ks.append(k)
        as_.append(a)
        al.append(alpha)
        ta.append(tau)
    dev = torch.device(device)
    cubes = torch.from_numpy(np.concatenate(pieces)).to(dev)
    offs = torch.from_numpy(np.arange(trials, dtype=np.int64) * (N0 * N0)).to(dev)
    alpha = torch.from_numpy(np.stack(al)).to(dev)
    tau = torch.from_numpy(np.stack(ta)).to(dev)
    plan = Plan(np.tile(np.array(dims, np.int64), (trials, 1)),
                Params(T=T_MAX, k_cap=2 * K + 64, theta0=1e-3, rho=1e-3, eta=0.05, early_stop=True))
    t0 = time.perf_counter()
    out = plan.recover(cubes, offs, alpha, tau)
    torch.cuda.synchronize()
    gpu_s = time.perf_counter() - t0
    kk, aa, cnt, it = out.k.cpu().numpy(), out.a.cpu().numpy(), out.count.cpu().numpy(), out.iters.cpu().numpy()
    ok, pct = [], []
    for t in range(trials):
        lin_true = ks[t][:, 0] * N0 + ks[t][:, 1]
        order = np.argsort(lin_true)
        n = int(cnt[t])
        lin = kk[t, :n, 0].astype(np.int64) * N0 + kk[t, :n, 1]
        good = n == K and np.array_equal(lin, lin_true[order]) and \
            np.allclose(aa[t, :n], as_[t][order], atol=1e-3, rtol=0)
        ok.append(good)
        if good:
            pct.append((int(it[t]) - 1) * 3 * N0 / (N0 * N0) * 100.0)
    plan.close()
    return {"K": K, "K_over_N0": K / N0, "cluster": block * block if block else 1, "trials": trials,
            "success": float(np.mean(ok)), "samples_pct": float(np.mean(pct)) if pct else None,
            "per_trial_success": [bool(v) for v in ok], "iters": [int(v) for v in it], "gpu_seconds": gpu_s}


def main(trials=100):
    rows = []
    for block in (0, 3, 5):
        for mult in (0.5, 1, 2, 3, 4, 5, 6):
            K = int(mult * N0)
            if block:
                K -= K % (block * block)
            r = run_point(K, block, trials)
            r.pop("per_trial_success")
            r.pop("iters")
            rows.append(r)
            print(json.dumps(r), flush=True)
    return rows


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 100)
