"""Recovery parameters for the synthetic workloads (thresholds of the 1-sparsity test).

Noiseless workloads: theta0 = 1e-3 absolute (planted |a| >= 0.5; FP32 residuals after peeling are
~1e-6), rho = 1e-3, eta = 0.05.  Noisy workloads: a bin of pure noise has standard deviation
sigma / sqrt(L) (the 1/L DFT of L samples of variance sigma^2), so theta0 = 4 sigma / sqrt(L);
rho = eta = 0.25.

Stop rule: early_stop = 2, a signal stops after an iteration in which no line-0 bin passes T0 or
every line-0 bin passing T0 was decoded (the library's default, 1, waits for an iteration that
finds nothing, one more on noiseless data).
"""
from __future__ import annotations

import math

import numpy as np

NOISELESS = dict(theta0=1e-3, rho=1e-3, eta=0.05)
NOISY = dict(rho=0.25, eta=0.25)

# iteration budget (T = 0: N / ((D+1) L) per signal) and recovered-set capacity
BUDGET = {
    "single_128x128": dict(T=10, k_cap=64),
    "single_240x256": dict(T=12, k_cap=640),
    "batched_64x64x64": dict(T=0, k_cap=1024),
    "uneven_2d": dict(T=0, k_cap=512),
    "images_1024x1024": dict(T=0, k_cap=4096),
    "sparse_image_512x576": dict(T=0, k_cap=20000),
    "batched_64x64x64_ps": dict(T=0, k_cap=1024),
    "images_1024x1024_ps": dict(T=0, k_cap=4096),
}


def threshold_values(wl):
    """(theta0, rho, eta) for a workload (noisy workloads use the mean noise level of the batch)."""
    if wl.noiseless:
        return NOISELESS["theta0"], NOISELESS["rho"], NOISELESS["eta"]
    L = math.lcm(*[int(v) for v in wl.dims[0]])
    sigma = float(np.mean(wl.sigma))
    return 4.0 * sigma / math.sqrt(L), NOISY["rho"], NOISY["eta"]


def params_for(wl, **over):
    """Params for the library (paper_1711_11407_gb300.api.Params)."""
    from .api import Params
    th0, rho, eta = threshold_values(wl)
    base = BUDGET.get(wl.name.split("[")[0], dict(T=0, k_cap=1024))
    kw = dict(T=base["T"], k_cap=base["k_cap"], theta0=th0, rho=rho, eta=eta, early_stop=2)
    kw.update(over)
    return Params(**kw)
