"""Thresholds of the 1-sparsity test for the workloads (no GPU): the noisy T0 threshold rests on the
standard deviation of a pure-noise bin after the 1/L line DFT (Eq. hs), sigma / sqrt(L)."""
import math

import numpy as np
import pytest

from paper_1711_11407_gb300 import configs, synth as S


def test_a_pure_noise_bin_has_standard_deviation_sigma_over_sqrt_l():
    rng = np.random.default_rng(4)
    L, sigma, n = 256, 0.7, 4000
    noise = (rng.normal(size=(n, L)) + 1j * rng.normal(size=(n, L))) * (sigma / math.sqrt(2.0))
    bins = np.fft.fft(noise, axis=-1) / L                 # Eq. hs, by the same definition the pins fix
    assert np.std(bins) == pytest.approx(sigma / math.sqrt(L), rel=0.01)


def test_workload_thresholds():
    quiet = S.make_workload("uneven_2d", batch=4)
    assert configs.threshold_values(quiet) == (1e-3, 1e-3, 0.05)
    noisy = S.make_workload("images_1024x1024", batch=2)
    th0, rho, eta = configs.threshold_values(noisy)
    L = math.lcm(*[int(v) for v in noisy.dims[0]])
    assert th0 == pytest.approx(4.0 * float(np.mean(noisy.sigma)) / math.sqrt(L))
    assert (rho, eta) == (0.25, 0.25)
    p = configs.params_for(noisy, T=3)
    assert p.T == 3 and p.theta0 == pytest.approx(th0) and p.early_stop
