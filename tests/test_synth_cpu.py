"""The seeded input generator both implementations read (no GPU): the cube is the signal model of
Sec. 2 / Sec. 2.3, slopes give every bin N/L frequencies, frequencies are distinct and on the grid,
noise has the stated SNR, and workloads are reproducible signal by signal."""
import math

import numpy as np
import pytest

from paper_1711_11407_gb300 import synth as S


def test_cube_is_the_signal_model_summed_term_by_term():
    rng = np.random.default_rng(3)
    for dims in [(6, 10), (4, 6, 3), (7,)]:
        k = S.draw_frequencies(rng, dims, 5)
        a = S.draw_amplitudes(rng, 5, "uniform")
        x = S.synthesize_cube(dims, k, a)
        grid = np.stack(np.meshgrid(*[np.arange(n) for n in dims], indexing="ij"), -1)
        ref = np.zeros(dims, np.complex128)
        for kk, aa in zip(k, a):
            ph = sum(kk[d] * grid[..., d] / dims[d] for d in range(len(dims)))
            ref += aa * np.exp(2j * np.pi * ph)
        assert np.allclose(x, ref, atol=1e-12)


@pytest.mark.parametrize("dims", [(8, 12), (6, 10), (4, 6, 3), (9,), (5, 7)])
def test_uniform_slopes_give_every_bin_n_over_l_frequencies(dims):
    """Counted by brute force over the grid, independently of the gcd test the sampler uses."""
    rng = np.random.default_rng(11)
    alpha, tau = S.draw_schedule(rng, dims, 30)
    N = int(np.prod(dims))
    L = math.lcm(*dims)
    grid = np.stack(np.meshgrid(*[np.arange(n) for n in dims], indexing="ij"), -1).reshape(-1, len(dims))
    for al, ta in zip(alpha, tau):
        assert all(0 <= al[d] < dims[d] and 0 <= ta[d] < dims[d] for d in range(len(dims)))
        m = sum((L // dims[d]) * int(al[d]) * grid[:, d] for d in range(len(dims))) % L
        assert np.array_equal(np.bincount(m, minlength=L), np.full(L, N // L)), (dims, al)


def test_lemma2_and_axis_policies():
    rng = np.random.default_rng(5)
    dims = (8, 12)
    L = math.lcm(*dims)
    c = (L // dims[0], L // dims[1])
    alpha, _ = S.draw_schedule(rng, dims, 40, policy="lemma2")
    for a0, a1 in alpha:
        assert math.gcd(a0, a1) == 1 and math.gcd(a0, c[1]) == 1 and math.gcd(a1, c[0]) == 1
    alpha, _ = S.draw_schedule(rng, dims, 6, policy="axis")
    assert [tuple(a) for a in alpha] == [(1, 0), (0, 1)] * 3
    with pytest.raises(ValueError):
        S.draw_schedule(rng, (4, 4, 4), 1, policy="lemma2")


def test_frequencies_are_distinct_on_grid_and_blocks_are_contiguous():
    rng = np.random.default_rng(9)
    dims = (32, 48)
    for kw in ({}, {"clusters": 3, "sigma": 2.0}, {"block": 3}):
        k = S.draw_frequencies(rng, dims, 40, **kw)
        assert k.shape == (40, 2)
        assert len({tuple(v) for v in k}) == 40
        assert np.all((k >= 0) & (k < np.asarray(dims)))
    k = S.draw_frequencies(rng, dims, 9 * 4 + 2, block=3)
    for i in range(4):                       # each block of 9 is a 3 x 3 square (modulo the grid)
        b = k[9 * i:9 * i + 9]
        d0 = np.mod(b - b[0], dims)
        assert sorted(map(tuple, d0)) == [(u, v) for u in range(3) for v in range(3)]
    with pytest.raises(ValueError):
        S.draw_frequencies(rng, (2, 2), 5)


def test_noise_has_the_stated_snr():
    rng = np.random.default_rng(2)
    dims = (256, 256)
    k = S.draw_frequencies(rng, dims, 50)
    a = S.draw_amplitudes(rng, 50, "lognormal")
    x = S.synthesize_cube(dims, k, a)
    for mode, power in (("total", np.sum(np.abs(a) ** 2)), ("per_sinusoid", np.mean(np.abs(a) ** 2))):
        y, sigma = S.add_awgn(rng, x, 10.0, a, mode)
        assert sigma == pytest.approx(math.sqrt(power / 10.0))
        noise = y - x
        assert np.var(noise.real) == pytest.approx(sigma ** 2 / 2, rel=0.02)
        assert np.var(noise.imag) == pytest.approx(sigma ** 2 / 2, rel=0.02)
    assert S.add_awgn(rng, x, None, a) == (x, 0.0)


def test_workloads_are_reproducible_and_signals_independent_of_the_batch_subset():
    w1 = S.make_workload("uneven_2d", batch=12)
    w2 = S.make_workload("uneven_2d", batch=12)
    assert np.array_equal(w1.cubes, w2.cubes) and np.array_equal(w1.alpha, w2.alpha)
    sub = S.make_workload("uneven_2d", batch=12, indices=[3, 7])
    for j, i in enumerate((3, 7)):
        assert np.array_equal(sub.cube(j), w1.cube(i))
        assert np.array_equal(sub.alpha[j, :sub.T[j]], w1.alpha[i, :w1.T[i]])
        assert np.array_equal(sub.k_true[j], w1.k_true[i])
    # the uneven recipe: shapes from the set, K = ceil(N / 200), T = N / (3 L)
    shapes = {(64, 64), (128, 128), (128, 256), (256, 256)}
    for b in range(w1.batch):
        dims = tuple(int(v) for v in w1.dims[b])
        N, L = int(np.prod(dims)), math.lcm(*dims)
        assert dims in shapes
        assert len(w1.k_true[b]) == math.ceil(N / 200)
        assert int(w1.T[b]) == N // (3 * L)
        assert w1.cubes.dtype == np.complex64 and int(w1.offsets[b]) + N <= w1.cubes.size
