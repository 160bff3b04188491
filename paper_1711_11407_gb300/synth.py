"""Seeded synthetic inputs for FPS-SFT: planted sparse spectra, their cubes, noise and line schedules.

This module is the only code shared by the CUDA path and the FP64 oracle.  It draws random numbers
and evaluates the signal model; it performs none of the recovery method's arithmetic (no line
sampling, no line DFT, no projection, no decoding).

Signal model (Sec. 2, Eq. sigModel2, generalised to D dimensions in Sec. 2.3 "Multi-dimensional
extension"): x(n) = sum_k a_k exp(j 2 pi sum_d k_d n_d / N_d), with K on-grid frequencies k and
complex amplitudes a_k != 0.  The cube is stored C-order (last dimension fastest).

Line schedule (Sec. 2.2 and Sec. 2.3): every iteration draws a slope alpha and an offset tau in
X_D = [N_0] x ... x [N_{D-1}].  Slopes are drawn uniformly and rejected until the projection
k -> [sum_d (L/N_d) alpha_d k_d]_L is onto Z_L (every bin receives N/L frequencies, the property
Lemma 2 proves for its set A in 2-D); the optional policy "lemma2" draws from A itself, and
"axis" uses the unit slopes e_0, e_1, ... in turn (the rows and columns of the row/column SFT the
paper compares against, Sec. 2.1).  The schedule is an input of the method: both implementations
receive the same integers.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload",
    "draw_frequencies",
    "draw_amplitudes",
    "synthesize_cube",
    "add_awgn",
    "draw_schedule",
    "make_signal",
    "make_workload",
    "WORKLOADS",
]


def _line_length(dims):
    """LCM of the dimensions and the per-dimension factors L/N_d (needed to test slope admissibility)."""
    L = 1
    for n in dims:
        L = L * int(n) // math.gcd(L, int(n))
    return L, [L // int(n) for n in dims]


def _admissible(alpha, dims, policy):
    L, c = _line_length(dims)
    if policy == "uniform":
        g = L
        for cd, ad in zip(c, alpha):
            g = math.gcd(g, cd * int(ad))
        return g == 1
    if policy == "lemma2":
        if len(dims) != 2:
            raise ValueError("the slope set A of Lemma 2 is stated for D = 2 only")
        a0, a1 = int(alpha[0]), int(alpha[1])
        return math.gcd(a0, a1) == 1 and math.gcd(a0, c[1]) == 1 and math.gcd(a1, c[0]) == 1
    if policy == "any":
        return True
    raise ValueError(f"unknown slope policy {policy!r}")


def draw_schedule(rng, dims, T, policy="uniform"):
    """T slopes and offsets for one signal: int32 arrays alpha[T][D], tau[T][D]."""
    dims = [int(n) for n in dims]
    D = len(dims)
    alpha = np.zeros((T, D), np.int32)
    tau = np.zeros((T, D), np.int32)
    for t in range(T):
        if policy == "axis":        # rows and columns in turn: the axis lines of the row/column SFT
            a = [1 if d == t % D else 0 for d in range(D)]
        else:
            for _ in range(100000):
                a = [int(rng.integers(0, n)) for n in dims]
                if _admissible(a, dims, policy):
                    break
            else:  # pragma: no cover - only reachable for degenerate policies
                raise RuntimeError(f"no admissible slope found for dims {dims}")
        alpha[t] = a
        tau[t] = [int(rng.integers(0, n)) for n in dims]
    return alpha, tau


def draw_frequencies(rng, dims, K, clusters=0, sigma=0.0, block=0):
    """K distinct on-grid frequencies k[K][D] (int64).

    clusters == 0 and block == 0: uniform over the grid without replacement.
    clusters > 0: Gaussian blobs of standard deviation sigma (bins) around uniform centres,
    wrapped modulo N_d; duplicates are rejected and redrawn.
    block = b > 0: K // b^D non-overlapping contiguous b x ... x b blocks at uniform positions
    (wrapped), plus K mod b^D uniform singletons (the paper's clusters of 9 and 25 frequencies).
    """
    dims = np.asarray(dims, np.int64)
    N = int(np.prod(dims))
    if K > N:
        raise ValueError("K exceeds the grid size")
    if block > 0:
        D = len(dims)
        offs = np.stack(np.meshgrid(*[np.arange(block)] * D, indexing="ij"), -1).reshape(-1, D)
        taken = set()
        out = []
        nblk = K // len(offs)
        while len(out) < nblk * len(offs):
            corner = np.asarray([rng.integers(0, n) for n in dims], np.int64)
            cells = [tuple(int(v) for v in np.mod(corner + o, dims)) for o in offs]
            if any(c in taken for c in cells):
                continue
            taken.update(cells)
            out.extend(cells)
        while len(out) < K:
            c = tuple(int(rng.integers(0, n)) for n in dims)
            if c not in taken:
                taken.add(c)
                out.append(c)
        return np.asarray(out, np.int64)
    if clusters <= 0:
        lin = rng.choice(N, size=K, replace=False)
        return np.stack(np.unravel_index(lin, tuple(dims)), axis=1).astype(np.int64)
    centres = np.stack([rng.integers(0, n, size=clusters) for n in dims], axis=1)
    seen = set()
    out = []
    while len(out) < K:
        c = centres[rng.integers(0, clusters)]
        k = np.mod(np.rint(c + rng.normal(0.0, sigma, size=len(dims))).astype(np.int64), dims)
        key = tuple(int(v) for v in k)
        if key in seen:
            continue
        seen.add(key)
        out.append(key)
    return np.asarray(out, np.int64)


def draw_amplitudes(rng, K, mode="unit"):
    """Complex amplitudes with uniform phase.  mode: 'unit' (|a| = 1), 'uniform' (|a| ~ U[0.5, 1.5]),
    'lognormal' (|a| = exp(N(0, 0.5^2))), 'uniform_real' (real, U[0.5, 1.5])."""
    phase = rng.uniform(0.0, 2.0 * np.pi, size=K)
    if mode == "unit":
        mag = np.ones(K)
    elif mode == "uniform":
        mag = rng.uniform(0.5, 1.5, size=K)
    elif mode == "lognormal":
        mag = np.exp(rng.normal(0.0, 0.5, size=K))
    elif mode == "uniform_real":     # positive real intensities U[0.5, 1.5] (pixels of an image)
        return rng.uniform(0.5, 1.5, size=K) + 0j
    else:
        raise ValueError(f"unknown amplitude mode {mode!r}")
    return mag * np.exp(1j * phase)


def synthesize_cube(dims, k, a):
    """x(n) = sum_i a_i exp(j 2 pi sum_d k_{i,d} n_d / N_d) on the full grid, complex128.

    Evaluated as N times the inverse D-D FFT of the planted spectrum, which is the signal model
    summed exactly (up to rounding)."""
    dims = tuple(int(n) for n in dims)
    spec = np.zeros(dims, np.complex128)
    np.add.at(spec, tuple(np.asarray(k).T), a)
    return np.fft.ifftn(spec) * float(np.prod(dims))


def add_awgn(rng, x, snr_db, a=None, mode="total"):
    """Circular complex Gaussian noise.  mode 'total': sigma^2 = sum|a|^2 / 10^(snr/10) (per-sample SNR);
    'per_sinusoid': sigma^2 = mean|a|^2 / 10^(snr/10).  Returns (noisy cube, sigma)."""
    if snr_db is None:
        return x, 0.0
    p = np.sum(np.abs(a) ** 2) if mode == "total" else np.mean(np.abs(a) ** 2)
    sigma = math.sqrt(p / 10.0 ** (snr_db / 10.0))
    noise = (rng.normal(size=x.shape) + 1j * rng.normal(size=x.shape)) * (sigma / math.sqrt(2.0))
    return x + noise, sigma


@dataclass
class Workload:
    """A batch of synthetic signals.  cubes holds every cube concatenated (complex64, C order) at
    element offsets `offsets`; alpha/tau are int32 [batch][T_max][D]; k_true/a_true list the planted
    spectra; T per signal is the iteration budget."""

    name: str
    D: int
    dims: np.ndarray            # int64 [batch][D]
    offsets: np.ndarray         # int64 [batch]
    cubes: np.ndarray           # complex64 [sum N]
    alpha: np.ndarray           # int32 [batch][T_max][D]
    tau: np.ndarray             # int32 [batch][T_max][D]
    T: np.ndarray               # int32 [batch]
    k_true: list = field(default_factory=list)
    a_true: list = field(default_factory=list)
    sigma: np.ndarray = None    # noise standard deviation per signal (0 when noiseless)
    noiseless: bool = True

    @property
    def batch(self):
        return int(self.dims.shape[0])

    def cube(self, i, dtype=np.complex128):
        n = int(np.prod(self.dims[i]))
        o = int(self.offsets[i])
        return self.cubes[o:o + n].reshape(tuple(int(v) for v in self.dims[i])).astype(dtype)

    def subset(self, idx):
        idx = [int(i) for i in idx]
        sizes = [int(np.prod(self.dims[i])) for i in idx]
        offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        cubes = np.concatenate([self.cubes[int(self.offsets[i]):int(self.offsets[i]) + s]
                                for i, s in zip(idx, sizes)]) if idx else np.zeros(0, np.complex64)
        Tm = int(max(self.T[i] for i in idx)) if idx else 1
        return Workload(self.name + "[subset]", self.D, self.dims[idx].copy(), offs, cubes,
                        self.alpha[idx, :Tm].copy(), self.tau[idx, :Tm].copy(), self.T[idx].copy(),
                        [self.k_true[i] for i in idx], [self.a_true[i] for i in idx],
                        None if self.sigma is None else self.sigma[idx].copy(), self.noiseless)


def make_signal(seed_seq, dims, K, T, *, clusters=0, sigma_bins=0.0, block=0, amp="unit", snr_db=None,
                snr_mode="total", policy="uniform"):
    """One signal: planted (k, a), its cube (complex128), the noise sigma and a T-row schedule.
    Draw order from the signal's own stream: frequencies, amplitudes, noise, schedule."""
    rng = np.random.Generator(np.random.PCG64(seed_seq))
    k = draw_frequencies(rng, dims, K, clusters, sigma_bins, block)
    a = draw_amplitudes(rng, K, amp)
    x = synthesize_cube(dims, k, a)
    x, sig = add_awgn(rng, x, snr_db, a, snr_mode)
    alpha, tau = draw_schedule(rng, dims, T, policy)
    return k, a, x, sig, alpha, tau


def _budget(dims):
    """Iterations that together read about every sample once: N / ((D+1) L) (Sec. 3, T_max = N/(3L))."""
    N = int(np.prod(dims))
    L, _ = _line_length(dims)
    return max(1, N // ((len(dims) + 1) * L))


# Workload recipes.  Shapes, sparsities and value distributions follow the workloads the paper
# simulates (Sec. 3) and the five benchmark configurations of this library.
WORKLOADS = {
    "single_128x128": dict(shapes=[(128, 128)], batch=1, K=lambda N: 20, T=lambda d: 10, amp="unit"),
    "single_240x256": dict(shapes=[(240, 256)], batch=1, K=lambda N: 300, T=lambda d: 12, amp="uniform",
                           clusters=4, sigma_bins=6.0),
    "batched_64x64x64": dict(shapes=[(64, 64, 64)], batch=256, K=lambda N: 500, T=_budget, amp="unit",
                             snr_db=10.0),
    "uneven_2d": dict(shapes=[(64, 64), (128, 128), (128, 256), (256, 256)], batch=4096,
                      K=lambda N: -(-N // 200), T=_budget, amp="unit"),
    "images_1024x1024": dict(shapes=[(1024, 1024)], batch=64, K=lambda N: 2000, T=_budget, amp="lognormal",
                             clusters=20, sigma_bins=10.0, snr_db=5.0),
    # a sparse image of the size of the paper's Fig. 3 (512 x 576, L = LCM = 4608): blobs of
    # non-zero "pixels" (frequencies) with positive intensities
    "sparse_image_512x576": dict(shapes=[(512, 576)], batch=8, K=lambda N: 8411, T=_budget, amp="uniform_real",
                                 clusters=60, sigma_bins=12.0),
    # the noisy workloads with the SNR read per sinusoid (sigma^2 = mean |a|^2 / 10^(snr/10))
    "batched_64x64x64_ps": dict(shapes=[(64, 64, 64)], batch=256, K=lambda N: 500, T=_budget, amp="unit",
                                snr_db=10.0, snr_mode="per_sinusoid"),
    "images_1024x1024_ps": dict(shapes=[(1024, 1024)], batch=64, K=lambda N: 2000, T=_budget, amp="lognormal",
                                clusters=20, sigma_bins=10.0, snr_db=5.0, snr_mode="per_sinusoid"),
}
WORKLOAD_IDS = {1: "single_128x128", 2: "single_240x256", 3: "batched_64x64x64", 4: "uneven_2d",
                5: "images_1024x1024", 6: "sparse_image_512x576", 13: "batched_64x64x64_ps",
                15: "images_1024x1024_ps"}


def make_workload(name, seed=None, batch=None, *, shapes=None, K=None, T=None, snr_db="default",
                  policy="uniform", indices=None):
    """Build a named workload (or a variant of it).  `batch` overrides the signal count; `indices`
    keeps only those signals (each signal has its own seed stream, so a subset costs only its own
    generation).  Seeds default to 1234 + workload id."""
    spec = dict(WORKLOADS[name])
    if seed is None:
        seed = 1234 + {v: k for k, v in WORKLOAD_IDS.items()}[name]
    nb = int(batch if batch is not None else spec["batch"])
    shp = shapes if shapes is not None else spec["shapes"]
    top = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), 0])))
    size_idx = top.integers(0, len(shp), size=nb) if len(shp) > 1 else np.zeros(nb, np.int64)
    dims_all = np.asarray([shp[int(i)] for i in size_idx], np.int64)
    children = np.random.SeedSequence([int(seed), 1]).spawn(nb)
    sel = list(range(nb)) if indices is None else [int(i) for i in indices]
    snr = spec.get("snr_db") if snr_db == "default" else snr_db
    Kf = K if K is not None else spec["K"]
    Tf = T if T is not None else spec["T"]
    Ts = [int(Tf(tuple(dims_all[i]))) if callable(Tf) else int(Tf) for i in sel]
    Tmax = max(Ts) if sel else 1
    D = dims_all.shape[1]
    alpha = np.zeros((len(sel), Tmax, D), np.int32)
    tau = np.zeros((len(sel), Tmax, D), np.int32)
    pieces, ks, as_, sigs = [], [], [], []
    for j, i in enumerate(sel):
        dims = tuple(int(v) for v in dims_all[i])
        N = int(np.prod(dims))
        Ki = int(Kf(N)) if callable(Kf) else int(Kf)
        k, a, x, sg, al, ta = make_signal(children[i], dims, Ki, Ts[j], clusters=spec.get("clusters", 0),
                                          sigma_bins=spec.get("sigma_bins", 0.0), amp=spec["amp"],
                                          snr_db=snr, snr_mode=spec.get("snr_mode", "total"), policy=policy)
        alpha[j, :Ts[j]] = al
        tau[j, :Ts[j]] = ta
        pieces.append(x.reshape(-1).astype(np.complex64))
        ks.append(k)
        as_.append(a)
        sigs.append(sg)
    sizes = [p.size for p in pieces]
    offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64) if sel else np.zeros(0, np.int64)
    cubes = np.concatenate(pieces) if pieces else np.zeros(0, np.complex64)
    return Workload(name, D, dims_all[sel].copy(), offsets, cubes, alpha, tau, np.asarray(Ts, np.int32),
                    ks, as_, np.asarray(sigs), snr is None)
