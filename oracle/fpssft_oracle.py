"""FP64 CPU oracle of the FPS-SFT recovery loop.

Paper: S. Wang, V. M. Patel, A. Petropulu, "FPS-SFT: A Multi-dimensional Sparse Fourier Transform
Based on the Fourier Projection-slice Theorem", arXiv 1711.11407 (ICASSP 2018).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference the CUDA library is checked
against.  Only the test suite, the smoke check and the CPU-baseline leg of the benchmark may import
it; the library itself never does, and this module imports nothing from the library.  Everything is
numpy in float64 / complex128; the one library primitive used as a step is numpy's FFT for the
L-point line DFT (pinned by the tests against a brute-force DFT and against the dense D-D DFT).

Notation follows the paper: dims N_d, d = 0..D-1; N = prod N_d; L = LCM(N_d) (Lemma 1);
c_d = L / N_d; slope alpha and offset tau in X_D = [N_0] x ... x [N_{D-1}]; lines j = 0..D where
line 0 starts at tau and line d+1 at tau + e_d (mod N_d) (Sec. 2.3, read as D+1 lines);
W = exp(j 2 pi / L).

Readings of points the paper leaves open (each one is stated where it is used):
  * the 1-sparsity test (Sec. 2.2 says only that a non-zero bin is 1-sparse with high probability;
    Sec. 2.1 tests 1-sparsity by equal magnitudes): tests T0..T3 in `classify_decode`;
  * rounding in the decode (Eq. decoding gives [.]_{N_d} without a rounding rule): floor(u + 1/2);
  * construction-subtraction (Sec. 2.2) done on the bins (identical by linearity of the DFT);
    the literal IDFT-subtract-DFT order is kept as `peel_mode="literal"`;
  * a frequency decoded again accumulates its amplitude; entries with |a| <= theta0 are dropped at
    output; the output is sorted by linear frequency index;
  * optional early stop (the paper runs T iterations): either when no bin of line 0 passes T0
    after peeling (the iteration that finds nothing is counted), or already after an iteration in
    which every line-0 bin passing T0 was decoded (what was left on the line is now recovered);
  * optional amplitude averaged over the D+1 phase-corrected lines (`decoded_amplitude`);
  * a full set (k_cap entries) drops new frequencies, flags the signal and stops it.

Every function here is pinned by tests/pins.py against the paper's closed forms, brute force or
printed values.  Parity unpinned: the outcome on noisy inputs, which the paper does not model; on
those the CUDA path is compared with this oracle one iteration at a time from the same set, and
over whole runs signal by signal.  Beyond the loop: FP64 least-squares amplitudes over many lines
(`refine_lstsq`, the counterpart of the library's refinement) and several offset sets per slope
(`recover_offset_sets`), both pinned the same way.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

STATUS_OK = 0
STATUS_CAPACITY = 4

TWO_PI = 2.0 * math.pi


@dataclass
class Params:
    """Thresholds and loop controls of the recovery (defaults are the noiseless reading)."""

    T: int = 10                 # iterations (Sec. 2.2, "after T iterations")
    k_cap: int = 1024           # capacity of the recovered set
    theta0: float = 1e-3        # T0: |s_0(m)| > theta0
    rho: float = 1e-3           # T1: ||s_{d+1}(m)| - |s_0(m)|| <= rho |s_0(m)|
    eta: float = 0.05           # T2: |N_d phi / (2 pi) - round| <= eta
    early_stop: int = 1         # 0: run T iterations; 1: stop when no bin of line 0 passes T0 after
                                # peeling; 2: also stop after an iteration whose line-0 bins passing
                                # T0 were all decoded
    peel_mode: str = "bins"     # "bins" (subtract projections from the bins) or "literal"
    amp_average: bool = False   # amplitude from line tau only (Eq. decoding) or averaged over the D+1 lines


# ---------------------------------------------------------------------------------------------
# Line design: Lemma 1 (length) and Lemma 2 (slopes)
# ---------------------------------------------------------------------------------------------

def line_length(dims):
    """Lemma 1: the line length is L = LCM(N_0, ..., N_{D-1}); returns (L, [c_d = L / N_d])."""
    L = 1
    for n in dims:
        n = int(n)
        L = L * n // math.gcd(L, n)
    return L, [L // int(n) for n in dims]


def uniform_projection(alpha, dims):
    """True when every bin m in [L] receives exactly N/L grid frequencies (the conclusion of Lemma 2).

    The bin map k -> [sum_d c_d alpha_d k_d]_L (Eq. orthogonality) is a group homomorphism from
    Z_{N_0} x ... x Z_{N_{D-1}} to Z_L; its image is generated by the c_d alpha_d, so it is onto
    (and then every fibre has N/L elements) exactly when gcd(L, c_0 alpha_0, ...) = 1."""
    L, c = line_length(dims)
    g = L
    for cd, ad in zip(c, alpha):
        g = math.gcd(g, cd * int(ad))
    return g == 1


def in_lemma2_set(alpha, dims):
    """Membership in the 2-D slope set A of Lemma 2: alpha_0 coprime alpha_1, alpha_0 coprime c_1,
    alpha_1 coprime c_0."""
    if len(dims) != 2:
        raise ValueError("Lemma 2 is stated for D = 2")
    _, c = line_length(dims)
    a0, a1 = int(alpha[0]), int(alpha[1])
    return math.gcd(a0, a1) == 1 and math.gcd(a0, c[1]) == 1 and math.gcd(a1, c[0]) == 1


# ---------------------------------------------------------------------------------------------
# Sampling along lines and the line DFT: Eq. sample_slice, Eq. hs, Sec. 2.3
# ---------------------------------------------------------------------------------------------

def line_points(dims, alpha, tau):
    """Grid points of the D+1 lines: n[j][l][d] = [alpha_d l + tau_d + delta_{j, d+1}]_{N_d}, l in [L].

    Eq. sample_slice gives line 0; Sec. 2.3 gives the offsets tau + e_d of the other lines (its
    index range is garbled; the reading used here is one extra line per dimension, D+1 lines)."""
    dims = [int(n) for n in dims]
    D = len(dims)
    L, _ = line_length(dims)
    l = np.arange(L, dtype=np.int64)
    pts = np.zeros((D + 1, L, D), np.int64)
    for j in range(D + 1):
        for d in range(D):
            shift = 1 if j == d + 1 else 0
            pts[j, :, d] = (int(alpha[d]) * l + int(tau[d]) + shift) % dims[d]
    return pts


def sample_lines(x, alpha, tau):
    """s_j(l) = x(n_j(l)) for the D+1 lines (Eq. sample_slice): complex128 [D+1][L]."""
    pts = line_points(x.shape, alpha, tau)
    return x[tuple(pts[..., d] for d in range(x.ndim))].astype(np.complex128)


def line_dft(s):
    """Eq. hs: s_hat(m) = (1/L) sum_l s(l) exp(-j 2 pi l m / L), along the last axis."""
    L = s.shape[-1]
    return np.fft.fft(s, axis=-1) / L


def line_idft(s_hat):
    """Inverse of `line_dft`: s(l) = sum_m s_hat(m) exp(+j 2 pi l m / L)."""
    L = s_hat.shape[-1]
    return np.fft.ifft(s_hat, axis=-1) * L


def project(x, alpha, tau):
    """The line-projection operator: D+1 line DFTs of the cube x at slope alpha, offset tau."""
    return line_dft(sample_lines(x, alpha, tau))


# ---------------------------------------------------------------------------------------------
# Where a frequency lands: Eq. orthogonality (proof of Lemma 1) and Eq. freqSum
# ---------------------------------------------------------------------------------------------

def bin_index(k, alpha, dims):
    """m(k) = [sum_d (L/N_d) alpha_d k_d]_L for k[..., D] (Eq. orthogonality)."""
    L, c = line_length(dims)
    k = np.asarray(k, np.int64)
    acc = np.zeros(k.shape[:-1], np.int64)
    for d in range(len(dims)):
        acc = acc + c[d] * int(alpha[d]) * k[..., d]
    return acc % L


def line_phase(k, tau, dims, j):
    """exp(j 2 pi sum_d k_d (tau_d + delta_{j, d+1}) / N_d): the factor Eq. freqSum attaches to a
    frequency k on line j.  The exponent is reduced exactly as the integer [sum_d c_d k_d t_d]_L."""
    L, c = line_length(dims)
    k = np.asarray(k, np.int64)
    q = np.zeros(k.shape[:-1], np.int64)
    for d in range(len(dims)):
        t = int(tau[d]) + (1 if j == d + 1 else 0)
        q = q + c[d] * k[..., d] * t
    q = q % L
    return np.exp(1j * TWO_PI * q / L)


def synth(k, a, alpha, tau, dims):
    """Line bins of a sparse spectrum {(k_i, a_i)} (Eq. freqSum): bins[j][m] = sum over i with
    m(k_i) = m of a_i * line_phase(k_i, tau, j).  This is the construction step of the
    construction-subtraction procedure (Sec. 2.2)."""
    dims = [int(n) for n in dims]
    D = len(dims)
    L, _ = line_length(dims)
    out = np.zeros((D + 1, L), np.complex128)
    k = np.asarray(k, np.int64).reshape(-1, D)
    a = np.asarray(a, np.complex128).reshape(-1)
    if k.shape[0] == 0:
        return out
    m = bin_index(k, alpha, dims)
    for j in range(D + 1):
        np.add.at(out[j], m, a * line_phase(k, tau, dims, j))
    return out


def peel_bins(bins, k, a, alpha, tau, dims):
    """Construction-subtraction done on the bins: bins - synth(recovered set)."""
    return bins - synth(k, a, alpha, tau, dims)


def peel_literal(samples, k, a, alpha, tau, dims):
    """Construction-subtraction as the paper orders it (Sec. 2.2): construct the bins of the
    recovered set, take their L-point IDFT and subtract the constructed line from the samples."""
    return samples - line_idft(synth(k, a, alpha, tau, dims))


# ---------------------------------------------------------------------------------------------
# 1-sparsity test and OFDM-trick decode: Sec. 2.1, Sec. 2.2, Eq. decoding
# ---------------------------------------------------------------------------------------------

def projects_to(m, k, alpha, dims):
    """T3: the decoded frequency k lies on bin m of the line with slope alpha (Eq. orthogonality).
    A bin that passed T0-T2 by accident (several frequencies) decodes to a k that lands on another
    bin with probability 1 - 1/L."""
    return int(bin_index(np.asarray(k), alpha, dims)) == int(m)


def decoded_amplitude(bins, m, k, tau, dims, average=False):
    """Eq. decoding: a = s_0(m) times the conjugate of line 0's offset phase.  With `average`
    (reading A12, for noisy data) the mean over the D+1 lines of s_j(m) times the conjugate of line
    j's offset phase: every line carries the same amplitude times its own phase (Eq. freqSum)."""
    kk = np.asarray(k)
    if not average:
        return complex(bins[0][m] * np.conj(line_phase(kk, tau, dims, 0)))
    n = len(dims) + 1
    return complex(sum(bins[j][m] * np.conj(line_phase(kk, tau, dims, j)) for j in range(n)) / n)


def classify_decode(bins, alpha, tau, dims, p):
    """Decode every bin that passes the 1-sparsity tests.

    For each m (in increasing order), with s_j = bins[j][m]:
      T0  |s_0| > theta0                                   (a non-zero bin, Sec. 2.2)
      T1  ||s_{d+1}| - |s_0|| <= rho |s_0| for every d      (equal magnitudes, Sec. 2.1)
      decode k_d = [floor(u_d + 1/2)]_{N_d}, u_d = N_d phi(s_{d+1} / s_0) / (2 pi)   (Eq. decoding)
      T2  |u_d - floor(u_d + 1/2)| <= eta for every d      (the phase sits on the frequency grid)
      T3  m(k) = m                                         (Eq. orthogonality)
      a = s_0 exp(-j 2 pi sum_d k_d tau_d / N_d)            (Eq. decoding)
    (with p.amp_average, a is the mean over the D+1 lines of s_j times the conjugate offset phase
    of line j, an option for noisy data).
    Returns (list of (m, k tuple, a), number of bins passing T0)."""
    dims = [int(n) for n in dims]
    D = len(dims)
    L = bins.shape[-1]
    s0 = bins[0]
    mag0 = np.abs(s0)
    t0 = mag0 > p.theta0
    out = []
    for m in np.nonzero(t0)[0]:
        ok = True
        for d in range(D):
            if abs(abs(bins[d + 1][m]) - mag0[m]) > p.rho * mag0[m]:
                ok = False
                break
        if not ok:
            continue
        k = []
        for d in range(D):
            phi = np.angle(bins[d + 1][m] / s0[m])          # phi in (-pi, pi]
            u = dims[d] * phi / TWO_PI
            r = math.floor(u + 0.5)
            if abs(u - r) > p.eta:
                ok = False
                break
            k.append(r % dims[d])
        if not ok:
            continue
        if not projects_to(m, k, alpha, dims):
            continue
        a = decoded_amplitude(bins, m, k, tau, dims, p.amp_average)
        out.append((int(m), tuple(int(v) for v in k), a))
    return out, int(np.count_nonzero(t0))


# ---------------------------------------------------------------------------------------------
# The iteration (Sec. 2.2): sample, DFT, subtract what is known, decode, merge
# ---------------------------------------------------------------------------------------------

@dataclass
class Result:
    k: np.ndarray         # int64 [n][D], sorted by linear index
    a: np.ndarray         # complex128 [n]
    iters: int            # iterations whose lines were sampled
    status: int           # STATUS_OK or STATUS_CAPACITY
    history: list = None  # per iteration: (set size after the iteration, number of T0 bins)


def linear_index(k, dims):
    """Row-major linear index of k[..., D] (last dimension fastest)."""
    k = np.asarray(k, np.int64)
    lin = np.zeros(k.shape[:-1], np.int64)
    for d, n in enumerate(dims):
        lin = lin * int(n) + k[..., d]
    return lin


def merge(S, cands, k_cap):
    """Merge one iteration's decoded (m, k, a) candidates into the recovered set S (dict k -> a).

    Sec. 2.2 adds each decoded frequency to the recovered set and is silent on a frequency that is
    already there; reading A9: its amplitude accumulates the decoded value, which is the residual
    left after that frequency's current amplitude was peeled.  A new frequency is dropped when S
    already holds k_cap entries.  Returns False when one was dropped."""
    ok = True
    for _, kk, aa in cands:
        if kk in S:
            S[kk] = S[kk] + aa
        elif len(S) < k_cap:
            S[kk] = aa
        else:
            ok = False
    return ok


def recover(x, alpha, tau, p, init=None, T=None, keep_history=False):
    """Run the FPS-SFT iterations on one cube x (complex, shape dims) with schedule alpha[t], tau[t].

    init: optional (k, a) recovered set to start from (resume / teacher forcing).
    Returns a Result with the recovered set sorted by linear index."""
    dims = list(x.shape)
    D = len(dims)
    T = p.T if T is None else T
    S = {}
    if init is not None:
        for kk, aa in zip(np.asarray(init[0]).reshape(-1, D), np.asarray(init[1]).reshape(-1)):
            S[tuple(int(v) for v in kk)] = complex(aa)
    status = STATUS_OK
    iters = 0
    hist = []
    for t in range(T):
        al, ta = alpha[t], tau[t]
        ks = np.asarray(list(S.keys()), np.int64).reshape(-1, D)
        as_ = np.asarray(list(S.values()), np.complex128)
        samples = sample_lines(x, al, ta)
        if p.peel_mode == "literal":
            bins = line_dft(peel_literal(samples, ks, as_, al, ta, dims))
        else:
            bins = peel_bins(line_dft(samples), ks, as_, al, ta, dims)
        cands, n_t0 = classify_decode(bins, al, ta, dims, p)
        iters = t + 1
        if p.early_stop and n_t0 == 0:
            hist.append((len(S), n_t0))
            break
        if not merge(S, cands, p.k_cap):
            status = STATUS_CAPACITY
        hist.append((len(S), n_t0))
        if status != STATUS_OK:
            break
        if p.early_stop == 2 and len(cands) == n_t0:
            break           # every bin with energy left on line 0 was one frequency, now recovered
    keep = [(kk, aa) for kk, aa in S.items() if abs(aa) > p.theta0]
    k = np.asarray([kk for kk, _ in keep], np.int64).reshape(-1, D)
    a = np.asarray([aa for _, aa in keep], np.complex128)
    order = np.argsort(linear_index(k, dims), kind="stable")
    return Result(k[order], a[order], iters, status, hist if keep_history else None)


# ---------------------------------------------------------------------------------------------
# Dense references and adjoints (tiny sizes)
# ---------------------------------------------------------------------------------------------

def dense_dft(x):
    """X_hat(k) = (1/N) sum_n x(n) exp(-j 2 pi sum_d k_d n_d / N_d), by explicit summation.  With the
    signal model of Eq. sigModel2, X_hat(k) is the amplitude planted at k."""
    dims = x.shape
    N = x.size
    grids = np.meshgrid(*[np.arange(n) for n in dims], indexing="ij")
    n_flat = [g.reshape(-1) for g in grids]
    out = np.zeros(N, np.complex128)
    xf = x.reshape(-1).astype(np.complex128)
    for i in range(N):
        kk = [n_flat[d][i] for d in range(len(dims))]
        ph = np.zeros(N)
        for d in range(len(dims)):
            ph = ph + kk[d] * n_flat[d] / dims[d]
        out[i] = np.sum(xf * np.exp(-1j * TWO_PI * ph)) / N
    return out.reshape(dims)


def project_matrix(dims, alpha, tau):
    """The matrix of `project` at (alpha, tau): columns are the projections of unit impulses."""
    dims = tuple(int(n) for n in dims)
    N = int(np.prod(dims))
    L, _ = line_length(dims)
    P = np.zeros(((len(dims) + 1) * L, N), np.complex128)
    for i in range(N):
        e = np.zeros(N, np.complex128)
        e[i] = 1.0
        P[:, i] = project(e.reshape(dims), alpha, tau).reshape(-1)
    return P


def project_adjoint(g, alpha, tau, dims):
    """Adjoint of `project`: scatter-add, at the line points, the inverse-direction DFT of each line
    scaled by 1/L: x_bar(n) = sum over (j, l) with n_j(l) = n of (1/L) sum_m g_j(m) exp(+j 2 pi l m / L)."""
    dims = tuple(int(n) for n in dims)
    pts = line_points(dims, alpha, tau)
    L = g.shape[-1]
    back = line_idft(g) / L
    out = np.zeros(dims, np.complex128)
    np.add.at(out, tuple(pts[..., d].reshape(-1) for d in range(len(dims))), back.reshape(-1))
    return out


def synth_adjoint(g, k, alpha, tau, dims):
    """Adjoint of `synth` with respect to a: grad_a_i = sum_j conj(line_phase(k_i, j)) g_j(m(k_i))."""
    dims = [int(n) for n in dims]
    D = len(dims)
    k = np.asarray(k, np.int64).reshape(-1, D)
    m = bin_index(k, alpha, dims)
    out = np.zeros(k.shape[0], np.complex128)
    for j in range(D + 1):
        out = out + np.conj(line_phase(k, tau, dims, j)) * g[j][m]
    return out


# ---------------------------------------------------------------------------------------------
# Least-squares amplitudes over many lines (the refinement the library adds after the loop; the
# paper's decode, Eq. decoding, reads each amplitude from one bin of one line)
# ---------------------------------------------------------------------------------------------

def refine_lstsq(x, alphas, taus, k, method="auto"):
    """argmin_a sum_r || project(x, alpha_r, tau_r) - synth(k, a, alpha_r, tau_r) ||^2 in FP64.

    The stacked system has one column per frequency k_i: the syntheses (Eq. freqSum) of a unit
    amplitude at k_i on every row, and the right-hand side stacks the line DFTs of x (Eq. hs).
    method "dense": numpy's least squares on the dense matrix; "sparse": the normal equations
    A^H A a = A^H y solved directly (scipy) with A stored sparse (each column has one non-zero per
    line and row); "auto": dense while the matrix has at most 4e6 entries."""
    dims = [int(n) for n in x.shape]
    D = len(dims)
    k = np.asarray(k, np.int64).reshape(-1, D)
    n = k.shape[0]
    R = len(alphas)
    y = np.concatenate([project(x, alphas[r], taus[r]).reshape(-1) for r in range(R)])
    if n == 0:
        return np.zeros(0, np.complex128)
    if method == "auto":
        method = "dense" if y.size * n <= 4_000_000 else "sparse"
    rows, cols, vals = [], [], []
    blk = y.size // R
    for i in range(n):
        e = np.zeros(n, np.complex128)
        e[i] = 1.0
        for r in range(R):
            col = synth(k, e, alphas[r], taus[r], dims).reshape(-1)
            nz = np.nonzero(col)[0]
            rows.append(r * blk + nz)
            cols.append(np.full(nz.size, i))
            vals.append(col[nz])
    rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    if method == "dense":
        A = np.zeros((y.size, n), np.complex128)
        np.add.at(A, (rows, cols), vals)
        return np.linalg.lstsq(A, y, rcond=None)[0]
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    A = sp.csr_matrix((vals, (rows, cols)), shape=(y.size, n))
    AH = A.conj().T.tocsr()
    return spla.spsolve((AH @ A).tocsc(), AH @ y)


# ---------------------------------------------------------------------------------------------
# Several offset sets per slope (an extension for noisy data; the paper samples one offset set,
# tau and tau + e_d, per slope in each iteration, Sec. 2.2 and 2.3)
# ---------------------------------------------------------------------------------------------

def classify_decode_sets(bins_s, alpha, taus, dims, p):
    """The tests and decode of `classify_decode` on S offset sets of one slope.

    bins_s[s] are the (peeled) D+1 line DFTs at offset taus[s].  A frequency k in bin m appears in
    every set with the same amplitude and with the offset phase of that set (Eq. freqSum), so the
    ratio s_{s,d+1}(m) / s_{s,0}(m) is the same for every s.  With E_j = mean_s |s_{s,j}(m)|^2:
      T0  sqrt(E_0) > theta0;   T1  |sqrt(E_{d+1}) - sqrt(E_0)| <= rho sqrt(E_0) for every d;
      decode k_d from the phase of the coherent sum sum_s s_{s,d+1}(m) conj(s_{s,0}(m));  T2, T3 as
      in `classify_decode`;  a = mean over the sets of s_{s,0}(m) times the conjugate offset phase
      of line 0 (with p.amp_average: mean over sets and lines).
    With one set this is `classify_decode`.  Returns (list of (m, k, a), number of bins passing T0)."""
    dims = [int(n) for n in dims]
    D = len(dims)
    S = len(bins_s)
    E = [np.mean([np.abs(bins_s[s][j]) ** 2 for s in range(S)], axis=0) for j in range(D + 1)]
    mag0 = np.sqrt(E[0])
    t0 = mag0 > p.theta0
    out = []
    for m in np.nonzero(t0)[0]:
        if any(abs(math.sqrt(E[d + 1][m]) - mag0[m]) > p.rho * mag0[m] for d in range(D)):
            continue
        k = []
        ok = True
        for d in range(D):
            r = sum(bins_s[s][d + 1][m] * np.conj(bins_s[s][0][m]) for s in range(S))
            u = dims[d] * np.angle(r) / TWO_PI
            q = math.floor(u + 0.5)
            if abs(u - q) > p.eta:
                ok = False
                break
            k.append(q % dims[d])
        if not ok or not projects_to(m, k, alpha, dims):
            continue
        a = sum(decoded_amplitude(bins_s[s], m, k, taus[s], dims, p.amp_average) for s in range(S)) / S
        out.append((int(m), tuple(int(v) for v in k), a))
    return out, int(np.count_nonzero(t0))


def recover_offset_sets(x, alpha, taus, p):
    """`recover` with S offset sets per slope: iteration t samples the D+1 lines at slope alpha[t]
    for each offset taus[t][s] (S (D+1) L samples), peels the recovered set from every set's bins
    and decodes with `classify_decode_sets`.  Merge, early stop and output as in `recover`."""
    dims = list(x.shape)
    D = len(dims)
    S = {}
    status = STATUS_OK
    iters = 0
    for t in range(len(alpha)):
        al = alpha[t]
        ks = np.asarray(list(S.keys()), np.int64).reshape(-1, D)
        as_ = np.asarray(list(S.values()), np.complex128)
        bins_s = [peel_bins(project(x, al, ta), ks, as_, al, ta, dims) for ta in taus[t]]
        cands, n_t0 = classify_decode_sets(bins_s, al, taus[t], dims, p)
        iters = t + 1
        if p.early_stop and n_t0 == 0:
            break
        if not merge(S, cands, p.k_cap):
            status = STATUS_CAPACITY
            break
        if p.early_stop == 2 and len(cands) == n_t0:
            break
    keep = [(kk, aa) for kk, aa in S.items() if abs(aa) > p.theta0]
    k = np.asarray([kk for kk, _ in keep], np.int64).reshape(-1, D)
    a = np.asarray([aa for _, aa in keep], np.complex128)
    order = np.argsort(linear_index(k, dims), kind="stable")
    return Result(k[order], a[order], iters, status)
