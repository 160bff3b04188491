"""Plant plausible mistakes in the oracle (on the CPU) and check that some pin catches each one.

A pin set that cannot tell a dropped term, a wrong sign, a wrong index or a transposed operand
from the correct oracle would not pin it; these tests show that it can."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import fpssft_oracle as O

import pins

CHECKS = [
    pins.check_line_dft_definition,
    pins.check_projection_slice,
    pins.check_bin_index_rational,
    pins.check_lemma1_minimal,
    pins.check_uniform_projection,
    pins.check_single_sinusoid,
    pins.check_tiny_support,
    pins.check_peel_equivalence,
    pins.check_synth_is_projection,
    pins.check_adjoints,
    pins.check_deadlock,
    pins.check_fig3_samples,
    pins.check_redecode_accumulates,
    pins.check_projection_test,
    pins.check_sparsity_tests,
    pins.check_early_stop,
    pins.check_capacity,
    pins.check_amplitude_average,
    pins.check_refine_lstsq,
    pins.check_offset_sets,
    pins.check_early_stop_decoded,
]

_orig = {name: getattr(O, name) for name in dir(O) if callable(getattr(O, name))}


def _dft_plus_sign(s):
    return np.fft.ifft(s, axis=-1)


def _dft_no_scale(s):
    return np.fft.fft(s, axis=-1)


def _points_no_shift(dims, alpha, tau):
    p = _orig["line_points"](dims, alpha, tau)
    return np.repeat(p[:1], p.shape[0], axis=0)


def _points_shift_wrong_dim(dims, alpha, tau):
    D = len(dims)
    out = _orig["line_points"](dims, alpha, tau)
    l = np.arange(out.shape[1])
    for j in range(1, D + 1):
        for d in range(D):
            shift = 1 if (j % D) == d else 0
            out[j, :, d] = (int(alpha[d]) * l + int(tau[d]) + shift) % int(dims[d])
    return out


def _bin_reversed_alpha(k, alpha, dims):
    return _orig["bin_index"](k, list(alpha)[::-1], dims)


def _phase_no_tau(k, tau, dims, j):
    return _orig["line_phase"](k, [0] * len(dims), dims, j)


def _phase_conj(k, tau, dims, j):
    return np.conj(_orig["line_phase"](k, tau, dims, j))


def _length_product(dims):
    L = int(np.prod(dims))
    return L, [L // int(n) for n in dims]


def _length_max(dims):
    L = max(int(n) for n in dims)
    return L, [max(1, L // int(n)) for n in dims]


def _uniform_no_L(alpha, dims):
    _, c = O.line_length(dims)
    g = 0
    for cd, ad in zip(c, alpha):
        g = math.gcd(g, cd * int(ad))
    return g == 1


def _adjoint_forward_dft(g, alpha, tau, dims):
    pts = O.line_points(dims, alpha, tau)
    back = np.fft.fft(g, axis=-1) / g.shape[-1]
    out = np.zeros(tuple(dims), np.complex128)
    np.add.at(out, tuple(pts[..., d].reshape(-1) for d in range(len(dims))), back.reshape(-1))
    return out


def _classify_inverted_ratio(bins, alpha, tau, dims, p):
    # decode from s_0 / s_{d+1} instead of s_{d+1} / s_0: the phase (and so k_d) changes sign
    flipped = bins.copy()
    with np.errstate(divide="ignore", invalid="ignore"):
        flipped[1:] = np.nan_to_num(bins[0] * np.conj(bins[1:] / bins[0]))
    return _orig["classify_decode"](flipped, alpha, tau, dims, p)


def _synth_line0_only(k, a, alpha, tau, dims):
    out = _orig["synth"](k, a, alpha, tau, dims)
    out[1:] = out[:1]
    return out


def _merge_overwrites(S, cands, k_cap):
    # a re-decoded frequency takes the decoded residual as its amplitude
    ok = True
    for _, kk, aa in cands:
        if kk in S or len(S) < k_cap:
            S[kk] = aa
        else:
            ok = False
    return ok


def _merge_ignores_known(S, cands, k_cap):
    # a frequency already in the set keeps its amplitude
    ok = True
    for _, kk, aa in cands:
        if kk in S:
            continue
        if len(S) < k_cap:
            S[kk] = aa
        else:
            ok = False
    return ok


def _projection_test_dropped(m, k, alpha, dims):
    return True


def _classify_without(field):
    def classify(bins, alpha, tau, dims, p):
        return _orig["classify_decode"](bins, alpha, tau, dims, dataclasses.replace(p, **{field: 1e9}))
    return classify


def _idft_unscaled(s_hat):
    return np.fft.ifft(s_hat, axis=-1)


def _classify_never_empty(bins, alpha, tau, dims, p):
    # the early stop never fires: every iteration reports a bin passing T0
    cands, n0 = _orig["classify_decode"](bins, alpha, tau, dims, p)
    return cands, n0 + 1


def _merge_hides_overflow(S, cands, k_cap):
    _orig["merge"](S, cands, k_cap)
    return True


def _average_with_line0_phase(bins, m, k, tau, dims, average=False):
    # every line corrected by line 0's offset phase (the e_d shift of lines 1..D forgotten)
    if not average:
        return _orig["decoded_amplitude"](bins, m, k, tau, dims, False)
    ph0 = np.conj(O.line_phase(np.asarray(k), tau, dims, 0))
    return complex(sum(bins[j][m] for j in range(len(dims) + 1)) * ph0 / (len(dims) + 1))


def _refine_line0_only(x, alphas, taus, k, method="auto"):
    # least squares over line 0 of every row only (the offset lines forgotten)
    dims = [int(n) for n in x.shape]
    k = np.asarray(k, np.int64).reshape(-1, len(dims))
    cols = []
    for i in range(k.shape[0]):
        e = np.zeros(k.shape[0], np.complex128)
        e[i] = 1
        cols.append(np.concatenate([O.synth(k, e, al, ta, dims)[0] for al, ta in zip(alphas, taus)]))
    y = np.concatenate([O.project(x, al, ta)[0] for al, ta in zip(alphas, taus)])
    return np.linalg.lstsq(np.stack(cols, axis=1), y, rcond=None)[0]


def _refine_mean_of_decodes(x, alphas, taus, k, method="auto"):
    # every amplitude taken as the mean of its phase-corrected bins, as if no two frequencies shared a bin
    dims = [int(n) for n in x.shape]
    k = np.asarray(k, np.int64).reshape(-1, len(dims))
    acc = np.zeros(k.shape[0], np.complex128)
    for al, ta in zip(alphas, taus):
        bins = O.project(x, al, ta)
        m = O.bin_index(k, al, dims)
        for j in range(len(dims) + 1):
            acc += bins[j][m] * np.conj(O.line_phase(k, ta, dims, j))
    return acc / (len(alphas) * (len(dims) + 1))


def _sets_phase_from_first(bins_s, alpha, taus, dims, p):
    # the decode phase taken from the first offset set only (no coherent sum)
    cands, n0 = _orig["classify_decode_sets"](bins_s[:1], alpha, taus[:1], dims, p)
    full, n0_all = _orig["classify_decode_sets"](bins_s, alpha, taus, dims, p)
    amp = {m: a for m, _, a in full}
    return [(m, k, amp.get(m, a)) for m, k, a in cands], n0_all


def _sets_amplitude_from_first(bins_s, alpha, taus, dims, p):
    # the amplitude taken from the first offset set only
    cands, n0 = _orig["classify_decode_sets"](bins_s, alpha, taus, dims, p)
    return [(m, k, O.decoded_amplitude(bins_s[0], m, k, taus[0], dims, p.amp_average)) for m, k, _ in cands], n0


def _classify_claims_every_bin_decoded(bins, alpha, tau, dims, p):
    # the decoded-stop fires after any iteration that decoded something (T0 count replaced by the
    # number of decodes whenever there is one)
    cands, n0 = _orig["classify_decode"](bins, alpha, tau, dims, p)
    return cands, (len(cands) if cands else n0)


MUTATIONS = {
    "dft sign flipped": ("line_dft", _dft_plus_sign),
    "dft 1/L dropped": ("line_dft", _dft_no_scale),
    "offset lines not shifted": ("line_points", _points_no_shift),
    "offset shifted on the wrong dimension": ("line_points", _points_shift_wrong_dim),
    "slope components transposed in the bin map": ("bin_index", _bin_reversed_alpha),
    "offset phase dropped": ("line_phase", _phase_no_tau),
    "offset phase conjugated": ("line_phase", _phase_conj),
    "line length is the product": ("line_length", _length_product),
    "line length is the max": ("line_length", _length_max),
    "uniformity test ignores L": ("uniform_projection", _uniform_no_L),
    "adjoint uses the forward DFT": ("project_adjoint", _adjoint_forward_dft),
    "decode uses the inverted ratio": ("classify_decode", _classify_inverted_ratio),
    "synthesis ignores the offset lines": ("synth", _synth_line0_only),
    "re-decoded amplitude overwrites": ("merge", _merge_overwrites),
    "re-decoded frequency ignored": ("merge", _merge_ignores_known),
    "projection test T3 dropped": ("projects_to", _projection_test_dropped),
    "magnitude test T1 dropped": ("classify_decode", _classify_without("rho")),
    "grid test T2 dropped": ("classify_decode", _classify_without("eta")),
    "inverse line DFT loses the factor L": ("line_idft", _idft_unscaled),
    "early stop never fires": ("classify_decode", _classify_never_empty),
    "a full set is not reported": ("merge", _merge_hides_overflow),
    "averaged amplitude ignores the lines' own offset phases": ("decoded_amplitude", _average_with_line0_phase),
    "least squares over line 0 only": ("refine_lstsq", _refine_line0_only),
    "least squares replaced by the mean of the decodes": ("refine_lstsq", _refine_mean_of_decodes),
    "offset sets: phase from the first set only": ("classify_decode_sets", _sets_phase_from_first),
    "offset sets: amplitude from the first set only": ("classify_decode_sets", _sets_amplitude_from_first),
    "decoded-stop fires after any decode": ("classify_decode", _classify_claims_every_bin_decoded),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(O, attr, fn)
    caught = []
    for check in CHECKS:
        try:
            check(O)
        except (AssertionError, ValueError, IndexError):
            caught.append(check.__name__)
    assert caught, f"no pin caught the planted mistake: {name}"
