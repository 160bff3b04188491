"""Autograd through the adjoint kernels, checked in FP64 against the oracle (needs a GB300).

The GPU computes in FP32; its gradients are compared with finite differences of the oracle's FP64
forward maps and with the oracle's explicit dense adjoints, on small cubes (8x8x8 and 2-D)."""

import numpy as np
import pytest
import torch

from oracle import fpssft_oracle as O
from paper_1711_11407_gb300 import configs
from paper_1711_11407_gb300 import synth as S

pytestmark = pytest.mark.gpu


def dev():
    return torch.device("cuda:0")


def _wl(shapes, batch, K, T, snr_db=None, seed=5):
    return S.make_workload("uneven_2d", seed=seed, batch=batch, shapes=shapes, K=K, T=T, snr_db=snr_db)


def test_line_project_backward_matches_fp64_finite_differences_8x8x8():
    from paper_1711_11407_gb300.api import Plan
    from paper_1711_11407_gb300.autograd import line_project
    wl = _wl([(8, 8, 8)], 1, K=lambda N: 5, T=3, snr_db=0.0)
    plan = Plan(wl.dims, configs.params_for(wl, T=3, k_cap=16))
    x = torch.from_numpy(wl.cubes).to(dev()).requires_grad_(True)
    offs, al, ta = (torch.from_numpy(v).to(dev()) for v in (wl.offsets, wl.alpha, wl.tau))
    rng = np.random.default_rng(0)
    L = int(plan.L[0])
    w = (rng.normal(size=(1, 3, 4, plan.L_max)) + 1j * rng.normal(size=(1, 3, 4, plan.L_max))).astype(np.complex64)
    w[..., L:] = 0
    y = line_project(x, plan, offs, al, ta)
    loss = torch.sum((torch.from_numpy(w).to(dev()).conj() * y).real)
    loss.backward()
    grad = x.grad.cpu().numpy().reshape(8, 8, 8).astype(np.complex128)
    # FP64 finite differences of the oracle's projection, l(x) = Re sum conj(w) P x
    x0 = wl.cube(0)

    def ell(z):
        tot = 0.0
        for s in range(3):
            tot += float(np.sum((np.conj(w[0, s, :, :L]).astype(np.complex128) * O.project(z, wl.alpha[0, s], wl.tau[0, s])).real))
        return tot

    h = 1e-6
    for idx in [tuple(int(v) for v in rng.integers(0, 8, 3)) for _ in range(6)]:
        e = np.zeros((8, 8, 8), np.complex128)
        e[idx] = 1.0
        dre = (ell(x0 + h * e) - ell(x0 - h * e)) / (2 * h)
        dim = (ell(x0 + 1j * h * e) - ell(x0 - 1j * h * e)) / (2 * h)
        ref = complex(dre, dim)
        assert abs(grad[idx] - ref) <= 1e-5 * max(1.0, abs(ref)), f"{idx}: GPU {grad[idx]} vs FD {ref}"
    # the explicit dense adjoint of the oracle
    dense = np.zeros((8, 8, 8), np.complex128)
    for s in range(3):
        dense += O.project_adjoint(w[0, s, :, :L].astype(np.complex128), wl.alpha[0, s], wl.tau[0, s], (8, 8, 8))
    assert np.linalg.norm(grad - dense) <= 1e-5 * np.linalg.norm(dense)


def test_sparse_synth_backward_matches_dense_adjoint_and_fd():
    from paper_1711_11407_gb300.api import Plan
    from paper_1711_11407_gb300.autograd import sparse_synth
    wl = _wl([(12, 18), (16, 16)], 2, K=lambda N: 6, T=4)
    plan = Plan(wl.dims, configs.params_for(wl, T=4, k_cap=8))
    al, ta = (torch.from_numpy(v).to(dev()) for v in (wl.alpha, wl.tau))
    k = np.zeros((2, 8, 2), np.int32)
    cnt = np.zeros(2, np.int32)
    for b in range(2):
        k[b, :6] = wl.k_true[b]
        cnt[b] = 6
    rng = np.random.default_rng(1)
    a = (rng.normal(size=(2, 8)) + 1j * rng.normal(size=(2, 8))).astype(np.complex64)
    at = torch.from_numpy(a).to(dev()).requires_grad_(True)
    kd, cd = torch.from_numpy(k).to(dev()), torch.from_numpy(cnt).to(dev())
    w = (rng.normal(size=(2, 4, 3, plan.L_max)) + 1j * rng.normal(size=(2, 4, 3, plan.L_max))).astype(np.complex64)
    y = sparse_synth(at, plan, kd, cd, al, ta)
    torch.sum((torch.from_numpy(w).to(dev()).conj() * y).real).backward()
    g = at.grad.cpu().numpy()
    for b in range(2):
        dims = tuple(int(v) for v in wl.dims[b])
        L = int(plan.L[b])
        ref = np.zeros(6, np.complex128)
        for s in range(4):
            ref += O.synth_adjoint(w[b, s, :, :L].astype(np.complex128), k[b, :6], wl.alpha[b, s], wl.tau[b, s], dims)
        assert np.allclose(g[b, :6], ref, rtol=1e-5, atol=1e-5)
        assert np.all(g[b, 6:] == 0)


def test_refine_reaches_the_fp64_least_squares_amplitudes_and_beats_the_decode():
    """Noisy 2-D batch, support from the recovery; the refined amplitudes equal the dense FP64
    least-squares solution over the same lines and are closer to the planted ones."""
    from paper_1711_11407_gb300.api import Plan
    from paper_1711_11407_gb300.autograd import refine
    wl = S.make_workload("uneven_2d", batch=4, shapes=[(64, 64)], K=lambda N: 12, T=24, snr_db=20.0)
    p = configs.params_for(wl, T=24, k_cap=64)
    plan = Plan(wl.dims, p)
    cubes, offs, al, ta = (torch.from_numpy(v).to(dev()) for v in (wl.cubes, wl.offsets, wl.alpha, wl.tau))
    out = plan.recover(cubes, offs, al, ta)
    torch.cuda.synchronize()
    planr = Plan(wl.dims, configs.params_for(wl, T=24, k_cap=64))
    a_ref, res = refine(planr, cubes, offs, out.k, out.a, out.count, al, ta)
    torch.cuda.synchronize()
    a_ref = a_ref.cpu().numpy()
    improved = 0
    for b in range(wl.batch):
        n = int(out.count[b])
        k = out.k[b, :n].cpu().numpy().astype(np.int64)
        a_dec = out.a[b, :n].cpu().numpy()
        dims = (64, 64)
        L = 64
        # dense least squares in FP64 over the same 24 schedule rows
        cols = []
        for i in range(n):
            e = np.zeros(n, np.complex128)
            e[i] = 1
            cols.append(np.concatenate([O.synth(k, e, wl.alpha[b, s], wl.tau[b, s], dims).reshape(-1) for s in range(24)]))
        A = np.stack(cols, axis=1)
        y = np.concatenate([O.project(wl.cube(b), wl.alpha[b, s], wl.tau[b, s]).reshape(-1) for s in range(24)])
        a_ls = np.linalg.lstsq(A, y, rcond=None)[0]
        assert np.allclose(a_ref[b, :n], a_ls, rtol=1e-4, atol=1e-5), "refined amplitudes differ from FP64 least squares"
        truth = dict(zip(map(tuple, wl.k_true[b]), wl.a_true[b]))
        common = [i for i in range(n) if tuple(k[i]) in truth]
        err_dec = np.linalg.norm([a_dec[i] - truth[tuple(k[i])] for i in common])
        err_ref = np.linalg.norm([a_ref[b, i] - truth[tuple(k[i])] for i in common])
        improved += int(err_ref < err_dec)
    assert improved >= 3
