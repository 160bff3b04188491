"""Precision statement: the measured error of the FP32 GPU path against the FP64 oracle (needs a
GB300).

All GPU arithmetic is FP32 (FP64 only for the decode's decisions and the refinement's CG
scalars).  For every workload this test measures, and prints as one JSON line:
  bins        relative L2 error per line of the line DFTs (Eq. hs), fpssft_project vs the oracle;
  amplitudes  relative error per recovered entry (Eq. decoding, accumulated over iterations),
              fpssft_recover vs the oracle, where both recovered the same set;
  gradients   relative L2 error of the two adjoints (fpssft_adjoint) against the oracle's explicit
              adjoints, and the largest relative error of the projection gradient against FP64
              central differences (8 x 8 x 8);
  refine      relative L2 error of fpssft_refine (planted support) against FP64 least squares.
Each figure must stay within the parity tolerances (1e-5 bins, 1e-4 amplitudes and gradients) and
within 10x of the value recorded here from a GB300 run, so a precision regression fails."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import fpssft_oracle as O
from paper_1711_11407_gb300 import configs
from paper_1711_11407_gb300 import synth as S

pytestmark = pytest.mark.gpu

TOL = {"bins": 1e-5, "amplitudes": 1e-4, "gradients": 1e-4, "refine": 1e-4}
# measured maxima on one GB300 (sm_103a); the test fails above 10x these
RECORDED = {
    "bins": {"single_128x128": 8.9e-08, "single_240x256": 1.3e-07, "batched_64x64x64": 9.9e-08,
             "uneven_2d": 9.9e-08, "images_1024x1024": 1.1e-07, "sparse_image_512x576": 1.3e-07},
    "amplitudes": {"single_128x128": 1.5e-07, "single_240x256": 2.1e-07, "uneven_2d": 6.9e-07,
                   "sparse_image_512x576": 2.3e-06, "images_1024x1024": 2.3e-07},
    "gradients": {"adjoint_project": 8.0e-08, "adjoint_synth": 1.5e-07, "project_gradient_vs_fd": 6.0e-08},
    "refine": {"batched_64x64x64": 1.9e-07, "images_1024x1024": 1.5e-07},
}

BIN_SAMPLES = {"single_128x128": 1, "single_240x256": 1, "batched_64x64x64": 2, "uneven_2d": 8,
               "images_1024x1024": 2, "sparse_image_512x576": 1}
AMP_CASES = {"single_128x128": None, "single_240x256": None, "uneven_2d": 16, "sparse_image_512x576": 2,
             "batched_64x64x64": 8, "images_1024x1024": 2}


def dev():
    return torch.device("cuda:0")


def to_dev(wl):
    d = dev()
    return (torch.from_numpy(wl.cubes).to(d), torch.from_numpy(wl.offsets).to(d),
            torch.from_numpy(wl.alpha).to(d), torch.from_numpy(wl.tau).to(d))


def _stats(v):
    v = np.asarray(v, np.float64)
    return {"max": float(v.max()), "median": float(np.median(v)), "n": int(v.size)} if v.size else None


def _bins_errors(name, nsig, rows=4):
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload(name, batch=nsig)
    plan = Plan(wl.dims)
    cubes, offs, al, ta = to_dev(wl)
    al, ta = al[:, :rows].contiguous(), ta[:, :rows].contiguous()
    bins = plan.project(cubes, offs, al, ta).cpu().numpy()
    errs = []
    for b in range(wl.batch):
        L = int(plan.L[b])
        for s in range(al.shape[1]):
            ref = O.project(wl.cube(b), wl.alpha[b, s], wl.tau[b, s])
            for j in range(wl.D + 1):
                errs.append(np.linalg.norm(bins[b, s, j, :L] - ref[j]) / np.linalg.norm(ref[j]))
    plan.close()
    return errs


def _amp_errors(name, nsig):
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload(name, batch=nsig)
    p = configs.params_for(wl)
    plan = Plan(wl.dims, p)
    cubes, offs, al, ta = to_dev(wl)
    out = plan.recover(cubes, offs, al, ta)
    torch.cuda.synchronize()
    errs, same = [], 0
    for b in range(wl.batch):
        T = int(plan.T[b])
        ref = O.recover(wl.cube(b), wl.alpha[b, :T], wl.tau[b, :T],
                        O.Params(T=T, k_cap=p.k_cap, theta0=p.theta0, rho=p.rho, eta=p.eta, early_stop=p.early_stop))
        k, a = out.signal(b)
        if not np.array_equal(k, ref.k):
            continue
        same += 1
        errs.extend((np.abs(a - ref.a) / np.abs(ref.a)).tolist())
    plan.close()
    return errs, same, wl.batch


def _gradient_errors():
    from paper_1711_11407_gb300.api import Plan
    out = {}
    rng = np.random.default_rng(3)
    # projection adjoint on 8x8x8 and 64x64 against the oracle's adjoint
    e_proj, e_syn = [], []
    for shapes, K in (([(8, 8, 8)], 5), ([(64, 64)], 20)):
        wl = S.make_workload("uneven_2d", seed=11, batch=2, shapes=shapes, K=lambda N, K=K: K, T=4, snr_db=0.0)
        plan = Plan(wl.dims, configs.params_for(wl, T=4, k_cap=32))
        cubes, offs, al, ta = to_dev(wl)
        D = wl.D
        g = (rng.normal(size=(2, 4, D + 1, plan.L_max)) + 1j * rng.normal(size=(2, 4, D + 1, plan.L_max))).astype(np.complex64)
        gt = torch.from_numpy(g).to(dev())
        grad = torch.zeros(wl.cubes.size, dtype=torch.complex64, device=dev())
        plan.adjoint_project(gt, offs, al, ta, grad)
        k = np.zeros((2, plan.k_cap, D), np.int32)
        cnt = np.zeros(2, np.int32)
        for b in range(2):
            k[b, :K] = wl.k_true[b]
            cnt[b] = K
        ga = plan.adjoint_synth(gt, al, ta, torch.from_numpy(k).to(dev()), torch.from_numpy(cnt).to(dev()))
        grad = grad.cpu().numpy()
        ga = ga.cpu().numpy()
        for b in range(2):
            dims = tuple(int(v) for v in wl.dims[b])
            L = int(plan.L[b])
            ref = sum(O.project_adjoint(g[b, s, :, :L].astype(np.complex128), wl.alpha[b, s], wl.tau[b, s], dims)
                      for s in range(4))
            o = int(wl.offsets[b])
            got = grad[o:o + int(np.prod(dims))].reshape(dims)
            e_proj.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
            refa = sum(O.synth_adjoint(g[b, s, :, :L].astype(np.complex128), k[b, :K], wl.alpha[b, s], wl.tau[b, s], dims)
                       for s in range(4))
            e_syn.append(np.linalg.norm(ga[b, :K] - refa) / np.linalg.norm(refa))
        plan.close()
    out["adjoint_project"] = _stats(e_proj)
    out["adjoint_synth"] = _stats(e_syn)
    # gradient of l(x) = Re sum conj(w) P x against FP64 central differences of the oracle (8x8x8)
    from paper_1711_11407_gb300.autograd import line_project
    wl = S.make_workload("uneven_2d", seed=5, batch=1, shapes=[(8, 8, 8)], K=lambda N: 5, T=3, snr_db=0.0)
    plan = Plan(wl.dims, configs.params_for(wl, T=3, k_cap=16))
    x = torch.from_numpy(wl.cubes).to(dev()).requires_grad_(True)
    offs, al, ta = (torch.from_numpy(v).to(dev()) for v in (wl.offsets, wl.alpha, wl.tau))
    L = int(plan.L[0])
    w = (rng.normal(size=(1, 3, 4, plan.L_max)) + 1j * rng.normal(size=(1, 3, 4, plan.L_max))).astype(np.complex64)
    w[..., L:] = 0
    y = line_project(x, plan, offs, al, ta)
    torch.sum((torch.from_numpy(w).to(dev()).conj() * y).real).backward()
    grad = x.grad.cpu().numpy().reshape(8, 8, 8).astype(np.complex128)
    x0 = wl.cube(0)

    def ell(z):
        return sum(float(np.sum((np.conj(w[0, s, :, :L]).astype(np.complex128) * O.project(z, wl.alpha[0, s], wl.tau[0, s])).real))
                   for s in range(3))

    h = 1e-6
    e_fd = []
    hit = [tuple(int(v) for v in i) for i in np.argwhere(np.abs(grad) > 0)]     # points some line samples
    for idx in [hit[int(i)] for i in rng.choice(len(hit), 12, replace=False)]:
        e = np.zeros((8, 8, 8), np.complex128)
        e[idx] = 1.0
        ref = complex((ell(x0 + h * e) - ell(x0 - h * e)) / (2 * h), (ell(x0 + 1j * h * e) - ell(x0 - 1j * h * e)) / (2 * h))
        e_fd.append(abs(grad[idx] - ref) / max(abs(ref), 1e-30))
    out["project_gradient_vs_fd"] = _stats(e_fd)
    plan.close()
    return out


def _refine_errors(name, nsig, R):
    """fpssft_refine on the planted support over R schedule rows against FP64 least squares."""
    from paper_1711_11407_gb300.api import Plan
    from paper_1711_11407_gb300.autograd import refine
    wl = S.make_workload(name, batch=nsig)
    p = configs.params_for(wl)
    plan = Plan(wl.dims, p)
    cubes, offs, al, ta = to_dev(wl)
    k = torch.zeros((wl.batch, plan.k_cap, wl.D), dtype=torch.int32)
    cnt = torch.zeros(wl.batch, dtype=torch.int32)
    for b in range(wl.batch):
        n = len(wl.k_true[b])
        k[b, :n] = torch.from_numpy(wl.k_true[b].astype(np.int32))
        cnt[b] = n
    k, cnt = k.to(dev()), cnt.to(dev())
    a0 = torch.zeros((wl.batch, plan.k_cap), dtype=torch.complex64, device=dev())
    a, _ = refine(plan, cubes, offs, k, a0, cnt, al[:, :R].contiguous(), ta[:, :R].contiguous(), iters=30)
    torch.cuda.synchronize()
    errs = []
    for b in range(wl.batch):
        n = int(cnt[b])
        ref = O.refine_lstsq(wl.cube(b), wl.alpha[b, :R], wl.tau[b, :R], wl.k_true[b])
        errs.append(np.linalg.norm(a[b, :n].cpu().numpy() - ref) / np.linalg.norm(ref))
    plan.close()
    return errs


def test_precision_against_the_fp64_oracle_is_stated_and_holds():
    res = {"bins": {}, "amplitudes": {}, "gradients": {}, "refine": {}}
    for name, n in BIN_SAMPLES.items():
        res["bins"][name] = _stats(_bins_errors(name, n))
    for name, n in AMP_CASES.items():
        errs, same, tot = _amp_errors(name, n)
        st = _stats(errs)
        if st is not None:
            st["signals_with_equal_sets"] = f"{same}/{tot}"
        res["amplitudes"][name] = st
    res["gradients"] = _gradient_errors()
    res["refine"]["batched_64x64x64"] = _stats(_refine_errors("batched_64x64x64", 2, 32))
    res["refine"]["images_1024x1024"] = _stats(_refine_errors("images_1024x1024", 1, 8))
    line = json.dumps(res)
    print(line)
    outdir = os.environ.get("FPSSFT_PRECISION_OUT")
    if outdir:
        with open(os.path.join(outdir, "precision.json"), "w") as f:
            f.write(line + "\n")
    for group, entries in res.items():
        for name, st in entries.items():
            if st is None:
                continue
            assert st["max"] <= TOL[group], f"{group}/{name}: max error {st['max']:.2e} above {TOL[group]:.0e}"
            rec = RECORDED.get(group, {}).get(name)
            if rec is not None:
                assert st["max"] <= 10 * rec, f"{group}/{name}: max error {st['max']:.2e} regressed past 10x {rec:.2e}"
