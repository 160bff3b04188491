"""CUDA path against the FP64 oracle, element by element, through the C ABI (needs a GB300).

Tolerances: integer work (gathered samples, frequency indices, iteration counts, status) is
compared exactly; FP32 line bins within 1e-5 relative L2 per line; amplitudes within 1e-4 relative
per entry.  The oracle receives the same complex64 cube (upcast to complex128) and the same
schedule."""
import math

import numpy as np
import pytest
import torch

from oracle import fpssft_oracle as O
from paper_1711_11407_gb300 import configs
from paper_1711_11407_gb300 import synth as S

pytestmark = pytest.mark.gpu

BIN_TOL = 1e-5
AMP_TOL = 1e-4


def dev():
    return torch.device("cuda:0")


def to_dev(wl):
    d = dev()
    return (torch.from_numpy(wl.cubes).to(d), torch.from_numpy(wl.offsets).to(d),
            torch.from_numpy(wl.alpha).to(d), torch.from_numpy(wl.tau).to(d))


def oracle_params(p, T):
    return O.Params(T=T, k_cap=p.k_cap, theta0=p.theta0, rho=p.rho, eta=p.eta, early_stop=p.early_stop)


def assert_same_set(k, a, ref, ctx=""):
    assert k.shape == ref.k.shape and np.array_equal(k, ref.k), f"support differs from the oracle {ctx}"
    err = np.abs(a - ref.a)
    assert np.all(err <= AMP_TOL * np.maximum(np.abs(ref.a), 1e-30)), f"amplitude error {err.max()} {ctx}"


def small_batch(shapes, batch, K, T, seed=7, snr_db=None):
    return S.make_workload("uneven_2d", seed=seed, batch=batch, shapes=shapes, K=K, T=T, snr_db=snr_db)


SHAPE_SETS = {
    "D1": [(16,), (30,), (7,), (64,)],
    "D2-ragged": [(6, 10), (5, 7), (1, 16), (7, 11), (12, 18), (64, 64)],
    "D2-large": [(128, 128), (240, 256), (256, 256)],
    "D3": [(4, 6, 3), (8, 8, 8), (5, 3, 2), (64, 64, 64)],
    "D4": [(4, 4, 2, 3), (2, 3, 2, 5)],
}


@pytest.mark.parametrize("name", sorted(SHAPE_SETS))
def test_lines_are_exact_copies_of_the_oracle_samples(name):
    from paper_1711_11407_gb300.api import Plan
    wl = small_batch(SHAPE_SETS[name], 12, K=lambda N: min(4, N), T=3)
    plan = Plan(wl.dims)
    cubes, offs, al, ta = to_dev(wl)
    lines = plan.lines(cubes, offs, al, ta).cpu().numpy()
    for b in range(wl.batch):
        L = int(plan.L[b])
        for s in range(wl.alpha.shape[1]):
            ref = O.sample_lines(wl.cube(b), wl.alpha[b, s], wl.tau[b, s])
            got = lines[b, s, :, :L].astype(np.complex128)
            assert np.array_equal(got, ref), f"gathered samples differ: signal {b} dims {wl.dims[b]} row {s}"
            assert np.all(lines[b, s, :, L:] == 0)


@pytest.mark.parametrize("name", sorted(SHAPE_SETS))
def test_project_matches_oracle_line_dft(name):
    from paper_1711_11407_gb300.api import Plan
    wl = small_batch(SHAPE_SETS[name], 10, K=lambda N: min(6, N), T=3, snr_db=0.0)   # noisy: dense bins
    plan = Plan(wl.dims)
    cubes, offs, al, ta = to_dev(wl)
    bins = plan.project(cubes, offs, al, ta).cpu().numpy()
    worst = 0.0
    for b in range(wl.batch):
        L = int(plan.L[b])
        for s in range(wl.alpha.shape[1]):
            ref = O.project(wl.cube(b), wl.alpha[b, s], wl.tau[b, s])
            for j in range(wl.D + 1):
                e = np.linalg.norm(bins[b, s, j, :L] - ref[j]) / max(np.linalg.norm(ref[j]), 1e-30)
                worst = max(worst, e)
                assert e <= BIN_TOL, f"line bins rel L2 {e:.2e} > {BIN_TOL}: dims {wl.dims[b]} line {j}"
            assert np.all(bins[b, s, :, L:] == 0)
    print(f"worst line-bin relative L2 error: {worst:.2e}")


RECOVER_CASES = {
    "config1_single_128x128": lambda: S.make_workload("single_128x128"),
    "config2_single_240x256": lambda: S.make_workload("single_240x256"),
    "uneven_2d_48": lambda: S.make_workload("uneven_2d", batch=48),
    "D3_16cubed": lambda: small_batch([(16, 16, 16)], 6, K=lambda N: 30, T=20),
    "D1": lambda: small_batch([(64,), (60,), (7,)], 6, K=lambda N: min(5, N // 2), T=6),
    "D4": lambda: small_batch([(4, 4, 4, 6)], 4, K=lambda N: 4, T=10),
    "D2-ragged": lambda: small_batch([(6, 10), (5, 7), (7, 11), (12, 18), (1, 16)], 10, K=lambda N: max(1, min(4, N // 8)), T=12),
}


@pytest.mark.parametrize("case", sorted(RECOVER_CASES))
def test_recover_matches_oracle(case):
    from paper_1711_11407_gb300.api import Plan
    wl = RECOVER_CASES[case]()
    if case.startswith("D"):     # small batches with a fixed schedule length
        p = configs.params_for(wl, T=int(wl.alpha.shape[1]), k_cap=64)
    else:
        p = configs.params_for(wl)
    plan = Plan(wl.dims, p)
    cubes, offs, al, ta = to_dev(wl)
    out = plan.recover(cubes, offs, al, ta)
    torch.cuda.synchronize()
    for b in range(wl.batch):
        T = int(plan.T[b])
        ref = O.recover(wl.cube(b), wl.alpha[b, :T], wl.tau[b, :T], oracle_params(p, T))
        k, a = out.signal(b)
        assert_same_set(k, a, ref, f"signal {b} dims {wl.dims[b]}")
        assert int(out.iters[b]) == ref.iters, f"iterations {int(out.iters[b])} vs oracle {ref.iters}"
        assert int(out.status[b]) == ref.status


@pytest.mark.parametrize("fft_path,gather_mode", [(1, 0), (2, 1), (2, 3), (2, 4), (2, 5), (3, 0)])
def test_decoded_stop_matches_the_oracle_on_every_kernel_path(fft_path, gather_mode):
    """early_stop = 2 (stop after an iteration whose line-0 T0 bins were all decoded): same sets,
    iteration counts and status as the oracle under the same reading, on every kernel path, one
    iteration earlier than the first reading on noiseless signals."""
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("uneven_2d", batch=24)
    for es in (1, 2):
        p = configs.params_for(wl, early_stop=es, fft_path=fft_path, gather_mode=gather_mode)
        plan = Plan(wl.dims, p)
        out = plan.recover(*to_dev(wl))
        torch.cuda.synchronize()
        for b in range(wl.batch):
            T = int(plan.T[b])
            ref = O.recover(wl.cube(b), wl.alpha[b, :T], wl.tau[b, :T], oracle_params(p, T))
            k, a = out.signal(b)
            assert_same_set(k, a, ref, f"early_stop {es} path {fft_path} signal {b}")
            assert int(out.iters[b]) == ref.iters and int(out.status[b]) == ref.status
        plan.close()


def test_recover_full_uneven_batch_sampled_against_oracle():
    """4096 uneven 2-D signals in the launch configuration the benchmark times; 40 sampled signals
    against the oracle, every signal against its planted spectrum."""
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("uneven_2d")
    p = configs.params_for(wl)
    plan = Plan(wl.dims, p)
    cubes, offs, al, ta = to_dev(wl)
    out = plan.recover(cubes, offs, al, ta)
    torch.cuda.synchronize()
    ks, as_, cnt = out.k.cpu().numpy(), out.a.cpu().numpy(), out.count.cpu().numpy()
    rng = np.random.default_rng(0)
    for b in rng.choice(wl.batch, 40, replace=False):
        T = int(plan.T[b])
        ref = O.recover(wl.cube(b), wl.alpha[b, :T], wl.tau[b, :T], oracle_params(p, T))
        assert_same_set(ks[b, :cnt[b]].astype(np.int64), as_[b, :cnt[b]].astype(np.complex128), ref, f"signal {b}")
        assert int(out.iters[b]) == ref.iters
    ok = 0
    for b in range(wl.batch):
        dims = tuple(int(v) for v in wl.dims[b])
        truth = np.sort(O.linear_index(wl.k_true[b], dims))
        got = O.linear_index(ks[b, :cnt[b]].astype(np.int64), dims)
        ok += int(np.array_equal(got, truth))
    assert ok / wl.batch >= 0.999, f"exact-support success {ok}/{wl.batch}"
    assert np.all(out.status.cpu().numpy() == 0)


def test_synth_peel_and_adjoints_match_oracle():
    from paper_1711_11407_gb300.api import Plan
    wl = small_batch([(6, 10), (16, 24), (240, 256), (7, 11)], 8, K=lambda N: min(12, N // 2), T=3, snr_db=3.0)
    plan = Plan(wl.dims, configs.params_for(wl, k_cap=32))
    cubes, offs, al, ta = to_dev(wl)
    B, kc, D, Lm = wl.batch, plan.k_cap, wl.D, plan.L_max
    rng = np.random.default_rng(3)
    k = np.zeros((B, kc, D), np.int32)
    a = np.zeros((B, kc), np.complex64)
    cnt = np.zeros(B, np.int32)
    for b in range(B):
        n = min(len(wl.k_true[b]), kc)
        k[b, :n] = wl.k_true[b][:n]
        a[b, :n] = (rng.normal(size=n) + 1j * rng.normal(size=n)).astype(np.complex64)
        cnt[b] = n
    kd, ad, cd = torch.from_numpy(k).to(dev()), torch.from_numpy(a).to(dev()), torch.from_numpy(cnt).to(dev())
    syn = plan.synth(al, ta, kd, ad, cd).cpu().numpy()
    bins = plan.project(cubes, offs, al, ta)
    peeled = plan.synth(al, ta, kd, ad, cd, accumulate=-1, bins=bins.clone()).cpu().numpy()
    g = (rng.normal(size=(B, 3, D + 1, Lm)) + 1j * rng.normal(size=(B, 3, D + 1, Lm))).astype(np.complex64)
    gd = torch.from_numpy(g).to(dev())
    grad_cube = plan.adjoint_project(gd, offs, al, ta, torch.zeros_like(cubes)).cpu().numpy()
    grad_a = plan.adjoint_synth(gd, al, ta, kd, cd).cpu().numpy()
    bins = bins.cpu().numpy()
    for b in range(B):
        L = int(plan.L[b])
        dims = tuple(int(v) for v in wl.dims[b])
        n = cnt[b]
        acc_cube = np.zeros(dims, np.complex128)
        acc_a = np.zeros(n, np.complex128)
        for s in range(3):
            ref = O.synth(k[b, :n], a[b, :n].astype(np.complex128), wl.alpha[b, s], wl.tau[b, s], dims)
            e = np.linalg.norm(syn[b, s, :, :L] - ref) / np.linalg.norm(ref)
            assert e <= BIN_TOL, f"synth rel L2 {e:.2e}"
            refp = O.project(wl.cube(b), wl.alpha[b, s], wl.tau[b, s]) - ref
            e = np.linalg.norm(peeled[b, s, :, :L] - refp) / np.linalg.norm(refp)
            assert e <= BIN_TOL, f"peel rel L2 {e:.2e}"
            gg = g[b, s, :, :L].astype(np.complex128)
            acc_cube += O.project_adjoint(gg, wl.alpha[b, s], wl.tau[b, s], dims)
            acc_a += O.synth_adjoint(gg, k[b, :n], wl.alpha[b, s], wl.tau[b, s], dims)
        o = int(wl.offsets[b])
        gc = grad_cube[o:o + int(np.prod(dims))].reshape(dims)
        e = np.linalg.norm(gc - acc_cube) / np.linalg.norm(acc_cube)
        assert e <= BIN_TOL, f"projection adjoint rel L2 {e:.2e}"
        e = np.linalg.norm(grad_a[b, :n] - acc_a) / np.linalg.norm(acc_a)
        assert e <= BIN_TOL, f"synthesis adjoint rel L2 {e:.2e}"
        # dot-product test on the GPU's own forward/adjoint pair
        lhs = np.vdot(g[b, :, :, :L].astype(np.complex128), bins[b, :, :, :L].astype(np.complex128))
        rhs = np.vdot(gc, wl.cube(b))
        assert abs(lhs - rhs) <= 1e-4 * abs(lhs)


def test_unfused_per_signal_form_equals_fused_kernel():
    from paper_1711_11407_gb300.api import Plan
    from paper_1711_11407_gb300.plain import PlainRecoverer
    wl = S.make_workload("uneven_2d", batch=12)
    p = configs.params_for(wl)
    plan = Plan(wl.dims, p)
    cubes, offs, al, ta = to_dev(wl)
    out = plan.recover(cubes, offs, al, ta)
    torch.cuda.synchronize()
    res = PlainRecoverer(p).recover(wl, cubes, al, ta, range(wl.batch))
    for b, (k, a, it, st) in enumerate(res):
        kf, af = out.signal(b)
        assert np.array_equal(k, kf) and np.allclose(a, af, rtol=AMP_TOL, atol=0)
        assert it == int(out.iters[b]) and st == int(out.status[b])


def test_resume_one_iteration_at_a_time_equals_one_run():
    """Checkpoint/resume: T single-iteration calls chained through init_count reach the same set."""
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("single_240x256")
    p = configs.params_for(wl)
    full = Plan(wl.dims, p)
    cubes, offs, al, ta = to_dev(wl)
    ref = full.recover(cubes, offs, al, ta)
    torch.cuda.synchronize()
    step = Plan(wl.dims, configs.params_for(wl, T=1))
    out = step.alloc_output()
    init = torch.zeros(1, dtype=torch.int32, device=dev())
    for t in range(int(ref.iters[0])):
        step.recover(cubes, offs, al[:, t:t + 1].contiguous(), ta[:, t:t + 1].contiguous(), out=out, init_count=init)
        init.copy_(out.count)
    torch.cuda.synchronize()
    k1, a1 = ref.signal(0)
    k2, a2 = out.signal(0)
    assert np.array_equal(k1, k2) and np.allclose(a1, a2, rtol=AMP_TOL, atol=0)


def test_teacher_forced_noisy_iterations_match_oracle():
    """Noisy 64^3 cube: feed the oracle's set before iteration t to both sides and compare what one
    iteration adds (decisions on noisy bins, compared one iteration at a time)."""
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("batched_64x64x64", batch=2)
    p = configs.params_for(wl, T=1)
    plan = Plan(wl.dims, p)
    cubes, offs, al, ta = to_dev(wl)
    for b in range(wl.batch):
        x = wl.cube(b)
        for t in (0, 3, 10):
            prev = O.recover(x, wl.alpha[b], wl.tau[b], oracle_params(p, t), T=t) if t else None
            init_k = prev.k if prev is not None else np.zeros((0, 3), np.int64)
            init_a = prev.a if prev is not None else np.zeros(0, np.complex128)
            nxt = O.recover(x, wl.alpha[b, t:t + 1], wl.tau[b, t:t + 1], oracle_params(p, 1), init=(init_k, init_a), T=1)
            out = plan.alloc_output()
            n0 = init_k.shape[0]
            kk = np.zeros((wl.batch, plan.k_cap, 3), np.int32)
            aa = np.zeros((wl.batch, plan.k_cap), np.complex64)
            kk[b, :n0] = init_k
            aa[b, :n0] = init_a
            out.k.copy_(torch.from_numpy(kk))
            out.a.copy_(torch.from_numpy(aa))
            init = torch.zeros(wl.batch, dtype=torch.int32, device=dev())
            init[b] = n0
            plan.recover(cubes, offs, al[:, t:t + 1].contiguous(), ta[:, t:t + 1].contiguous(), out=out, init_count=init)
            torch.cuda.synchronize()
            k, a = out.signal(b)
            assert np.array_equal(k, nxt.k), f"teacher-forced iteration {t} of cube {b}: support differs"
            assert np.allclose(a, nxt.a, rtol=1e-3, atol=0)


def test_capacity_overflow_reports_status_and_keeps_k_cap_entries():
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("single_128x128")
    p = configs.params_for(wl, k_cap=8)
    plan = Plan(wl.dims, p)
    out = plan.recover(*to_dev(wl))
    torch.cuda.synchronize()
    ref = O.recover(wl.cube(0), wl.alpha[0], wl.tau[0], oracle_params(p, p.T))
    assert int(out.status[0]) == O.STATUS_CAPACITY == ref.status
    assert int(out.count[0]) == ref.k.shape[0] == 8
    assert int(out.iters[0]) == ref.iters


def test_recover_host_buffers_equal_device_buffers():
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("uneven_2d", batch=64)
    p = configs.params_for(wl)
    plan = Plan(wl.dims, p)
    dv = plan.recover(*to_dev(wl))
    torch.cuda.synchronize()
    for _ in range(2):
        hv = plan.recover_host(wl.cubes, wl.offsets, wl.alpha, wl.tau)
        assert torch.equal(hv.count, dv.count.cpu()) and torch.equal(hv.iters, dv.iters.cpu())
        for b in range(wl.batch):
            n = int(hv.count[b])
            assert torch.equal(hv.k[b, :n], dv.k[b, :n].cpu())
            assert torch.allclose(hv.a[b, :n], dv.a[b, :n].cpu(), rtol=AMP_TOL, atol=0)


@pytest.mark.parametrize("pinned", [True, False])
def test_recover_host_reading_pinned_cubes_in_place_equals_device_buffers(pinned):
    """host_cubes = 1: pinned cubes are read in place over the host link (nothing of them copied);
    pageable cubes are copied as before.  Either way the sets equal the device run's, on two calls
    in a row (the second reuses the plan's staging)."""
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("uneven_2d", batch=64)
    p = configs.params_for(wl, host_cubes=1)
    plan = Plan(wl.dims, p)
    dv = plan.recover(*to_dev(wl))
    torch.cuda.synchronize()
    cubes = torch.from_numpy(wl.cubes)
    if pinned:
        cubes = cubes.pin_memory()
    for _ in range(2):
        hv = plan.recover_host(cubes, wl.offsets, wl.alpha, wl.tau)
        assert torch.equal(hv.count, dv.count.cpu()) and torch.equal(hv.iters, dv.iters.cpu())
        for b in range(wl.batch):
            n = int(hv.count[b])
            assert torch.equal(hv.k[b, :n], dv.k[b, :n].cpu())
            assert torch.allclose(hv.a[b, :n], dv.a[b, :n].cpu(), rtol=AMP_TOL, atol=0)


def test_empty_batch_is_a_no_op():
    from paper_1711_11407_gb300.api import Plan
    plan = Plan(np.zeros((0, 2), np.int64))
    e = torch.zeros(0, dtype=torch.complex64, device=dev())
    z = torch.zeros((0, plan.T_max, 2), dtype=torch.int32, device=dev())
    out = plan.recover(e, torch.zeros(0, dtype=torch.int64, device=dev()), z, z)
    torch.cuda.synchronize()
    assert out.count.numel() == 0


def test_plans_of_different_sizes_coexist():
    """A later plan with shorter lines must not lower the shared-memory limit of an earlier plan's
    kernels (the limit is per kernel, shared by all plans)."""
    from paper_1711_11407_gb300.api import Plan
    big = S.make_workload("single_240x256")
    small = small_batch([(8, 8)], 2, K=lambda N: 2, T=3)
    p_big = Plan(big.dims, configs.params_for(big))
    Plan(small.dims, configs.params_for(small, T=3, k_cap=8))
    cubes, offs, al, ta = to_dev(big)
    p_big.project(cubes, offs, al, ta)
    out = p_big.recover(cubes, offs, al, ta)
    torch.cuda.synchronize()
    ref = O.recover(big.cube(0), big.alpha[0], big.tau[0], oracle_params(configs.params_for(big), 12))
    k, a = out.signal(0)
    assert_same_set(k, a, ref)


@pytest.mark.parametrize("which", ["uneven_2d", "batched_64x64x64", "single_240x256"])
def test_certified_fp32_decisions_equal_fp64_decisions(which):
    """The default path decides T0..T2 in FP32 when the value is outside a guard band and in FP64
    otherwise; forcing FP64 everywhere must give bit-identical sets, counts and iterations."""
    from paper_1711_11407_gb300.api import Plan
    if which == "batched_64x64x64":
        wl = S.make_workload(which, batch=8, T=64)          # noisy: many bins near the thresholds
    elif which == "uneven_2d":
        wl = S.make_workload(which, batch=256)
    else:
        wl = S.make_workload(which)
    outs = []
    for fp64 in (False, True):
        p = configs.params_for(wl, fp64_decisions=fp64)
        if which == "batched_64x64x64":
            p.T = 64
        plan = Plan(wl.dims, p)
        outs.append(plan.recover(*to_dev(wl)))
        torch.cuda.synchronize()
    a, b = outs
    assert torch.equal(a.count, b.count) and torch.equal(a.iters, b.iters) and torch.equal(a.status, b.status)
    assert torch.equal(a.k, b.k)
    # amplitudes carry the rounding of the peel's float atomics, whose order varies between runs
    assert torch.allclose(a.a, b.a, rtol=1e-5, atol=0)


@pytest.mark.parametrize("case", ["uneven_2d", "D1_L64", "D3_32cubed", "D2_256", "D4_L32"])
def test_register_fft_path_equals_shared_memory_path(case):
    """One warp per line with a register FFT (fft_path 2) against one CTA per signal with the
    shared-memory mixed-radix FFT (fft_path 1): same sets, counts and iterations; both against the
    oracle on a few signals."""
    from paper_1711_11407_gb300.api import Plan
    if case == "uneven_2d":
        wl = S.make_workload("uneven_2d", batch=128)
        T = None
    else:
        shapes = {"D1_L64": [(64,)], "D3_32cubed": [(32, 32, 32)], "D2_256": [(256, 128), (16, 256)],
                  "D4_L32": [(4, 8, 2, 32)]}[case]
        wl = small_batch(shapes, 8, K=lambda N: max(2, min(40, N // 64)), T=12)
        T = 12
    outs = []
    for path, gm in ((1, 1), (2, 1), (2, 3)):
        p = configs.params_for(wl, fft_path=path, gather_mode=gm, k_cap=512)
        if T is not None:
            p.T = T
        plan = Plan(wl.dims, p)
        assert plan.info["fft_path"] == path and plan.info["prefetch"] == (gm == 3)
        outs.append(plan.recover(*to_dev(wl)))
        torch.cuda.synchronize()
    a = outs[0]
    for b in outs[1:]:
        assert torch.equal(a.count, b.count) and torch.equal(a.iters, b.iters) and torch.equal(a.status, b.status)
        for i in range(wl.batch):
            n = int(a.count[i])
            assert torch.equal(a.k[i, :n], b.k[i, :n])
            assert torch.allclose(a.a[i, :n], b.a[i, :n], rtol=AMP_TOL, atol=0)
    for i in range(min(4, wl.batch)):
        Ti = int(wl.T[i]) if T is None else T
        ref = O.recover(wl.cube(i), wl.alpha[i, :Ti], wl.tau[i, :Ti], oracle_params(p, Ti))
        k, aa = b.signal(i)
        assert_same_set(k, aa, ref, f"signal {i}")


@pytest.mark.parametrize("name,batch", [("uneven_2d", 256), ("single_240x256", None), ("sparse_image_512x576", 2)])
def test_autotuned_launch_computes_the_same_sets(name, batch):
    """The tuned launch (kernel path, gather, CTA size and, for the long lines, the FFT's radix plan)
    recovers what the default launch recovers."""
    from paper_1711_11407_gb300 import autotune
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload(name, batch=batch)
    p = configs.params_for(wl)
    t = to_dev(wl)
    best, timings = autotune.tune(wl.dims, p, *t, reps=2, cache_path=None)
    assert len(timings) >= 2
    if name != "uneven_2d":
        assert any("radix_plan" in d for d in timings), f"no radix plan was timed: {sorted(timings)}"
    ref = Plan(wl.dims, p).recover(*t)
    got = Plan(wl.dims, best).recover(*t)
    torch.cuda.synchronize()
    assert torch.equal(ref.count, got.count) and torch.equal(ref.iters, got.iters)
    for b in range(wl.batch):
        n = int(ref.count[b])
        assert torch.equal(ref.k[b, :n], got.k[b, :n])
        assert torch.allclose(ref.a[b, :n], got.a[b, :n], rtol=AMP_TOL, atol=0)


@pytest.mark.parametrize("fft_path", [1, 3])
def test_prime_line_lengths_match_the_oracle(fft_path):
    """A line length that is a large prime (1009) or has one (2 x 509, 97 x 101 = 9797): the generic
    radix stage, one work item per output, gives the oracle's line DFTs and sets."""
    from paper_1711_11407_gb300 import _lib
    from paper_1711_11407_gb300.api import Plan
    for shapes in ([(1009, 1009)], [(509, 2, 2)], [(97, 101)]):
        wl = small_batch(shapes, 2, K=lambda N: 20, T=6, seed=23)
        p = configs.params_for(wl, T=6, k_cap=64, fft_path=fft_path)
        try:
            plan = Plan(wl.dims, p)
        except _lib.FpssftError as e:                    # 9797-point lines exceed one CTA (path 3)
            assert fft_path == 3 and e.status == _lib.ERR_UNSUPPORTED
            continue
        t = to_dev(wl)
        out = plan.recover(*t)
        try:                                             # the projection needs the lines in shared memory
            bins = plan.project(t[0], t[1], t[2][:, :1].contiguous(), t[3][:, :1].contiguous()).cpu().numpy()
        except _lib.FpssftError as e:
            assert e.status == _lib.ERR_UNSUPPORTED
            bins = None
        torch.cuda.synchronize()
        for b in range(wl.batch):
            L = int(plan.L[b])
            if bins is not None:
                ref = O.project(wl.cube(b), wl.alpha[b, 0], wl.tau[b, 0])
                for j in range(wl.D + 1):
                    e = np.linalg.norm(bins[b, 0, j, :L] - ref[j]) / np.linalg.norm(ref[j])
                    assert e <= BIN_TOL, f"L = {L}: line bins rel L2 {e:.2e}"
            ref = O.recover(wl.cube(b), wl.alpha[b], wl.tau[b], oracle_params(p, 6))
            k, a = out.signal(b)
            assert_same_set(k, a, ref, f"L = {L} path {fft_path} signal {b}")
            assert int(out.iters[b]) == ref.iters
        plan.close()


@pytest.mark.parametrize("radix_plan", [1, 2, 3])
@pytest.mark.parametrize("fft_path", [1, 3])
def test_every_radix_plan_matches_the_oracle(radix_plan, fft_path):
    """Each radix plan of the shared-memory FFT (stage orders and radix splits of L = 3840, 1440,
    1024 and 360) gives the oracle's line DFTs and recovered sets."""
    from paper_1711_11407_gb300.api import Plan
    wl = small_batch([(240, 256), (96, 120), (32, 1024), (40, 72)], 4, K=lambda N: 24, T=8, seed=17, snr_db=None)
    p = configs.params_for(wl, T=8, k_cap=64, fft_path=fft_path, radix_plan=radix_plan)
    plan = Plan(wl.dims, p)
    t = to_dev(wl)
    out = plan.recover(*t)
    bins = plan.project(t[0], t[1], t[2][:, :2].contiguous(), t[3][:, :2].contiguous()).cpu().numpy()
    torch.cuda.synchronize()
    for b in range(wl.batch):
        L = int(plan.L[b])
        for s in range(2):
            ref = O.project(wl.cube(b), wl.alpha[b, s], wl.tau[b, s])
            for j in range(wl.D + 1):
                e = np.linalg.norm(bins[b, s, j, :L] - ref[j]) / np.linalg.norm(ref[j])
                assert e <= BIN_TOL, f"radix plan {radix_plan}: line bins rel L2 {e:.2e}, dims {wl.dims[b]}"
        ref = O.recover(wl.cube(b), wl.alpha[b], wl.tau[b], oracle_params(p, 8))
        k, a = out.signal(b)
        assert_same_set(k, a, ref, f"radix plan {radix_plan} path {fft_path} dims {wl.dims[b]}")
        assert int(out.iters[b]) == ref.iters


def test_1024_thread_cta_equals_512_thread_cta_and_oracle():
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("single_240x256")
    outs = []
    for th in (512, 1024):
        p = configs.params_for(wl, fft_path=1, threads=th)
        plan = Plan(wl.dims, p)
        assert plan.info["threads"] == th
        outs.append(plan.recover(*to_dev(wl)))
        torch.cuda.synchronize()
    a, b = outs
    assert torch.equal(a.count, b.count) and torch.equal(a.iters, b.iters)
    n = int(a.count[0])
    assert torch.equal(a.k[0, :n], b.k[0, :n]) and torch.allclose(a.a[0, :n], b.a[0, :n], rtol=AMP_TOL, atol=0)
    ref = O.recover(wl.cube(0), wl.alpha[0], wl.tau[0], oracle_params(configs.params_for(wl), 12))
    k, aa = b.signal(0)
    assert_same_set(k, aa, ref)


@pytest.mark.parametrize("K,block", [(256, 0), (1280, 0), (1278, 3)])
def test_fig2_trials_on_gpu_equal_the_oracle_trial_by_trial(K, block):
    """The paper's Fig. 2 setting (256 x 256, T_max = 85): every trial's outcome and iteration count
    on the GPU equals the oracle's."""
    from paper_1711_11407_gb300 import fig2
    trials = 12
    r = fig2.run_point(K, block, trials=trials, seed=7)
    for t in range(trials):
        k, a, x, _, al, ta = S.make_signal(np.random.SeedSequence([7, K, block, t]), (256, 256), K, fig2.T_MAX, block=block)
        ref = O.recover(x.astype(np.complex64).astype(np.complex128), al, ta,
                        O.Params(T=fig2.T_MAX, k_cap=2 * K + 64))
        truth = np.sort(k[:, 0] * 256 + k[:, 1])
        ok = ref.k.shape[0] == K and np.array_equal(ref.k[:, 0] * 256 + ref.k[:, 1], truth)
        assert r["per_trial_success"][t] == ok, f"trial {t}"
        assert r["iters"][t] == ref.iters, f"trial {t}: iterations {r['iters'][t]} vs oracle {ref.iters}"


def test_long_lines_and_large_sets_use_global_workspace_and_match_oracle():
    """512 x 576 (L = 4608, the size of the paper's Fig. 3 image, K = 8411) and a 240 x 256 signal
    with a 20000-entry set: both exceed one CTA's shared memory, so the plan keeps lines and set in
    global workspace; the recovered sets equal the oracle's."""
    from paper_1711_11407_gb300.api import Plan
    for wl, kcap in ((S.make_workload("sparse_image_512x576", batch=2), 20000),
                     (S.make_workload("single_240x256"), 20000)):
        p = configs.params_for(wl, k_cap=kcap, fft_path=1)
        plan = Plan(wl.dims, p)
        assert plan.info["global_workspace"] == 1 and plan.info["fft_path"] == 1
        out = plan.recover(*to_dev(wl))
        torch.cuda.synchronize()
        for b in range(wl.batch):
            T = int(plan.T[b])
            ref = O.recover(wl.cube(b), wl.alpha[b, :T], wl.tau[b, :T], oracle_params(p, T))
            k, a = out.signal(b)
            assert_same_set(k, a, ref, f"{wl.name} signal {b}")
            assert int(out.iters[b]) == ref.iters


def test_unfused_steps_reject_sets_larger_than_shared_memory():
    """fpssft_decode / fpssft_finalize keep one signal's set in one CTA: with k_cap = 20000 they
    return FPSSFT_ERR_UNSUPPORTED before launching anything, and the fused recovery still works."""
    from paper_1711_11407_gb300 import _lib
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("sparse_image_512x576", batch=1)
    plan = Plan(wl.dims, configs.params_for(wl, k_cap=20000, T=1))
    D, d = wl.D, dev()
    k = torch.zeros((1, plan.k_cap, D), dtype=torch.int32, device=d)
    a = torch.zeros((1, plan.k_cap), dtype=torch.complex64, device=d)
    count = torch.zeros(1, dtype=torch.int32, device=d)
    t0 = torch.zeros(1, dtype=torch.int32, device=d)
    status = torch.zeros(1, dtype=torch.int32, device=d)
    al = torch.from_numpy(wl.alpha[:, :1]).to(d).contiguous()
    ta = torch.from_numpy(wl.tau[:, :1]).to(d).contiguous()
    bins = torch.zeros((1, 1, D + 1, plan.L_max), dtype=torch.complex64, device=d)
    for call in (lambda: plan.decode(bins, al, ta, k, a, count, t0, status), lambda: plan.finalize(k, a, count)):
        with pytest.raises(_lib.FpssftError) as e:
            call()
        assert e.value.status == _lib.ERR_UNSUPPORTED
    cubes, offs, _, _ = to_dev(wl)
    out = plan.recover(cubes, offs, al, ta)
    torch.cuda.synchronize()
    assert int(out.status[0]) == 0 and int(out.iters[0]) == 1


def test_axis_schedule_stays_in_deadlock_where_random_slopes_recover():
    """Rows and columns only (the row/column SFT's lines, Sec. 2.1) against random slopes on the
    Fig. 1 deadlock instance and at K = 2 N0 on 256 x 256: the GPU matches the oracle either way."""
    import pins
    from paper_1711_11407_gb300.api import Plan
    dims, k, a, _ = pins.load_deadlock()
    x = S.synthesize_cube(dims, k, a).astype(np.complex64)
    d = dev()
    for policy, expect in (("axis", 0), ("uniform", 4)):
        al, ta = S.draw_schedule(np.random.default_rng(3), dims, 6, policy)
        plan = Plan(np.array([dims], np.int64), configs.params_for(S.make_workload("single_128x128"), T=6, k_cap=16))
        out = plan.recover(torch.from_numpy(x.reshape(-1)).to(d), torch.zeros(1, dtype=torch.int64, device=d),
                           torch.from_numpy(al[None]).to(d), torch.from_numpy(ta[None]).to(d))
        torch.cuda.synchronize()
        ref = O.recover(x.astype(np.complex128), al, ta, O.Params(T=6, k_cap=16))
        assert int(out.count[0]) == ref.k.shape[0] == expect, policy
    ok = {}
    for policy in ("axis", "uniform"):
        wl = S.make_workload("uneven_2d", batch=6, shapes=[(256, 256)], K=lambda N: 512, T=85, policy=policy)
        p = configs.params_for(wl, T=85, k_cap=1100)
        out = Plan(wl.dims, p).recover(*to_dev(wl))
        torch.cuda.synchronize()
        ok[policy] = 0
        for b in range(wl.batch):
            ref = O.recover(wl.cube(b), wl.alpha[b], wl.tau[b], oracle_params(p, 85))
            kk, aa = out.signal(b)
            assert_same_set(kk, aa, ref, f"{policy} {b}")
            ok[policy] += int(kk.shape[0] == 512)
    assert ok["axis"] == 0 and ok["uniform"] == 6


def test_recovery_reading_cubes_in_place_from_pinned_host_memory():
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("uneven_2d", batch=96)
    plan = Plan(wl.dims, configs.params_for(wl))
    cubes, offs, al, ta = to_dev(wl)
    ref = plan.recover(cubes, offs, al, ta)
    host = torch.from_numpy(wl.cubes).pin_memory()
    got = plan.recover_mapped(host, offs, al, ta)
    torch.cuda.synchronize()
    assert torch.equal(ref.count, got.count) and torch.equal(ref.iters, got.iters)
    for b in range(wl.batch):
        n = int(ref.count[b])
        assert torch.equal(ref.k[b, :n], got.k[b, :n])
        assert torch.allclose(ref.a[b, :n], got.a[b, :n], rtol=AMP_TOL, atol=0)
    with pytest.raises(ValueError):
        plan.recover_mapped(torch.from_numpy(wl.cubes), offs, al, ta)      # not pinned


def test_offsets_that_leave_the_cube_buffer_are_rejected_before_launch():
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("uneven_2d", batch=8)
    plan = Plan(wl.dims, configs.params_for(wl))
    cubes, offs, al, ta = to_dev(wl)
    bad = offs.clone()
    bad[-1] += 1
    with pytest.raises(ValueError):
        plan.recover(cubes, bad, al, ta)
    with pytest.raises(ValueError):
        plan.recover(cubes[:-1], offs, al, ta)
    plan.recover(cubes, offs, al, ta)
    torch.cuda.synchronize()


def test_amplitude_averaging_matches_oracle_teacher_forced_on_noisy_data():
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("uneven_2d", batch=4, shapes=[(64, 64)], K=lambda N: 20, T=4, snr_db=15.0)
    p = configs.params_for(wl, T=1, k_cap=64, amp_average=True)
    plan = Plan(wl.dims, p)
    cubes, offs, al, ta = to_dev(wl)
    for t in (0, 2):
        out = plan.alloc_output()
        init = torch.zeros(wl.batch, dtype=torch.int32, device=dev())
        prevs = []
        for b in range(wl.batch):
            prev = O.recover(wl.cube(b), wl.alpha[b], wl.tau[b], O.Params(T=t, k_cap=64, theta0=p.theta0, rho=p.rho,
                             eta=p.eta, amp_average=True), T=t) if t else None
            prevs.append(prev)
            if prev is not None:
                n0 = prev.k.shape[0]
                out.k[b, :n0] = torch.from_numpy(prev.k.astype(np.int32)).to(dev())
                out.a[b, :n0] = torch.from_numpy(prev.a.astype(np.complex64)).to(dev())
                init[b] = n0
        plan.recover(cubes, offs, al[:, t:t + 1].contiguous(), ta[:, t:t + 1].contiguous(), out=out, init_count=init)
        torch.cuda.synchronize()
        for b in range(wl.batch):
            pv = prevs[b]
            nxt = O.recover(wl.cube(b), wl.alpha[b, t:t + 1], wl.tau[b, t:t + 1],
                            O.Params(T=1, k_cap=64, theta0=p.theta0, rho=p.rho, eta=p.eta, amp_average=True),
                            init=(pv.k, pv.a) if pv is not None else None, T=1)
            k, a = out.signal(b)
            assert np.array_equal(k, nxt.k), f"iteration {t} signal {b}"
            assert np.allclose(a, nxt.a, rtol=1e-3, atol=0)


def _random_case(rng):
    D = int(rng.integers(1, 5))
    choices = [2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 16, 20, 24, 30, 32, 64]
    while True:
        dims = tuple(int(rng.choice(choices)) for _ in range(D))
        L = math.lcm(*dims)
        N = int(np.prod(dims))
        if L <= 2048 and N <= 65536 and N >= 4:
            break
    K = int(rng.integers(1, max(2, min(N // 3, L // 2)) + 1))
    return dims, K


@pytest.mark.parametrize("seed", range(32))
def test_random_shapes_match_oracle_on_every_kernel_path(seed):
    """Seeded random D, shapes (prime and mixed-radix line lengths), sparsity and budgets: every
    applicable kernel path recovers exactly the oracle's set."""
    from paper_1711_11407_gb300.api import Plan
    from paper_1711_11407_gb300 import _lib
    rng = np.random.default_rng(1000 + seed)
    dims, K = _random_case(rng)
    T = int(rng.integers(3, 16))
    wl = small_batch([dims], 3, K=lambda N: K, T=T, seed=2000 + seed)
    refs = {}
    # the last entry forces the cluster path's set into global workspace (k_cap beyond shared memory)
    for path, gm, kcap in ((1, 1, 2 * K + 8), (1, 3, 2 * K + 8), (2, 1, 2 * K + 8), (2, 4, 2 * K + 8), (2, 5, 2 * K + 8),
                           (3, 1, 2 * K + 8), (3, 3, 2 * K + 8), (3, 1, 16000)):
        p = configs.params_for(wl, T=T, k_cap=kcap, fft_path=path, gather_mode=gm)
        try:
            plan = Plan(wl.dims, p)
        except _lib.FpssftError as e:
            assert path == 2 and e.status == _lib.ERR_UNSUPPORTED     # register path needs L in 32..256
            continue
        out = plan.recover(*to_dev(wl))
        torch.cuda.synchronize()
        for b in range(wl.batch):
            # k_cap > K on every path, so no set overflows and the oracle's result is the same for all
            if b not in refs:
                refs[b] = O.recover(wl.cube(b), wl.alpha[b], wl.tau[b], oracle_params(p, T))
            ref = refs[b]
            k, a = out.signal(b)
            assert_same_set(k, a, ref, f"dims {dims} K {K} path {path} gather {gm} k_cap {kcap} signal {b}")
            assert int(out.iters[b]) == ref.iters and int(out.status[b]) == ref.status


@pytest.mark.parametrize("fft_path,k_cap", [(1, 64), (2, 64), (3, 64), (3, 16000)])
def test_redecoded_frequencies_accumulate_their_residual_like_the_oracle(fft_path, k_cap):
    """Reading A9 on every kernel path (and the cluster path's set in global workspace): resumed
    from the planted support with every amplitude off by delta, the next iteration decodes each
    residual -delta at the same frequency and adds it, giving the oracle's set, which is the planted
    spectrum; keeping or replacing the old amplitude would leave delta or -delta."""
    from paper_1711_11407_gb300.api import Plan
    wl = small_batch([(32, 64)], 3, K=lambda N: 12, T=8, seed=11)    # L = 64: every path applies
    # the first stop reading, so that the iteration after the residuals' decode is run and compared too
    p = configs.params_for(wl, T=8, k_cap=k_cap, fft_path=fft_path, early_stop=1)
    plan = Plan(wl.dims, p)
    assert plan.info["fft_path"] == fft_path
    cubes, offs, al, ta = to_dev(wl)
    rng = np.random.default_rng(11)
    kk = np.zeros((wl.batch, plan.k_cap, 2), np.int32)
    aa = np.zeros((wl.batch, plan.k_cap), np.complex64)
    counts = np.zeros(wl.batch, np.int32)
    inits = []
    for b in range(wl.batch):
        k = np.asarray(wl.k_true[b], np.int64)
        a0 = (np.asarray(wl.a_true[b]) + 0.1 * np.exp(2j * np.pi * rng.random(len(k)))).astype(np.complex64)
        kk[b, :len(k)] = k
        aa[b, :len(k)] = a0
        counts[b] = len(k)
        inits.append((k, a0.astype(np.complex128)))
    out = plan.alloc_output()
    out.k.copy_(torch.from_numpy(kk))
    out.a.copy_(torch.from_numpy(aa))
    plan.recover(cubes, offs, al, ta, out=out, init_count=torch.from_numpy(counts).to(dev()))
    torch.cuda.synchronize()
    for b in range(wl.batch):
        ref = O.recover(wl.cube(b), wl.alpha[b], wl.tau[b], oracle_params(p, 8), init=inits[b])
        k, a = out.signal(b)
        assert_same_set(k, a, ref, f"path {fft_path} k_cap {k_cap} signal {b}")
        assert int(out.iters[b]) == ref.iters >= 2 and int(out.status[b]) == 0
        order = np.argsort(O.linear_index(np.asarray(wl.k_true[b], np.int64), tuple(int(v) for v in wl.dims[b])))
        assert np.allclose(ref.a, np.asarray(wl.a_true[b])[order], atol=1e-5)
    plan.close()


@pytest.mark.parametrize("fp64", [0, 1])
def test_decode_rejects_a_bin_that_decodes_off_its_bin(fp64):
    """T3 on the GPU with bins made by hand (the oracle pin's case): the values of k = (1, 1) on an
    8 x 8 grid with slope (1, 3) and offset (3, 5) decode to k and a in k's own bin 4, and the same
    values placed in bin 0 pass T0-T2 but are rejected; FP32-certified and FP64 decisions alike."""
    from paper_1711_11407_gb300.api import Params, Plan
    dims, alpha, tau, k, a = (8, 8), (1, 3), (3, 5), (1, 1), 0.8 * np.exp(0.7j)
    s0 = a * np.exp(2j * np.pi * (k[0] * tau[0] + k[1] * tau[1]) / 8)
    vals = np.asarray([s0, s0 * np.exp(2j * np.pi * k[0] / 8), s0 * np.exp(2j * np.pi * k[1] / 8)])
    plan = Plan(np.asarray([dims, dims], np.int64), Params(T=1, k_cap=8, fp64_decisions=fp64))
    bins = np.zeros((2, 1, 3, plan.L_max), np.complex64)
    bins[0, 0, :, 4] = vals
    bins[1, 0, :, 0] = vals
    d = dev()
    al = torch.tensor([[alpha], [alpha]], dtype=torch.int32, device=d)
    ta = torch.tensor([[tau], [tau]], dtype=torch.int32, device=d)
    kk = torch.zeros((2, plan.k_cap, 2), dtype=torch.int32, device=d)
    aa = torch.zeros((2, plan.k_cap), dtype=torch.complex64, device=d)
    count = torch.zeros(2, dtype=torch.int32, device=d)
    t0 = torch.zeros(2, dtype=torch.int32, device=d)
    status = torch.zeros(2, dtype=torch.int32, device=d)
    plan.decode(torch.from_numpy(bins).to(d), al, ta, kk, aa, count, t0, status)
    torch.cuda.synchronize()
    assert t0.tolist() == [1, 1] and status.tolist() == [0, 0]
    assert count.tolist() == [1, 0], "the bin whose decoded k lies on another bin must be rejected (T3)"
    assert tuple(kk[0, 0].tolist()) == k and abs(complex(aa[0, 0].item()) - a) < 1e-5
    ref, n0 = O.classify_decode(bins[0, 0].astype(np.complex128), alpha, tau, dims, O.Params(T=1, k_cap=8))
    assert n0 == 1 and len(ref) == 1 and ref[0][1] == k
    plan.close()


@pytest.mark.parametrize("fp64", [0, 1])
def test_decode_applies_magnitude_and_grid_tolerances_like_the_oracle(fp64):
    """T1 and T2 on the GPU with the oracle pin's hand-made bins: a line phase 0.3 of a grid step
    off (eta = 0.05) or a line magnitude 1 % off (rho = 1e-3) rejects the bin, 0.02 of a step or
    0.05 % decodes it; one signal per case, FP32-certified and FP64 decisions alike."""
    import pins
    from paper_1711_11407_gb300.api import Params, Plan
    cases = pins.sparsity_test_bins()
    B = len(cases)
    plan = Plan(np.asarray([(8, 8)] * B, np.int64), Params(T=1, k_cap=8, fp64_decisions=fp64))
    bins = np.zeros((B, 1, 3, plan.L_max), np.complex64)
    for b, (_, bb, _) in enumerate(cases):
        bins[b, 0, :, :8] = bb
    d = dev()
    al = torch.tensor([[(1, 3)]] * B, dtype=torch.int32, device=d)
    ta = torch.tensor([[(3, 5)]] * B, dtype=torch.int32, device=d)
    kk = torch.zeros((B, plan.k_cap, 2), dtype=torch.int32, device=d)
    aa = torch.zeros((B, plan.k_cap), dtype=torch.complex64, device=d)
    count = torch.zeros(B, dtype=torch.int32, device=d)
    t0 = torch.zeros(B, dtype=torch.int32, device=d)
    status = torch.zeros(B, dtype=torch.int32, device=d)
    plan.decode(torch.from_numpy(bins).to(d), al, ta, kk, aa, count, t0, status)
    torch.cuda.synchronize()
    p = O.Params(T=1, k_cap=8, theta0=1e-3, rho=1e-3, eta=0.05)
    for b, (name, _, accept) in enumerate(cases):
        ref, n0 = O.classify_decode(bins[b, 0, :, :8].astype(np.complex128), (1, 3), (3, 5), (8, 8), p)
        assert int(t0[b]) == n0 == 1 and int(status[b]) == 0, name
        assert int(count[b]) == len(ref) == (1 if accept else 0), name
        if accept:
            assert tuple(kk[b, 0].tolist()) == ref[0][1] == (1, 1), name
    plan.close()


def test_register_path_library_choice_stages_resident_batches_only():
    """gather_mode 0 on the register path: a batch the staged-prefetch kernel holds resident at once
    gets the cp.async prefetch, a larger one none; either way the sets are those of the explicit
    modes and, on a sample, the oracle's."""
    from paper_1711_11407_gb300.api import Plan
    small = S.make_workload("uneven_2d", batch=64)
    large = S.make_workload("uneven_2d", batch=4096, shapes=[(64, 64)])
    for wl, staged in ((small, True), (large, False)):
        p = configs.params_for(wl)
        plan = Plan(wl.dims, p)
        assert plan.info["fft_path"] == 2 and plan.info["prefetch"] == (1 if staged else 0)
        out = plan.recover(*to_dev(wl))
        explicit = Plan(wl.dims, configs.params_for(wl, gather_mode=3 if staged else 4))
        ref = explicit.recover(*to_dev(wl))
        torch.cuda.synchronize()
        assert torch.equal(out.count, ref.count) and torch.equal(out.iters, ref.iters)
        for b in range(wl.batch):
            n = int(out.count[b])
            assert torch.equal(out.k[b, :n], ref.k[b, :n])
            assert torch.allclose(out.a[b, :n], ref.a[b, :n], rtol=AMP_TOL, atol=0)
        for b in (0, wl.batch - 1):
            T = int(plan.T[b])
            o = O.recover(wl.cube(b), wl.alpha[b, :T], wl.tau[b, :T], oracle_params(p, T))
            k, a = out.signal(b)
            assert_same_set(k, a, o, f"signal {b}")
        plan.close()
        explicit.close()


def test_persistent_launches_replayed_back_to_back_give_the_same_sets():
    """More signals than resident CTAs, so every CTA claims several signals from the plan's work
    counter; the launch leaves that counter at zero for the next one (no reset is enqueued), so
    replaying the same launch from a CUDA graph gives the first launch's sets every time."""
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("uneven_2d", batch=3000, shapes=[(64, 64), (128, 128)])
    plan = Plan(wl.dims, configs.params_for(wl))
    assert plan.info["grid"] < wl.batch
    args = to_dev(wl)
    first = plan.recover(*args)
    torch.cuda.synchronize()
    keep = {f: getattr(first, f).clone() for f in ("k", "a", "count", "iters", "status")}
    out = plan.alloc_output(torch.device("cuda:0"))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.recover(*args, out=out, stream=s)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            plan.recover(*args, out=out, stream=s)
    for _ in range(3):
        out.count.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out.count, keep["count"]) and torch.equal(out.iters, keep["iters"])
        assert torch.equal(out.status, keep["status"])
        for b in range(0, wl.batch, 97):
            n = int(keep["count"][b])
            assert torch.equal(out.k[b, :n], keep["k"][b, :n])
    plan.close()
