"""The cluster recovery path (fft_path 3: one CTA per line, a thread-block cluster of D+1 CTAs per
signal exchanging bins through distributed shared memory) against the FP64 oracle, through the
C ABI (needs a GB300).  Same tolerances as the other parity tests: supports, iteration counts and
statuses exact; amplitudes within 1e-4 relative per entry."""
import numpy as np
import pytest
import torch

from oracle import fpssft_oracle as O
from paper_1711_11407_gb300 import configs
from paper_1711_11407_gb300 import synth as S

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-4


def dev():
    return torch.device("cuda:0")


def to_dev(wl):
    d = dev()
    return (torch.from_numpy(wl.cubes).to(d), torch.from_numpy(wl.offsets).to(d),
            torch.from_numpy(wl.alpha).to(d), torch.from_numpy(wl.tau).to(d))


def oracle_params(p, T):
    return O.Params(T=T, k_cap=p.k_cap, theta0=p.theta0, rho=p.rho, eta=p.eta, early_stop=p.early_stop,
                    amp_average=p.amp_average)


def assert_same_set(k, a, ref, ctx=""):
    assert k.shape == ref.k.shape and np.array_equal(k, ref.k), f"support differs from the oracle {ctx}"
    err = np.abs(a - ref.a)
    assert np.all(err <= AMP_TOL * np.maximum(np.abs(ref.a), 1e-30)), f"amplitude error {err.max()} {ctx}"


def small_batch(shapes, batch, K, T, seed=7, snr_db=None):
    return S.make_workload("uneven_2d", seed=seed, batch=batch, shapes=shapes, K=K, T=T, snr_db=snr_db)


CASES = {
    # name: (workload factory, T override or None, k_cap, threads, gather_mode)
    "D2_240x256_1024thr": (lambda: S.make_workload("single_240x256"), None, 640, 0, 1),
    "D2_240x256_256thr_prefetch": (lambda: S.make_workload("single_240x256"), None, 640, 256, 3),
    "D2_240x256_L2only": (lambda: S.make_workload("single_240x256"), None, 640, 512, 2),
    "D2_1024_noiseless": (lambda: S.make_workload("images_1024x1024", batch=3, snr_db=None), None, 4096, 0, 3),
    "D1_4096": (lambda: small_batch([(4096,), (3000,)], 4, K=lambda N: 40, T=8), 8, 128, 0, 1),
    "D3_24x32x40": (lambda: small_batch([(24, 32, 40)], 3, K=lambda N: 60, T=10), 10, 256, 0, 3),
    "D4_4x6x8x10": (lambda: small_batch([(4, 6, 8, 10)], 3, K=lambda N: 10, T=12), 12, 64, 128, 1),
    "D2_mixed_lengths": (lambda: small_batch([(30, 64), (48, 40), (7, 11), (100, 96)], 8,
                                             K=lambda N: max(1, N // 400), T=12), 12, 64, 0, 3),
}


def _run_case(case, cluster_set=0):
    from paper_1711_11407_gb300.api import Plan
    make, T, kcap, threads, gm = CASES[case]
    wl = make()
    kw = dict(k_cap=kcap, fft_path=3, threads=threads, gather_mode=gm, cluster_set=cluster_set)
    if T is not None:
        kw["T"] = T
    p = configs.params_for(wl, **kw)
    plan = Plan(wl.dims, p)
    assert plan.info["fft_path"] == 3
    assert plan.info["grid"] == wl.batch * (wl.D + 1)
    if threads:
        assert plan.info["threads"] == threads
    if cluster_set == 2:
        assert plan.info["global_workspace"] == 1
    out = plan.recover(*to_dev(wl))
    torch.cuda.synchronize()
    for b in range(wl.batch):
        Tb = int(plan.T[b])
        ref = O.recover(wl.cube(b), wl.alpha[b, :Tb], wl.tau[b, :Tb], oracle_params(p, Tb))
        k, a = out.signal(b)
        assert_same_set(k, a, ref, f"{case} signal {b} dims {wl.dims[b]}")
        assert int(out.iters[b]) == ref.iters, f"iterations {int(out.iters[b])} vs oracle {ref.iters}"
        assert int(out.status[b]) == ref.status


@pytest.mark.parametrize("case", sorted(CASES))
def test_cluster_path_matches_oracle(case):
    _run_case(case)


@pytest.mark.parametrize("case", ["D2_240x256_256thr_prefetch", "D2_1024_noiseless", "D3_24x32x40", "D4_4x6x8x10",
                                  "D2_mixed_lengths"])
def test_cluster_path_with_the_set_in_global_workspace_matches_oracle(case):
    """cluster_set 2: each signal's list and index in plan-owned global workspace (L2-resident)
    instead of shared memory; the oracle's sets, iteration counts and statuses."""
    _run_case(case, cluster_set=2)


def test_set_in_global_workspace_keeps_a_batch_larger_than_the_gpu_resident_and_equal():
    """More clusters than SMs (1024-point lines): with the sets in global workspace and 256-thread
    CTAs two CTAs share an SM and the whole batch is resident at once; the sets equal those of the
    library's shared-memory layout and, on a sample, the oracle's."""
    from paper_1711_11407_gb300.api import Plan
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    wl = S.make_workload("images_1024x1024", batch=sms // 3 + 2, snr_db=None)
    auto = Plan(wl.dims, configs.params_for(wl, fft_path=3, cluster_set=2, threads=256))
    assert auto.info["global_workspace"] == 1 and auto.info["threads"] == 256
    shared = Plan(wl.dims, configs.params_for(wl))
    assert shared.info["fft_path"] == 3 and shared.info["global_workspace"] == 0 and shared.info["threads"] == 512
    few = Plan(wl.dims[:8], configs.params_for(wl, fft_path=3, cluster_set=1))
    assert few.info["global_workspace"] == 0 and few.info["threads"] == 512
    args = to_dev(wl)
    a = auto.recover(*args)
    b = shared.recover(*args)
    torch.cuda.synchronize()
    assert torch.equal(a.count, b.count) and torch.equal(a.iters, b.iters) and torch.equal(a.status, b.status)
    for s in range(wl.batch):
        n = int(a.count[s])
        assert torch.equal(a.k[s, :n], b.k[s, :n])
        assert torch.allclose(a.a[s, :n], b.a[s, :n], rtol=AMP_TOL, atol=0)
    p = configs.params_for(wl)
    for s in (0, wl.batch - 1):
        Tb = int(auto.T[s])
        ref = O.recover(wl.cube(s), wl.alpha[s, :Tb], wl.tau[s, :Tb], oracle_params(p, Tb))
        k, aa = a.signal(s)
        assert_same_set(k, aa, ref, f"signal {s}")
    for pl in (auto, shared, few):
        pl.close()


def test_cluster_path_equals_the_one_cta_per_signal_path():
    """Same batch through fft_path 1 and 3: identical supports, counts and iterations."""
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("images_1024x1024", batch=4, snr_db=None)
    outs = []
    for path in (1, 3):
        plan = Plan(wl.dims, configs.params_for(wl, fft_path=path))
        outs.append(plan.recover(*to_dev(wl)))
        torch.cuda.synchronize()
    a, b = outs
    assert torch.equal(a.count, b.count) and torch.equal(a.iters, b.iters) and torch.equal(a.status, b.status)
    for s in range(wl.batch):
        n = int(a.count[s])
        assert torch.equal(a.k[s, :n], b.k[s, :n])
        assert torch.allclose(a.a[s, :n], b.a[s, :n], rtol=AMP_TOL, atol=0)


def test_cluster_path_amplitude_averaging_and_fp64_decisions():
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("single_240x256")
    p = configs.params_for(wl, fft_path=3, amp_average=True, fp64_decisions=True)
    out = Plan(wl.dims, p).recover(*to_dev(wl))
    torch.cuda.synchronize()
    ref = O.recover(wl.cube(0), wl.alpha[0], wl.tau[0], oracle_params(p, p.T))
    k, a = out.signal(0)
    assert_same_set(k, a, ref)
    assert int(out.iters[0]) == ref.iters


def test_cluster_path_resume_one_iteration_at_a_time_equals_one_run():
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("single_240x256")
    full = Plan(wl.dims, configs.params_for(wl, fft_path=3))
    cubes, offs, al, ta = to_dev(wl)
    ref = full.recover(cubes, offs, al, ta)
    torch.cuda.synchronize()
    step = Plan(wl.dims, configs.params_for(wl, T=1, fft_path=3))
    out = step.alloc_output()
    init = torch.zeros(1, dtype=torch.int32, device=dev())
    for t in range(int(ref.iters[0])):
        step.recover(cubes, offs, al[:, t:t + 1].contiguous(), ta[:, t:t + 1].contiguous(), out=out, init_count=init)
        init.copy_(out.count)
    torch.cuda.synchronize()
    k1, a1 = ref.signal(0)
    k2, a2 = out.signal(0)
    assert np.array_equal(k1, k2) and np.allclose(a1, a2, rtol=AMP_TOL, atol=0)


def test_cluster_path_capacity_overflow_reports_status_and_keeps_k_cap_entries():
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("single_128x128")
    p = configs.params_for(wl, k_cap=8, fft_path=3)
    out = Plan(wl.dims, p).recover(*to_dev(wl))
    torch.cuda.synchronize()
    ref = O.recover(wl.cube(0), wl.alpha[0], wl.tau[0], oracle_params(p, p.T))
    assert int(out.status[0]) == O.STATUS_CAPACITY == ref.status
    assert int(out.count[0]) == ref.k.shape[0] == 8
    assert int(out.iters[0]) == ref.iters


def test_cluster_path_teacher_forced_noisy_1024_images():
    """Noisy 1024 x 1024 images (5 dB): the oracle's set before iteration t is fed to both sides and
    what one iteration adds is compared (decisions on noisy bins, one iteration at a time)."""
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("images_1024x1024", batch=2)
    p = configs.params_for(wl, T=1, fft_path=3)
    plan = Plan(wl.dims, p)
    assert plan.info["fft_path"] == 3
    cubes, offs, al, ta = to_dev(wl)
    for t in (0, 4):
        out = plan.alloc_output()
        init = torch.zeros(wl.batch, dtype=torch.int32, device=dev())
        prevs = []
        for b in range(wl.batch):
            prev = O.recover(wl.cube(b), wl.alpha[b], wl.tau[b], oracle_params(p, t), T=t) if t else None
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
            nxt = O.recover(wl.cube(b), wl.alpha[b, t:t + 1], wl.tau[b, t:t + 1], oracle_params(p, 1),
                            init=(pv.k, pv.a) if pv is not None else None, T=1)
            k, a = out.signal(b)
            assert np.array_equal(k, nxt.k), f"teacher-forced iteration {t} of image {b}: support differs"
            assert np.allclose(a, nxt.a, rtol=1e-3, atol=0)


@pytest.mark.parametrize("case", ["sparse_image_512x576", "single_240x256", "D3_24x32x40"])
def test_cluster_path_with_the_set_in_global_workspace_matches_oracle(case):
    """Sets too large for shared memory (k_cap 20000): the cluster path keeps the lines in shared
    memory and the list, index and counter in global workspace; sets equal the oracle's."""
    from paper_1711_11407_gb300.api import Plan
    if case == "sparse_image_512x576":
        wl, T = S.make_workload("sparse_image_512x576", batch=2), None
    elif case == "single_240x256":
        wl, T = S.make_workload("single_240x256"), None
    else:
        wl, T = small_batch([(24, 32, 40)], 3, K=lambda N: 60, T=10), 10
    kw = dict(k_cap=20000, fft_path=3)
    if T is not None:
        kw["T"] = T
    p = configs.params_for(wl, **kw)
    plan = Plan(wl.dims, p)
    assert plan.info["fft_path"] == 3 and plan.info["global_workspace"] == 1
    out = plan.recover(*to_dev(wl))
    torch.cuda.synchronize()
    for b in range(wl.batch):
        Tb = int(plan.T[b])
        ref = O.recover(wl.cube(b), wl.alpha[b, :Tb], wl.tau[b, :Tb], oracle_params(p, Tb))
        k, a = out.signal(b)
        assert_same_set(k, a, ref, f"{case} signal {b}")
        assert int(out.iters[b]) == ref.iters and int(out.status[b]) == ref.status


def test_cluster_path_global_set_capacity_overflow():
    """K = 8411 frequencies with room for 8000 (a set still too large for shared memory): status
    FPSSFT_ERR_CAPACITY, 8000 entries kept, the oracle's iteration count."""
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("sparse_image_512x576", batch=1)
    p = configs.params_for(wl, k_cap=8000, fft_path=3)
    plan = Plan(wl.dims, p)
    assert plan.info["global_workspace"] == 1
    out = plan.recover(*to_dev(wl))
    torch.cuda.synchronize()
    T = int(plan.T[0])
    ref = O.recover(wl.cube(0), wl.alpha[0, :T], wl.tau[0, :T], oracle_params(p, T))
    assert int(out.status[0]) == O.STATUS_CAPACITY == ref.status
    assert int(out.iters[0]) == ref.iters
    assert int(out.count[0]) == ref.k.shape[0]


def test_cluster_path_global_set_resume_equals_one_run():
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("single_240x256")
    full = Plan(wl.dims, configs.params_for(wl, fft_path=3, k_cap=20000))
    assert full.info["global_workspace"] == 1
    cubes, offs, al, ta = to_dev(wl)
    ref = full.recover(cubes, offs, al, ta)
    torch.cuda.synchronize()
    step = Plan(wl.dims, configs.params_for(wl, T=1, fft_path=3, k_cap=20000))
    out = step.alloc_output()
    init = torch.zeros(1, dtype=torch.int32, device=dev())
    for t in range(int(ref.iters[0])):
        step.recover(cubes, offs, al[:, t:t + 1].contiguous(), ta[:, t:t + 1].contiguous(), out=out, init_count=init)
        init.copy_(out.count)
    torch.cuda.synchronize()
    k1, a1 = ref.signal(0)
    k2, a2 = out.signal(0)
    assert np.array_equal(k1, k2) and np.allclose(a1, a2, rtol=AMP_TOL, atol=0)


@pytest.mark.parametrize("kcap", [640, 20000])
def test_cluster_path_host_buffers_and_pinned_in_place_reads_equal_device_buffers(kcap):
    """fpssft_recover_host (host buffers copied in and out) and the in-place read of pinned host
    cubes give the device-buffer sets on the cluster path (set in shared memory and in global
    workspace)."""
    from paper_1711_11407_gb300.api import Plan
    wl = S.make_workload("single_240x256")
    plan = Plan(wl.dims, configs.params_for(wl, fft_path=3, k_cap=kcap))
    assert plan.info["fft_path"] == 3 and plan.info["global_workspace"] == (1 if kcap > 640 else 0)
    cubes, offs, al, ta = to_dev(wl)
    ref = plan.recover(cubes, offs, al, ta)
    torch.cuda.synchronize()
    hv = plan.recover_host(wl.cubes, wl.offsets, wl.alpha, wl.tau)
    mp = plan.recover_mapped(torch.from_numpy(wl.cubes).pin_memory(), offs, al, ta)
    torch.cuda.synchronize()
    n = int(ref.count[0])
    for got in (hv, mp):
        assert int(got.count[0]) == n and int(got.iters[0]) == int(ref.iters[0])
        assert torch.equal(got.k[0, :n].cpu(), ref.k[0, :n].cpu())
        assert torch.allclose(got.a[0, :n].cpu(), ref.a[0, :n].cpu(), rtol=AMP_TOL, atol=0)
