"""fpssft_recover_noalloc against fpssft_recover, through the C ABI (needs a GB300).

The no-allocation entry point serves callers that cannot allocate device memory when they recover
(code running under a memory pool or arena owned by someone else, inside regions where cudaMalloc
is forbidden or would synchronise, or within a fixed device-memory budget).  It keeps the tables a
plan would allocate in one fixed device array, so two calls in a row -- each overwriting what the
previous one left there -- must both reproduce the plan-based recovery."""
import ctypes
import dataclasses

import numpy as np
import pytest
import torch

from paper_1711_11407_gb300 import _lib, configs
from paper_1711_11407_gb300 import synth as S

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-4   # relative amplitude tolerance used by the parity tests


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _noalloc(lib, wl, p, dev_tensors, out, init_count=None):
    cubes, offs, al, ta = dev_tensors
    dims = np.ascontiguousarray(wl.dims.astype(np.int64))
    cp = p.c()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.fpssft_recover_noalloc(wl.D, wl.batch, dims.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cp),
                                      _ptr(cubes), _ptr(offs), _ptr(al), _ptr(ta), _ptr(init_count), _ptr(out.k),
                                      _ptr(out.a), _ptr(out.count), _ptr(out.iters), _ptr(out.status), stream)


def _same(ref, out):
    assert torch.equal(ref.count, out.count)
    assert torch.equal(ref.iters, out.iters)
    assert torch.equal(ref.status, out.status)
    for b in range(ref.count.numel()):
        n = int(ref.count[b])
        assert torch.equal(ref.k[b, :n], out.k[b, :n])
        assert torch.allclose(ref.a[b, :n], out.a[b, :n], rtol=AMP_TOL, atol=0)


def test_noalloc_entry_point_matches_plan_based_recovery_on_consecutive_calls():
    from paper_1711_11407_gb300.api import Plan
    lib = _lib.load()
    dev = torch.device("cuda:0")
    for name, batch in (("uneven_2d", 256), ("uneven_2d", 256), ("single_240x256", None)):
        wl = S.make_workload(name, batch=batch)
        p = configs.params_for(wl)
        plan = Plan(wl.dims, p)
        t = [torch.from_numpy(x).to(dev) for x in (wl.cubes, wl.offsets, wl.alpha, wl.tau)]
        ref = plan.recover(*t)
        out = plan.alloc_output(dev)
        out.k.fill_(-7)
        out.count.fill_(-1)
        st = _noalloc(lib, wl, p, t, out)
        assert st == _lib.OK, lib.fpssft_last_error().decode()
        torch.cuda.synchronize()
        _same(ref, out)
        plan.close()


def test_noalloc_results_equal_the_oracle_on_a_sample():
    """The same call checked against the FP64 oracle directly, on 6 signals of the uneven batch."""
    from oracle import fpssft_oracle as O
    lib = _lib.load()
    dev = torch.device("cuda:0")
    wl = S.make_workload("uneven_2d", batch=6)
    p = configs.params_for(wl)
    from paper_1711_11407_gb300.api import Plan
    plan = Plan(wl.dims, p)
    t = [torch.from_numpy(x).to(dev) for x in (wl.cubes, wl.offsets, wl.alpha, wl.tau)]
    out = plan.alloc_output(dev)
    assert _noalloc(lib, wl, p, t, out) == _lib.OK, lib.fpssft_last_error().decode()
    torch.cuda.synchronize()
    for b in range(wl.batch):
        T = int(wl.T[b])
        op = O.Params(T=T, k_cap=p.k_cap, theta0=p.theta0, rho=p.rho, eta=p.eta, early_stop=p.early_stop)
        ref = O.recover(wl.cube(b), wl.alpha[b, :T], wl.tau[b, :T], op)
        k, a = out.signal(b)
        assert np.array_equal(k, ref.k)
        assert np.all(np.abs(a - ref.a) <= AMP_TOL * np.abs(ref.a))
        assert int(out.iters[b]) == ref.iters
    plan.close()


def test_noalloc_resume_and_prefetch_match_plan_based_recovery():
    """init_count (resume from a given set) and gather_mode 3 (cp.async prefetch, a third line
    buffer in shared memory) through the no-allocation call against the plan path."""
    from paper_1711_11407_gb300.api import Plan
    lib = _lib.load()
    dev = torch.device("cuda:0")
    wl = S.make_workload("uneven_2d", batch=64)
    t = [torch.from_numpy(x).to(dev) for x in (wl.cubes, wl.offsets, wl.alpha, wl.tau)]
    base = configs.params_for(wl)
    for variant in ("resume", "prefetch"):
        p = dataclasses.replace(base, fft_path=2, gather_mode=3 if variant == "prefetch" else base.gather_mode)
        plan = Plan(wl.dims, p)
        init = None
        seed_out = None
        if variant == "resume":   # a partial set: the planted frequencies' first half, amplitudes off by 10 %
            seed_out = plan.alloc_output(dev)
            counts = np.zeros(wl.batch, np.int32)
            for b in range(wl.batch):
                kt = wl.k_true[b][: len(wl.k_true[b]) // 2]
                counts[b] = len(kt)
                seed_out.k[b, :len(kt)] = torch.from_numpy(kt.astype(np.int32)).to(dev)
                seed_out.a[b, :len(kt)] = torch.from_numpy((1.1 * wl.a_true[b][:len(kt)]).astype(np.complex64)).to(dev)
            init = torch.from_numpy(counts).to(dev)
        ref = plan.alloc_output(dev)
        out = plan.alloc_output(dev)
        if seed_out is not None:
            for dst in (ref, out):
                dst.k.copy_(seed_out.k)
                dst.a.copy_(seed_out.a)
        plan.recover(*t, out=ref, init_count=init)
        assert _noalloc(lib, wl, p, t, out, init_count=init) == _lib.OK, lib.fpssft_last_error().decode()
        torch.cuda.synchronize()
        _same(ref, out)
        plan.close()


def test_noalloc_rejects_a_set_beyond_shared_memory():
    """The plan path moves a set this large to global memory; the no-allocation call has no such
    variant and must refuse before launching anything."""
    lib = _lib.load()
    dev = torch.device("cuda:0")
    wl = S.make_workload("uneven_2d", batch=2)
    p = dataclasses.replace(configs.params_for(wl), k_cap=20000)
    t = [torch.from_numpy(x).to(dev) for x in (wl.cubes, wl.offsets, wl.alpha, wl.tau)]
    from paper_1711_11407_gb300.api import Plan
    plan = Plan(wl.dims, p)
    out = plan.alloc_output(dev)
    out.count.fill_(-5)
    st = _noalloc(lib, wl, p, t, out)
    assert st == _lib.ERR_UNSUPPORTED
    assert b"shared memory" in lib.fpssft_last_error()
    torch.cuda.synchronize()
    assert torch.all(out.count == -5)        # nothing was launched
    plan.close()


def test_noalloc_rejects_batches_beyond_its_fixed_scratch():
    lib = _lib.load()
    dev = torch.device("cuda:0")
    batch = 100000                                   # ~1.2 MB of per-signal tables > 1 MiB
    dims = np.full((batch, 2), 4, np.int64)
    p = configs.params_for(S.make_workload("single_128x128"))
    cp = p.c()
    z = torch.zeros(16, dtype=torch.int32, device=dev)
    st = lib.fpssft_recover_noalloc(2, batch, dims.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cp),
                                    _ptr(z), _ptr(z), _ptr(z), _ptr(z), None, _ptr(z), _ptr(z), _ptr(z), _ptr(z),
                                    _ptr(z), None)
    assert st == _lib.ERR_UNSUPPORTED
    assert b"scratch" in lib.fpssft_last_error()
