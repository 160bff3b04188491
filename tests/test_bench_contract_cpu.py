"""The benchmark's CPU-side contract (no GPU): the reference arm's JSON line and the kernel-source
hash that decides whether a committed DRAM-traffic record still applies."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--workload", "single_128x128"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "signals/s" and d["higher_is_better"] is True
    assert d["metric"] == bench.METRIC and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "signals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "single_128x128"


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    """Launched like the multi-GPU benchmark (two ranks), only rank 0 runs the oracle and prints;
    the other rank exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1", "--workload", "single_128x128"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_source_hash_ignores_comments_and_whitespace_but_not_code():
    a = "int f(int x) {  // twice\n  return 2 * x; /* done */ }\n"
    b = "int f(int x) { return 2 * x; }"
    c = "int f(int x) { return 3 * x; }"
    assert bench.strip_comments(a) == bench.strip_comments(b)
    assert bench.strip_comments(a) != bench.strip_comments(c)
    assert bench.strip_comments('const char* s = "// kept"; // dropped') == 'const char* s = "// kept";'
    h = bench.source_hash()
    assert len(h) == 16 and h == bench.source_hash()


def test_traffic_record_scales_by_signals_and_expires_with_the_kernel_code(tmp_path, monkeypatch):
    """roofline.traffic comes from the committed DRAM record, scaled from its batch to the bench's,
    only while the record's hash matches the kernel code (a comment-only edit keeps it)."""
    csrc = tmp_path / "paper_1711_11407_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "k.cu").write_text("__global__ void k() { }  // v1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = {"source_hash": bench.source_hash(), "batch": 1024, "dram_bytes_per_launch": 1000.0}
    (tmp_path / "profiles" / "k_recover_wl.json").write_text(json.dumps(rec))
    traffic, path = bench.profiled_traffic("wl", 4096)
    assert traffic == 4000.0 and path.endswith("k_recover_wl.json")
    (csrc / "k.cu").write_text("__global__ void k() { }  // v2, comment only\n")
    assert bench.profiled_traffic("wl", 4096)[0] == 4000.0
    (csrc / "k.cu").write_text("__global__ void k() { int x = 1; }\n")
    assert bench.profiled_traffic("wl", 4096)[0] is None
    assert bench.profiled_traffic("other", 4096) == (None, None)


def test_clock_summary_keeps_this_gpu_inside_the_timed_region():
    """The clocks record: only this GPU's samples that arrived inside the timed region count; the
    median SM clock, the max clock and every throttle reason seen active are reported."""
    cs = bench.ClockSampler.__new__(bench.ClockSampler)
    cs.uuid, cs.proc = "GPU-aaa", None

    def row(uuid, sm, reasons=("Not Active",) * 4):
        return ", ".join(["0", uuid, str(sm), "2070", "900.5", "0x0", *reasons]) + "\n"

    cs.lines = [(0.5, row("GPU-aaa", 1000)),                                   # before the region
                (1.1, row("GPU-aaa", 2070)),
                (1.2, row("GPU-bbb", 500, ("Active",) * 4)),                  # another GPU
                (1.3, row("GPU-aaa", 2040, ("Not Active", "Not Active", "Not Active", "Active"))),
                (1.4, row("GPU-aaa", 2055)),
                (9.0, row("GPU-aaa", 300, ("Active",) * 4))]                  # after the region
    cs.t0, cs.t1 = 1.0, 1.5
    s = cs.summary()
    assert s == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    cs.t0, cs.t1 = 20.0, 21.0
    assert cs.summary()["samples"] == 0


def test_e2e_self_check_compares_whole_sets_not_counts():
    """The bench line's matches_device_run flags: equal counts are not enough -- a different
    frequency, an amplitude off by more than 1e-4 relative or a different iteration count fails."""
    import torch

    from paper_1711_11407_gb300.api import RecoverOutput

    def out():
        k = torch.zeros((2, 4, 2), dtype=torch.int32)
        k[0, :2] = torch.tensor([[1, 2], [3, 4]])
        k[1, :1] = torch.tensor([[5, 6]])
        a = torch.zeros((2, 4), dtype=torch.complex64)
        a[0, :2] = torch.tensor([1 + 1j, 2 - 1j])
        a[1, :1] = torch.tensor([0.5j])
        return RecoverOutput(k, a, torch.tensor([2, 1], dtype=torch.int32), torch.tensor([3, 2], dtype=torch.int32),
                             torch.zeros(2, dtype=torch.int32))

    ref = out()
    assert bench.same_sets(ref, out())
    o = out()
    o.k[2:] = 9                                  # rows beyond count are not part of the set
    o.a[1, 3] = 7
    assert bench.same_sets(ref, o)
    o = out()
    o.k[0, 1, 0] = 8
    assert not bench.same_sets(ref, o)
    o = out()
    o.a[0, 0] *= 1 + 1e-3
    assert not bench.same_sets(ref, o)
    o = out()
    o.a[0, 0] *= 1 + 1e-6
    assert bench.same_sets(ref, o)
    o = out()
    o.iters[1] = 5
    assert not bench.same_sets(ref, o)


def test_cpu_baseline_repeats_the_signals_of_a_workload_smaller_than_the_core_count():
    """A workload with fewer signals than host cores (a single image, say) is timed with one core
    per signal, each recovering its signal over and over until the round takes a second, so that the
    pool's start-up and hand-over do not dominate a few milliseconds of oracle work."""
    from paper_1711_11407_gb300 import configs, synth
    if len(os.sched_getaffinity(0)) < 3:
        import pytest
        pytest.skip("needs at least 3 host cores")
    wl = synth.make_workload("uneven_2d", batch=2, shapes=[(16, 16)], K=lambda N: 4, T=6)
    rate, n, wall, cores = bench.oracle_rate(wl, configs.params_for(wl), 12.0, [0, 1])
    assert cores == 2 and wall >= 1.0
    assert n % 2 == 0 and n >= 4 and rate == n / wall
