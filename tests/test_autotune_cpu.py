"""Autotuner host logic (no GPU): candidate launch configurations and the cache key."""
import numpy as np

from paper_1711_11407_gb300 import autotune
from paper_1711_11407_gb300.api import Params


def test_candidates_offer_the_register_path_only_for_eligible_line_lengths():
    p = Params(T=0, k_cap=512)
    c = autotune.candidates(np.array([[64, 64], [128, 256], [256, 256]]), p)
    assert any(x.fft_path == 2 for x in c) and any(x.fft_path == 1 for x in c)
    assert not any(x.fft_path == 3 for x in c)                  # lines of 256 points at most
    c = autotune.candidates(np.array([[240, 256]]), p)          # L = 3840
    assert {x.fft_path for x in c} == {1, 3}
    assert all(x.gather_mode in (1, 2, 3, 4, 5) for x in c)
    assert {x.threads for x in c if x.fft_path == 3} == {256, 512, 1024}
    # every cluster-path launch is offered with the set in shared memory and in global workspace
    assert {(x.threads, x.gather_mode, x.cluster_set) for x in c if x.fft_path == 3} == \
        {(t, g, s) for t in (256, 512, 1024) for g in (1, 3) for s in (1, 2)}
    assert all(x.cluster_set == 0 for x in c if x.fft_path != 3)
    c = autotune.candidates(np.array([[512, 512]]), p)          # L = 512: no register path
    assert {x.fft_path for x in c} == {1, 3}
    assert {x.threads for x in c if x.fft_path == 3} == {256}


def test_cache_key_ignores_batch_order_and_size():
    p = Params(T=0, k_cap=512)
    a = autotune.cache_key(np.array([[64, 64], [128, 128]]), p, "GB300")
    b = autotune.cache_key(np.array([[128, 128], [64, 64], [64, 64]]), p, "GB300")
    assert a == b
    assert a != autotune.cache_key(np.array([[64, 64]]), p, "GB300")
    assert a != autotune.cache_key(np.array([[64, 64], [128, 128]]), Params(T=0, k_cap=256), "GB300")
    # the stop rule changes how many iterations a signal runs, and with it the best launch
    assert a != autotune.cache_key(np.array([[64, 64], [128, 128]]), Params(T=0, k_cap=512, early_stop=2), "GB300")


def test_cache_hit_returns_the_stored_choice_without_timing(tmp_path, monkeypatch):
    """A batch whose shapes, budget and capacity were tuned before on this GPU takes the stored
    launch choice from the JSON cache; nothing is launched (here: no device at all)."""
    import json

    import torch

    monkeypatch.setattr(torch.cuda, "get_device_name", lambda device=None: "GB300 (test)")
    dims = np.asarray([[64, 64], [128, 128], [64, 64]])
    p = Params(T=0, k_cap=512)
    key = autotune.cache_key(dims, p, "GB300 (test)")
    path = tmp_path / "tune.json"
    stored = {"choice": {"fft_path": 2, "gather_mode": 1, "threads": 96}, "timings": {"path=2": 0.2}}
    path.write_text(json.dumps({key: stored}))
    best, timings = autotune.tune(dims, p, torch.zeros(4, dtype=torch.complex64), None, None, None,
                                  cache_path=str(path))
    assert (best.fft_path, best.gather_mode, best.threads, best.k_cap) == (2, 1, 96, 512)
    assert timings == stored["timings"]


def test_radix_plan_candidates_only_where_the_stage_sequence_changes():
    """Radix plans are offered for the shared-memory FFT paths, and only those whose stage sequence
    differs from the default for some line length of the batch (3840 = 8 8 4 3 5 by default)."""
    from dataclasses import replace
    p = Params(T=0, k_cap=640)
    dims = np.array([[240, 256]])
    assert autotune.radix_candidates(dims, replace(p, fft_path=2)) == []
    c = autotune.radix_candidates(dims, replace(p, fft_path=3, threads=512))
    assert {x.radix_plan for x in c} == {1, 2}          # plan 3 gives 8 8 4 3 5 as well
    assert all(x.fft_path == 3 and x.threads == 512 for x in c)
    assert autotune.fft_stages(3840, 1) == [4, 4, 4, 4, 3, 5]
    assert autotune.fft_stages(3840, 2) == [3, 5, 8, 8, 4]
    c = autotune.radix_candidates(np.array([[1024, 1024]]), replace(p, fft_path=3))   # 1024 = 8 8 8 2
    assert {x.radix_plan for x in c} == {1, 3}
    assert autotune.fft_stages(1024, 3) == [8, 8, 4, 4]
