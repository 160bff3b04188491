"""The phase-timer read-out arithmetic (no GPU): counters summed over CTAs become microseconds per
CTA and per iteration at the clock the CTAs measured."""
import pytest

from paper_1711_11407_gb300 import phases


def test_summarize_converts_cycles_at_the_measured_clock():
    # 4 CTAs at 2 cycles/ns, 10 iterations in all; phase cycles 8000, 4000, ... (total 40000)
    cyc = [8000, 4000, 12000, 2000, 6000, 0, 4000]
    raw = cyc + [4, 10, 40000, 20000]
    s = phases.summarize(raw)
    assert s["ctas"] == 4 and s["iterations_per_cta"] == 2.5
    assert s["sm_clock_mhz"] == pytest.approx(2000.0)
    assert s["cta_us"] == pytest.approx(40000 / 4 / 2 / 1e3)
    per_cta = s["phase_us_per_cta"]
    assert per_cta["setup"] == pytest.approx(8000 / 4 / 2 / 1e3)
    assert per_cta["fft"] == pytest.approx(12000 / 4 / 2 / 1e3)
    assert per_cta["unmarked"] == pytest.approx((40000 - sum(cyc)) / 4 / 2 / 1e3)
    assert sum(per_cta.values()) == pytest.approx(s["cta_us"])
    assert s["phase_us_per_iteration"]["peel"] == pytest.approx(2000 / 10 / 2 / 1e3)


def test_summarize_rejects_empty_counters():
    with pytest.raises(ValueError):
        phases.summarize([0] * 11)
