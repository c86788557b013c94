"""Host logic of the benchmark that needs no GPU: the time-to-solution
arithmetic (runs for 99% confidence, for one instance and for a batch of
instances), the ladder's optimum, the plain form at that optimum, and the
peak figures' fallback.  CPU only."""
import math

import numpy as np
import pytest

import bench


def test_runs_for_99_is_the_confidence_formula():
    assert bench.runs_for_99(0.0) is None
    assert bench.runs_for_99(1.0) == 1.0
    assert bench.runs_for_99(0.995) == 1.0            # at least one run
    p = 0.01
    r = bench.runs_for_99(p)
    assert r == pytest.approx(math.log(0.01) / math.log(0.99))
    assert 1.0 - (1.0 - p) ** r == pytest.approx(0.99)


def test_runs_for_all_99_covers_every_instance():
    assert bench.runs_for_all_99([0.5, 0.0]) is None
    assert bench.runs_for_all_99([1.0, 1.0]) == 1.0
    # one instance: the single-instance formula
    assert bench.runs_for_all_99([0.01]) == pytest.approx(bench.runs_for_99(0.01), rel=1e-9)
    p = np.array([0.5, 0.1, 0.02])
    r = bench.runs_for_all_99(p)
    assert np.prod(1.0 - (1.0 - p) ** r) == pytest.approx(0.99, abs=1e-9)
    assert r > bench.runs_for_99(0.02)                 # more than the hardest instance alone


def test_ladder_optimum_trades_length_against_success():
    target = 0.0
    B = 100

    def run(S):      # success share grows with S; time grows linearly
        k = min(B, S)
        E = np.array([-1.0] * k + [1.0] * (B - k))
        return E, float(S)

    r = bench.tts_ladder(run, target, B, ladder=(1, 10, 100, 200))
    ps = [g["p_success"] for g in r["rungs"]]
    assert ps == [0.01, 0.1, 1.0, 1.0]
    tts = [g["tts99_ms"] for g in r["rungs"]]
    assert tts[0] == pytest.approx(1.0 / B * math.log(0.01) / math.log(0.99))
    assert tts[2] == pytest.approx(100.0 / B)
    assert r["best"]["sweeps"] == min(r["rungs"], key=lambda g: g["tts99_ms"])["sweeps"]


def test_ladder_without_success_has_no_optimum():
    r = bench.tts_ladder(lambda S: (np.array([1.0, 2.0]), 1.0), target=0.0, B=2, ladder=(5, 10))
    assert r["best"] is None and all(g["tts99_ms"] is None for g in r["rungs"])


def test_plain_form_is_timed_at_the_tuned_optimum():
    best = {"sweeps": 50, "p_success": 0.25, "tts99_ms": 1.0}
    calls = []

    def run_plain(S):
        calls.append(S)
        return np.zeros(4), 80.0, 0.25

    pl = bench._plain_at(best, run_plain, B=4)
    assert calls == [50] and pl["same_p_as_tuned"]
    assert pl["tts99_ms"] == pytest.approx(80.0 / 4 * bench.runs_for_99(0.25))
    assert bench._speedup(pl, best) == pytest.approx(pl["tts99_ms"])
    assert bench._plain_at(None, run_plain, B=4) is None


def test_peaks_come_from_the_measured_file_or_the_stated_fallback():
    pk, kind = bench.peaks()
    assert kind in ("measured", "fallback")
    assert pk["hbm_gbs"] > 0 and pk["bf16_tflops"] > 0
    if kind == "fallback":
        assert pk["hbm_gbs"] == 6800.0 and pk["bf16_tflops"] == 1900.0


def test_traffic_record_is_tied_to_the_kernel_sources():
    rec = bench.sweep_traffic_record()
    assert rec["dram_bytes"] is None or rec["dram_bytes"] > 0
    assert len(bench.sources_sha256()) == 64
