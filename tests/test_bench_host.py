"""Host logic of the benchmark that needs no GPU: the time-to-target
ladder (the first schedule of growing length whose best state
reaches the target, with the time of the misses kept apart) and the peak
figures' fallback.  CPU only."""
import numpy as np

import bench


def test_ladder_takes_the_first_schedule_that_reaches_the_target():
    calls = []

    def run(S):                      # best energy falls with the schedule length
        calls.append(S)
        return np.array([100.0 - S, 200.0]), float(S) / 10.0

    r = bench._ladder(run, target=100.0 - 20)
    assert r["sweeps"] == 20 and calls == [5, 10, 15, 20]
    assert r["ms"] == 2.0 and r["ms_including_misses"] == 0.5 + 1.0 + 1.5 + 2.0
    assert r["best"] == 80.0


def test_ladder_reports_a_miss_over_the_whole_ladder():
    r = bench._ladder(lambda S: (np.array([1.0]), 1.0), target=0.0, ladder=(5, 10))
    assert r["sweeps"] is None and r["ms"] is None and r["ms_including_misses"] == 2.0 and r["best"] == 1.0


def test_peaks_come_from_the_measured_file_or_the_stated_fallback():
    pk, kind = bench.peaks()
    assert kind in ("measured", "fallback")
    assert pk["hbm_gbs"] > 0 and pk["bf16_tflops"] > 0
    if kind == "fallback":
        assert pk["hbm_gbs"] == 6800.0 and pk["bf16_tflops"] == 1900.0
