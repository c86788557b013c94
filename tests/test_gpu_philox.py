"""The library's Philox4x32-10 on the GPU against the generator's
implementation in the CUDA toolkit's cuRAND device header
(curand_Philox4x32_10), bit for bit, on random counters and keys and on
the counters the sweep and the initial states use; and against the CPU
oracle's Philox (pinned by the published known-answer vectors)."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _run(ctr: np.ndarray, key: np.ndarray):
    import torch

    import paper_2407_19987_gb300 as H
    c = torch.from_numpy(np.ascontiguousarray(ctr, dtype=np.uint32).view(np.int32)).cuda()
    k = torch.from_numpy(np.ascontiguousarray(key, dtype=np.uint32).view(np.int32)).cuda()
    ours, ref = H.selftest_philox(c, k)
    return ours.cpu().numpy().view(np.uint32), ref.cpu().numpy().view(np.uint32)


def test_philox_matches_curand_on_random_counters_and_keys():
    rng = np.random.default_rng(11)
    n = 1 << 20
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ours, ref = _run(ctr, key)
    np.testing.assert_array_equal(ours, ref)
    for i in range(0, n, n // 64):
        assert O.philox(ctr[i].tolist(), key[i].tolist()).tolist() == ours[i].tolist()


def test_philox_matches_curand_on_the_annealer_counters():
    # Metropolis draws: counter (bit / 4, sweep, state, 0); initial states:
    # (bit / 4, 0, state, 1); key = (seed low, seed high)
    rows = []
    for stream in (0, 1):
        for sweep in (0, 1, 999, 19999):
            for state in (0, 1, 4095, 8191, 2 ** 31 + 5):
                for q in range(0, 64):
                    rows.append((q, sweep if stream == 0 else 0, state, stream))
    ctr = np.array(rows, dtype=np.uint64).astype(np.uint32)
    seed = 0x123456789
    key = np.tile(np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32), (len(rows), 1))
    ours, ref = _run(ctr, key)
    np.testing.assert_array_equal(ours, ref)


def test_philox_selftest_arguments():
    import torch

    import paper_2407_19987_gb300 as H
    e = torch.empty((0, 4), dtype=torch.int32, device="cuda")
    ours, ref = H.selftest_philox(e, torch.empty((0, 2), dtype=torch.int32, device="cuda"))
    assert ours.numel() == 0 and ref.numel() == 0
