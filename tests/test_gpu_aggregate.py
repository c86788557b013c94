"""GPU parity of the result table (hobo_aggregate) against the oracle's
plain dictionary-and-sort statement of it: distinct states by energy, ties
by first index, with occurrence counts."""
import numpy as np
import pytest

import gpuh
import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _H():
    import paper_2407_19987_gb300 as H
    return H


def _gpu_table(X_u8, E):
    T = gpuh.torch()
    r = _H().aggregate(gpuh.to_dev(X_u8), T.from_numpy(np.ascontiguousarray(E, dtype=np.float64)).cuda())
    N = X_u8.shape[1]
    return (gpuh.to_host_bits(r["states"], N), r["energy"].cpu().numpy(), r["count"].cpu().numpy(),
            r["first"].cpu().numpy())


def _compare(X_u8, E):
    got = _gpu_table(X_u8, E)
    ref = O.aggregate(X_u8, E)
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g, r)


@pytest.mark.parametrize("B,distinct,N", [(1, 1, 12), (2, 2, 12), (2047, 40, 12), (2048, 40, 33),
                                          (5000, 300, 70), (70001, 5000, 12), (1100000, 900, 40)])
def test_aggregate_matches_oracle(B, distinct, N):
    """States drawn with repetition from a pool; integer energies of an
    instance, so distinct states share energies (ties by first index)."""
    rng = np.random.default_rng(B)
    pool = rng.integers(0, 2, size=(distinct, N)).astype(np.uint8)
    X = pool[rng.integers(0, distinct, size=B)]
    inst = W.random_sparse(B % 97, N, 3, 0.2, "int")
    E = O.energy(inst, X)
    _compare(X, E)


def test_aggregate_empty_and_arguments():
    T = gpuh.torch()
    r = _H().aggregate(T.zeros((0, 1), dtype=T.int32, device="cuda"), T.zeros(0, dtype=T.float64, device="cuda"))
    assert r["states"].shape[0] == 0
    with pytest.raises(_H().HoboError):
        _H().aggregate(T.zeros((4, 33), dtype=T.int32, device="cuda"), T.zeros(4, dtype=T.float64, device="cuda"))


def test_anneal_then_aggregate_matches_oracle_run():
    """The sampler's run output end to end on an integer instance: anneal,
    re-score, aggregate, against the oracle's anneal and aggregate."""
    inst = W.tiny_dense(1)
    betas = W.geometric_betas(5.0, 0.05, 100)
    h = gpuh.make(inst)
    r = h.anneal(1, 256, betas)
    T = _H().aggregate(r["bestX"], r["bestE"])
    ref_run = O.anneal(inst, 1, 256, betas)
    ref = O.aggregate(ref_run["bestX"], ref_run["bestE"])
    np.testing.assert_array_equal(gpuh.to_host_bits(T["states"], inst.N), ref[0])
    np.testing.assert_array_equal(T["energy"].cpu().numpy(), ref[1])
    np.testing.assert_array_equal(T["count"].cpu().numpy(), ref[2])
    np.testing.assert_array_equal(T["first"].cpu().numpy(), ref[3])
    assert T["energy"][0].item() == O.bruteforce(inst).min()
    h.close()
