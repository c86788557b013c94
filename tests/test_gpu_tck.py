"""GPU parity of the order-5/6 tensor-core contraction (top degree on
tcgen05 from rows over sorted index prefixes, lower degrees in a child
instance that may take a tensor-core path of its own): integer instances
bit-exact against the oracle, float instances within the float32-sum bar
of the float32-accumulating kernels, the same results as the term-list
path, and an anneal initialised by it following the oracle trajectory for
trajectory."""
import numpy as np
import pytest

import gpuh
import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _H():
    import paper_2407_19987_gb300 as H
    return H


def _dense(seed, N, k, integer, lower=True):
    return W.dense_all_degrees(seed, N, k, "int" if integer else "normal", 2, top_only=not lower)


INT_CASES = [(5, 9, 300, True), (5, 20, 129, True), (5, 32, 257, False), (6, 8, 200, True), (6, 16, 130, True),
             (6, 21, 64, False)]


@pytest.mark.parametrize("k,N,B,lower", INT_CASES, ids=[f"k{c[0]}_N{c[1]}_B{c[2]}" for c in INT_CASES])
def test_tck_integer_exact(k, N, B, lower):
    """Exact energies and flip deltas: every partial sum is an integer below
    2^24; ragged state tiles (B not a multiple of 128), ragged row chunks
    (C(N, k-2) not a multiple of 256) and N not a multiple of 32."""
    inst = _dense(400 + N + k, N, k, True, lower)
    if np.abs(inst.coef).sum() >= 2 ** 24:
        pytest.skip("not an exact-integer instance")
    h = gpuh.make(inst)
    X = W.random_states(N + k, B, N)
    E, dE = h.energy(gpuh.to_dev(X), path=_H().PATH_TENSOR_CORE)
    E = E.cpu().numpy().astype(np.float64)
    dE = dE.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(E, O.energy_int(inst, X).astype(np.float64))
    for b in range(0, B, max(1, B // 12)):
        np.testing.assert_array_equal(dE[b], (1.0 - 2.0 * X[b]) * O.fields(inst, X[b]))
    # the term-list path gives the same integers
    E1, dE1 = h.energy(gpuh.to_dev(X), path=_H().PATH_TERMS)
    np.testing.assert_array_equal(E1.cpu().numpy(), E.astype(np.float32))
    np.testing.assert_array_equal(dE1.cpu().numpy(), dE.astype(np.float32))
    h.check()
    h.close()


@pytest.mark.parametrize("k,N,B", [(5, 24, 300), (6, 18, 4096)])
def test_tck_float_within_bar(k, N, B):
    inst = _dense(500 + N, N, k, False)
    h = gpuh.make(inst)
    X = W.random_states(N + 1, B, N)
    E, dE = h.energy(gpuh.to_dev(X), path=_H().PATH_TENSOR_CORE)
    E = E.cpu().numpy().astype(np.float64)
    dE = dE.cpu().numpy().astype(np.float64)
    absi = gpuh.abs_instance(inst)
    rows = np.arange(0, B, max(1, B // 24))
    assert gpuh.rel_err(E[rows], O.energy(inst, X[rows]), O.energy(absi, X[rows]),
                        gpuh.COND_MAX_F32ACC).max() <= gpuh.FLOAT_RTOL
    for b in rows[:8]:
        g, ga = O.fields(inst, X[b]), O.fields(absi, X[b])
        assert gpuh.rel_err(dE[b], (1.0 - 2.0 * X[b]) * g, ga, gpuh.COND_MAX_F32ACC).max() <= gpuh.FLOAT_RTOL
    h.close()


def test_anneal_on_order5_dense_instance_follows_oracle():
    inst = _dense(600, 14, 5, True)
    h = gpuh.make(inst)
    betas = W.geometric_betas(20.0, 0.1, 15)
    r = h.anneal(7, 40, betas, want_final=True, want_accepts=True)
    ref = O.anneal(inst, 7, 40, betas)
    np.testing.assert_array_equal(gpuh.to_host_bits(r["bestX"], inst.N), ref["bestX"])
    np.testing.assert_array_equal(r["bestE"].cpu().numpy(), ref["bestE"])
    np.testing.assert_array_equal(r["accepts"].cpu().numpy(), ref["accepts"])
    h.close()


def test_order6_sparse_instance_refuses_tensor_core_path():
    inst = W.random_sparse(601, 30, 6, 0.001, "int")
    h = gpuh.make(inst)
    with pytest.raises(_H().HoboError):
        h.energy(gpuh.to_dev(W.random_states(1, 4, inst.N)), path=_H().PATH_TENSOR_CORE)
    h.close()
