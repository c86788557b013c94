"""GPU parity of the order-4 tensor-core contraction (quartic part on
tcgen05 from the (N^3 x N) reshaped symmetric tensor, lower degrees on the
term-list path): integer instances bit-exact against the oracle, float
instances within the float bar, and an anneal initialised by it following
the oracle trajectory for trajectory."""
import numpy as np
import pytest

import gpuh
import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _H():
    import paper_2407_19987_gb300 as H
    return H


def _dense4(seed, N, integer, lower=True):
    return W.dense_all_degrees(seed, N, 4, "int" if integer else "normal", 3, top_only=not lower)


@pytest.mark.parametrize("N,B,lower", [(12, 300, True), (33, 129, True), (40, 4096, False), (64, 256, True)])
def test_tc4_integer_exact(N, B, lower):
    inst = _dense4(100 + N, N, True, lower)
    if np.abs(inst.coef).sum() >= 2 ** 24:
        pytest.skip("not an exact-integer instance")
    h = gpuh.make(inst)
    X = W.random_states(N, B, N)
    E, dE = h.energy(gpuh.to_dev(X), path=_H().PATH_TENSOR_CORE)
    E = E.cpu().numpy().astype(np.float64)
    dE = dE.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(E, O.energy_int(inst, X).astype(np.float64))
    for b in range(0, B, max(1, B // 16)):
        np.testing.assert_array_equal(dE[b], (1.0 - 2.0 * X[b]) * O.fields(inst, X[b]))
    h.check()
    h.close()


@pytest.mark.parametrize("N,B", [(16, 300), (37, 200), (64, 4096)])
def test_tc4_float_within_bar(N, B):
    inst = _dense4(200 + N, N, False)
    h = gpuh.make(inst)
    X = W.random_states(N + 1, B, N)
    E, dE = h.energy(gpuh.to_dev(X), path=_H().PATH_TENSOR_CORE)
    E = E.cpu().numpy().astype(np.float64)
    dE = dE.cpu().numpy().astype(np.float64)
    absi = gpuh.abs_instance(inst)
    rows = np.arange(0, B, max(1, B // 24))
    assert gpuh.rel_err(E[rows], O.energy(inst, X[rows]), O.energy(absi, X[rows]), gpuh.COND_MAX_F32ACC).max() <= gpuh.FLOAT_RTOL
    for b in rows[:8]:
        g, ga = O.fields(inst, X[b]), O.fields(absi, X[b])
        assert gpuh.rel_err(dE[b], (1.0 - 2.0 * X[b]) * g, ga, gpuh.COND_MAX_F32ACC).max() <= gpuh.FLOAT_RTOL
    # the term-list path of the same instance agrees within the same bar
    E1, dE1 = h.energy(gpuh.to_dev(X[rows]), path=_H().PATH_TERMS)
    assert gpuh.rel_err(E[rows], E1.cpu().numpy().astype(np.float64), O.energy(absi, X[rows]),
                        gpuh.COND_MAX_F32ACC).max() <= 2 * gpuh.FLOAT_RTOL
    h.close()


def test_anneal_on_order4_dense_instance_follows_oracle():
    inst = _dense4(300, 20, True)
    h = gpuh.make(inst)
    betas = W.geometric_betas(20.0, 0.1, 15)
    r = h.anneal(7, 40, betas, want_final=True, want_accepts=True)
    ref = O.anneal(inst, 7, 40, betas)
    np.testing.assert_array_equal(gpuh.to_host_bits(r["bestX"], inst.N), ref["bestX"])
    np.testing.assert_array_equal(r["bestE"].cpu().numpy(), ref["bestE"])
    np.testing.assert_array_equal(r["accepts"].cpu().numpy(), ref["accepts"])
    h.close()


def test_order4_sparse_instance_refuses_tensor_core_path():
    inst = W.random_sparse(301, 40, 4, 0.02, "int")
    h = gpuh.make(inst)
    with pytest.raises(_H().HoboError):
        h.energy(gpuh.to_dev(W.random_states(1, 4, inst.N)), path=_H().PATH_TENSOR_CORE)
    h.close()
