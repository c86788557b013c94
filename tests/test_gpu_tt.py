"""GPU parity of the tensor-train contraction (hobo_tt_energy, Sec. VI)
against the oracle's float64 train contraction and, for the paper's TSP
tensor, against the energies of the tensor itself."""
import numpy as np
import pytest

import gpuh
import polyexp
import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _tol(cores32, X):
    """Float32 bound: every output of core c sums at most N * r_{c-1}
    products (each relative error <= 2^-24 per operation), plus the
    rounding of the cores to float32, against the energy of the train with
    |cores| (the sum of the magnitudes of all terms)."""
    N = cores32[0].shape[1]
    n = sum(N * G.shape[0] + 2 for G in cores32)
    absE = O.tt_energy([np.abs(G.astype(np.float64)) for G in cores32], X)
    return n * 2.0 ** -24 * absE


def _check(cores, X):
    from paper_2407_19987_gb300.tt import TensorTrain
    c32 = [np.asarray(G, np.float32) for G in cores]
    tt = TensorTrain(c32)
    got = tt.energy(gpuh.to_dev(X)).cpu().numpy().astype(np.float64)
    ref = O.tt_energy([G.astype(np.float64) for G in c32], X)
    assert np.all(np.abs(got - ref) <= _tol(c32, X)), np.max(np.abs(got - ref) / np.maximum(_tol(c32, X), 1e-30))
    tt.close()
    return got


def test_tsp_train_reproduces_the_tensor_energies():
    from paper_2407_19987_gb300.tt import tt_svd
    inst = polyexp.tsp_intenc()
    T = inst.dense().astype(np.float64)
    cores = tt_svd(T)
    # the bond dimensions printed in Sec. VI.F
    assert [G.shape for G in cores] == [(1, 6, 2), (2, 6, 3), (3, 6, 4), (4, 6, 4), (4, 6, 2), (2, 6, 1)]
    X = np.array([[(s >> i) & 1 for i in range(6)] for s in range(64)], np.uint8)
    got = _check(cores, X)
    np.testing.assert_allclose(got, O.energy(inst, X), atol=2e-3)


@pytest.mark.parametrize("order,N,ranks,B", [(1, 50, [1, 1], 70), (3, 256, [1, 16, 16, 1], 4096),
                                             (6, 32, [1, 8, 16, 16, 16, 8, 1], 1000), (2, 1024, [1, 64, 1], 300),
                                             (3, 64, [1, 256, 40, 1], 129), (8, 12, [1, 2, 3, 4, 5, 4, 3, 2, 1], 77)])
def test_random_trains_match_oracle(order, N, ranks, B):
    rng = np.random.default_rng(order * 1000 + N)
    cores = [rng.standard_normal((ranks[c], N, ranks[c + 1])) / np.sqrt(N * ranks[c]) for c in range(order)]
    X = W.random_states(order + N, B, N)
    _check(cores, X)


def test_tt_arguments():
    import paper_2407_19987_gb300 as H
    from paper_2407_19987_gb300.tt import TensorTrain
    with pytest.raises(H.HoboError):
        TensorTrain([np.ones((2, 5, 1), np.float32)])          # r_0 != 1
    with pytest.raises(ValueError):
        TensorTrain([np.ones((1, 5, 2), np.float32), np.ones((3, 5, 1), np.float32)])
    tt = TensorTrain([np.ones((1, 5, 1), np.float32)])
    T = gpuh.torch()
    assert tt.energy(T.zeros((0, 1), dtype=T.int32, device="cuda")).numel() == 0
