"""The package's host tensor-train decomposition (Sec. VI), against the
oracle's contraction of trains: the TSP tensor's printed bond dimensions
and exact reconstruction, recovery of known ranks, the rank cap and the
zero tensor.  CPU only."""
import numpy as np

import polyexp
from oracle import oracle as O
from paper_2407_19987_gb300.tt import tt_svd


def test_tsp_tensor_train_has_the_printed_shapes_and_reproduces_the_tensor():
    T = polyexp.tsp_intenc().dense().astype(np.float64)
    cores = tt_svd(T)
    assert [G.shape for G in cores] == [(1, 6, 2), (2, 6, 3), (3, 6, 4), (4, 6, 4), (4, 6, 2), (2, 6, 1)]
    np.testing.assert_allclose(O.tt_full(cores), T, atol=1e-9 * np.abs(T).max())


def test_known_ranks_are_recovered_and_the_cap_holds():
    rng = np.random.default_rng(4)
    ranks = [1, 3, 2, 4, 1]
    train = [rng.standard_normal((ranks[c], 5, ranks[c + 1])) for c in range(4)]
    A = O.tt_full(train)
    cores = tt_svd(A)
    assert [G.shape[2] for G in cores] == ranks[1:]
    np.testing.assert_allclose(O.tt_full(cores), A, atol=1e-10 * np.abs(A).max())
    capped = tt_svd(A, max_rank=2)
    assert max(G.shape[2] for G in capped) <= 2
    zero = tt_svd(np.zeros((3, 3, 3)))
    assert [G.shape for G in zero] == [(1, 3, 1), (1, 3, 1), (1, 3, 1)]
    assert not np.any(O.tt_full(zero))
