"""hobo_energy_fp64_noalloc: the float64 re-score for callers that cannot let
the library allocate device memory (their GPU memory is reserved by their
own pool, or their loop must not risk an allocation's synchronisation).
Its scratch is a fixed array in device memory shared by all calls, so the
test makes two calls in a row and checks both against hobo_energy_fp64."""
import numpy as np
import pytest

import gpuh
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("maker", [lambda: W.int_encoded(3), lambda: W.dense_float(7, 96),
                                   lambda: W.random_sparse(8, 70, 4, 0.05, "normal")],
                         ids=["integer", "dense_float", "sparse_order4"])
def test_noalloc_matches_allocating_rescore_twice(maker):
    import torch
    inst = maker()
    h = gpuh.make(inst)
    # first call: a larger batch; second call: a smaller one on the same
    # scratch, which must not see the first call's sums
    for seed, B in ((1, 3000), (2, 1000)):
        X = gpuh.to_dev(W.random_states(seed, B, inst.N))
        ref = h.energy_fp64(X)
        got = h.energy_fp64_noalloc(X)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        if inst.integer:
            np.testing.assert_array_equal(g, r)
        else:
            np.testing.assert_allclose(g, r, rtol=1e-12, atol=1e-9)
    h.check()


def test_noalloc_rejects_batches_beyond_its_scratch():
    import paper_2407_19987_gb300 as H
    import torch
    inst = W.tiny_dense(1)
    h = gpuh.make(inst)
    X = torch.zeros((H.binding.HOBO_NOALLOC_MAX_B + 1, 1), dtype=torch.int32, device="cuda")
    with pytest.raises(H.HoboError) as ei:
        h.energy_fp64_noalloc(X)
    assert ei.value.code == -1 and "exceeds" in str(ei.value)
    E0 = h.energy_fp64_noalloc(X[:0])
    assert E0.numel() == 0
