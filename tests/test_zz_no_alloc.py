"""hobo_energy_fp64_noalloc: the float64 re-score for callers that cannot let
the library allocate device memory (their GPU memory is reserved by their
own pool, or their loop must not risk an allocation's synchronisation).
Its scratch is a fixed array in device memory shared by all calls, so each
case makes two calls in a row, the second on fewer states than the first
(it must not see the first call's sums), and checks both against the CPU
oracle and against hobo_energy_fp64.  A second test reads the high-water
mark of the device's memory pool around the calls: the allocating re-score
raises it, this one must not."""
import ctypes

import numpy as np
import pytest

import gpuh
import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu

CASES = [
    # (instance, batch sizes of the two calls); the instances take the three
    # re-score routes: term list (sparse), limb planes on the tensor cores
    # (dense, N <= 256) and the CUDA-core dense kernel (dense, N > 256)
    ("integer", lambda: W.int_encoded(3), (3000, 1000)),
    ("dense_float_N96", lambda: W.dense_float(7, 96), (3000, 1000)),
    ("dense_float_N300", lambda: W.dense_float(9, 300), (160, 48)),
    ("sparse_order4", lambda: W.random_sparse(8, 70, 4, 0.05, "normal"), (3000, 1000)),
]


@pytest.mark.parametrize("maker,sizes", [(c[1], c[2]) for c in CASES], ids=[c[0] for c in CASES])
def test_noalloc_matches_oracle_and_allocating_rescore_twice(maker, sizes):
    import torch
    inst = maker()
    h = gpuh.make(inst)
    for seed, B in zip((1, 2), sizes):
        Xh = W.random_states(seed, B, inst.N)
        X = gpuh.to_dev(Xh)
        ref = h.energy_fp64(X)
        got = h.energy_fp64_noalloc(X)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        np.testing.assert_array_equal(g, r)
        if inst.integer:
            np.testing.assert_array_equal(g, O.energy_int(inst, Xh).astype(np.float64))
        else:
            # exact fixed-point sums rounded once; the fixed-point scale keeps
            # the coefficient rounding below 1e-9 of any energy here
            np.testing.assert_allclose(g, O.energy(inst, Xh), rtol=1e-12, atol=1e-9)
    h.check()
    h.close()


class _Pool:
    """The current memory pool of a device, through the CUDA driver API:
    the pool that stream-ordered allocations of the library draw from."""
    USED_MEM_HIGH = 8      # CU_MEMPOOL_ATTR_USED_MEM_HIGH

    def __init__(self, ordinal: int):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), ordinal) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetMemPool(ctypes.byref(self.pool), dev) == 0

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(zero)) == 0

    def high(self) -> int:
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(v)) == 0
        return int(v.value)


def test_noalloc_leaves_the_memory_pool_untouched():
    import torch
    inst = W.dense_float(7, 96)
    h = gpuh.make(inst)
    X = gpuh.to_dev(W.random_states(3, 4096, inst.N))
    E = torch.empty(4096, dtype=torch.float64, device="cuda")
    h.energy_fp64_noalloc(X, E=E)
    torch.cuda.synchronize()
    pool = _Pool(torch.cuda.current_device())
    # the allocating re-score shows up in the pool's high-water mark ...
    pool.reset_high()
    base = pool.high()
    h.energy_fp64(X)
    torch.cuda.synchronize()
    assert pool.high() >= base + 4096 * 8
    # ... and the one without allocations does not, over two calls
    pool.reset_high()
    base = pool.high()
    for _ in range(2):
        h.energy_fp64_noalloc(X, E=E)
    torch.cuda.synchronize()
    assert pool.high() == base
    h.close()


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
