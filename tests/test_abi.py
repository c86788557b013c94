"""The C ABI library loads, exports every symbol include/hobo.h declares, and
rejects bad arguments on the host (no GPU work).  CPU only."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2407_19987_gb300 as H
from paper_2407_19987_gb300 import binding as Bd
from paper_2407_19987_gb300 import build as Bld

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(Bd.LIB_PATH):
        Bld.build()
    return H.load_library()


def declared_symbols():
    out = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if not name.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", name)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(hobo_[a-z0-9_]+)\s*\(", src):
            out.add(m.group(1))
    return out


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert {"hobo_create", "hobo_create_terms", "hobo_energy", "hobo_anneal", "hobo_destroy",
            "hobo_last_error"} <= syms
    for s in sorted(syms):
        assert hasattr(lib, s), s


def test_version(lib):
    assert H.version().startswith("hobo-gb300")


def test_create_rejects_bad_arguments(lib):
    h = C.c_void_p(123)
    T = np.zeros(8, np.float32)
    assert lib.hobo_create(None, T.ctypes.data_as(C.c_void_p), 3, 2, 0) == Bd.HOBO_ERR_ARG
    assert lib.hobo_create(C.byref(h), None, 3, 2, 0) == Bd.HOBO_ERR_ARG
    assert h.value is None
    assert lib.hobo_create(C.byref(h), T.ctypes.data_as(C.c_void_p), 0, 2, 0) == Bd.HOBO_ERR_ORDER
    assert lib.hobo_create(C.byref(h), T.ctypes.data_as(C.c_void_p), 9, 2, 0) == Bd.HOBO_ERR_ORDER
    assert lib.hobo_create(C.byref(h), T.ctypes.data_as(C.c_void_p), 3, 0, 0) == Bd.HOBO_ERR_ARG
    assert lib.hobo_create(C.byref(h), T.ctypes.data_as(C.c_void_p), 3, 1025, 0) == Bd.HOBO_ERR_ARG
    assert b"N must be" in lib.hobo_last_error()


def test_create_terms_index_checks(lib):
    h = C.c_void_p()
    idx = np.array([[0, 1, 5]], np.int32)
    coef = np.ones(1, np.float32)
    rc = lib.hobo_create_terms(C.byref(h), idx.ctypes.data_as(C.c_void_p), coef.ctypes.data_as(C.c_void_p),
                               1, 3, 5, 0)
    assert rc == Bd.HOBO_ERR_ARG and b"out of range" in lib.hobo_last_error()
    idx = np.array([[0, -1, 2]], np.int32)
    rc = lib.hobo_create_terms(C.byref(h), idx.ctypes.data_as(C.c_void_p), coef.ctypes.data_as(C.c_void_p),
                               1, 3, 5, 0)
    assert rc == Bd.HOBO_ERR_ARG
    bad = np.array([np.nan], np.float32)
    idx = np.array([[0, 1, 2]], np.int32)
    rc = lib.hobo_create_terms(C.byref(h), idx.ctypes.data_as(C.c_void_p), bad.ctypes.data_as(C.c_void_p),
                               1, 3, 5, 0)
    assert rc == Bd.HOBO_ERR_ARG
    rc = lib.hobo_create_terms(C.byref(h), None, None, 1, 3, 5, 0)
    assert rc == Bd.HOBO_ERR_ARG


def test_integer_flag_checks_on_host(lib):
    """HOBO_INTEGER is refused before any device work when coefficients are
    not integers or their absolute sum reaches 2^24."""
    h = C.c_void_p()
    idx = np.array([[0, 1, 2], [1, 1, 2]], np.int32)
    frac = np.array([1.5, 2.0], np.float32)
    rc = lib.hobo_create_terms(C.byref(h), idx.ctypes.data_as(C.c_void_p), frac.ctypes.data_as(C.c_void_p),
                               2, 3, 3, Bd.HOBO_INTEGER)
    assert rc == Bd.HOBO_ERR_NOT_EXACT
    big = np.array([2.0 ** 23, 2.0 ** 23], np.float32)
    rc = lib.hobo_create_terms(C.byref(h), idx.ctypes.data_as(C.c_void_p), big.ctypes.data_as(C.c_void_p),
                               2, 3, 3, Bd.HOBO_INTEGER)
    assert rc == Bd.HOBO_ERR_NOT_EXACT and b"2^24" in lib.hobo_last_error()
    # folding makes +3 and -3 cancel: nothing left, still integer-exact (no GPU
    # work is reached only if the instance is refused; here it is accepted and
    # the device query fails without a GPU, or succeeds with one)


def test_null_instance_calls(lib):
    assert lib.hobo_energy(None, None, 0, None, None, None) == Bd.HOBO_ERR_ARG
    assert lib.hobo_energy_fp64(None, None, 0, None, None) == Bd.HOBO_ERR_ARG
    assert lib.hobo_anneal(None, 0, 0, None, 0, None, None, None, None) == Bd.HOBO_ERR_ARG
    assert lib.hobo_info(None, None) == Bd.HOBO_ERR_ARG
    lib.hobo_destroy(None)


def test_null_handles_and_bad_arguments_of_the_other_entry_points(lib):
    """Network, tensor-train, batch and result-table calls refuse NULL
    handles and out-of-range arguments before any device work."""
    ARG = Bd.HOBO_ERR_ARG
    h = C.c_void_p()
    # network
    assert lib.hobo_mlp_create(C.byref(h), 33, C.c_uint64(0)) == ARG            # not a multiple of 32
    assert lib.hobo_mlp_create(C.byref(h), 2048, C.c_uint64(0)) == ARG
    assert lib.hobo_mlp_create(None, 64, C.c_uint64(0)) == ARG
    assert lib.hobo_mlp_num_params(None) == -1
    assert lib.hobo_mlp_get(None, None, 1) == ARG
    assert lib.hobo_mlp_set(None, None) == ARG
    assert lib.hobo_mlp_forward(None, None, 1, None, None) == ARG
    assert lib.hobo_mlp_score_tables(None, None, 1, 16, C.c_float(32.0), None, None) == ARG
    assert lib.hobo_mlp_set_tensor_cores(None, 1) == ARG
    assert lib.hobo_mlp_check(None, None) == ARG
    assert lib.hobo_mlp_loss_grad(None, None, None, 1, None, None, None) == ARG
    assert lib.hobo_mlp_train_step(None, None, None, 1, C.c_float(1e-3), None, None) == ARG
    assert lib.hobo_mlp_save(None, b"x") == ARG
    assert lib.hobo_mlp_load(C.byref(h), b"/nonexistent/net.bin") == ARG
    assert lib.hobo_anneal_learned(None, None, C.c_uint64(0), 1, None, 0, None, None, None, None) == ARG
    lib.hobo_mlp_destroy(None)
    # tensor train
    ranks = (C.c_int * 3)(1, 2, 1)
    cores = np.zeros(64, np.float32)
    assert lib.hobo_tt_create(None, 2, 4, ranks, cores.ctypes.data_as(C.c_void_p)) == ARG
    assert lib.hobo_tt_create(C.byref(h), 0, 4, ranks, cores.ctypes.data_as(C.c_void_p)) == Bd.HOBO_ERR_ORDER
    bad = (C.c_int * 3)(2, 2, 1)                                                # ranks[0] must be 1
    assert lib.hobo_tt_create(C.byref(h), 2, 4, bad, cores.ctypes.data_as(C.c_void_p)) == ARG
    assert lib.hobo_tt_create(C.byref(h), 2, 4, ranks, None) == ARG
    assert lib.hobo_tt_energy(None, None, 1, None, None) == ARG
    lib.hobo_tt_destroy(None)
    # batches
    assert lib.hobo_batch_create(None, None, 1, None) == ARG
    assert lib.hobo_batch_create(C.byref(h), None, 0, None) == ARG
    assert lib.hobo_batch_layout(None, None, None) == ARG
    assert lib.hobo_batch_anneal(None, None, None, 0, None, None, None, None) == ARG
    assert lib.hobo_batch_launch_shape(None, 0, None, None) == ARG
    # result table
    assert lib.hobo_aggregate(0, None, None, 1, None, None, None, None, None, None) == ARG   # W
    assert lib.hobo_aggregate(1, None, None, -1, None, None, None, None, None, None) == ARG  # B
    assert lib.hobo_aggregate(1, None, None, 4, None, None, None, None, None, None) == ARG   # K NULL


def test_no_exception_crosses_the_abi(lib):
    """A term count no host container can hold is refused with an error code
    (the reservation fails before any index is read) instead of an
    exception escaping the C interface."""
    h = C.c_void_p()
    idx = np.zeros(3, np.int32)
    coef = np.ones(1, np.float32)
    rc = lib.hobo_create_terms(C.byref(h), idx.ctypes.data_as(C.c_void_p), coef.ctypes.data_as(C.c_void_p),
                               C.c_int64(1 << 62), 3, 10, 0)
    assert rc in (Bd.HOBO_ERR_ARG, Bd.HOBO_ERR_OOM)
    assert h.value is None
    assert b"hobo_create_terms" in lib.hobo_last_error()
