"""GPU parity of the batched contraction (hobo_energy, hobo_energy_fp64)
against the CPU oracle, through the C ABI."""
import numpy as np
import pytest

import gpuh
import polyexp
import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _check_int(inst, X, flags=0, path=0):
    import paper_2407_19987_gb300 as H
    h = gpuh.make(inst, flags)
    Xd = gpuh.to_dev(X)
    E, dE = h.energy(Xd, path=path)
    E = E.cpu().numpy().astype(np.float64)
    dE = dE.cpu().numpy().astype(np.float64)
    refE = O.energy_int(inst, X).astype(np.float64)
    np.testing.assert_array_equal(E, refE)
    for b in range(X.shape[0]):
        g = O.fields(inst, X[b])
        np.testing.assert_array_equal(dE[b], (1.0 - 2.0 * X[b]) * g)
    E64 = h.energy_fp64(Xd).cpu().numpy()
    np.testing.assert_array_equal(E64, refE)
    h.close()


INT_CASES = [
    ("tiny_dense", lambda: W.tiny_dense(1)),
    ("order1_N1", lambda: W.Instance(1, 1, np.array([[0]], np.int32), np.array([-3], np.float32), integer=True)),
    ("order2_N33", lambda: W.random_sparse(31, 33, 2, 0.4, "int")),
    ("order3_N32", lambda: W.random_sparse(32, 32, 3, 0.2, "int")),
    ("order3_N70", lambda: W.random_sparse(33, 70, 3, 0.05, "int")),
    ("order4_N40", lambda: W.random_sparse(34, 40, 4, 0.02, "int")),
    ("order5_N20", lambda: W.random_sparse(35, 20, 5, 0.05, "int")),
    ("order6_N16", lambda: W.random_sparse(36, 16, 6, 0.05, "int")),
    ("order7_N14", lambda: W.random_sparse(37, 14, 7, 0.05, "int")),
    ("order8_N13", lambda: W.random_sparse(38, 13, 8, 0.06, "int")),
    ("pythagorean", polyexp.pythagorean),
    ("tsp", polyexp.tsp_intenc),
    ("seating", polyexp.seating),
    ("int_encoded", lambda: W.int_encoded(3)),
]


@pytest.mark.parametrize("name,maker", INT_CASES, ids=[c[0] for c in INT_CASES])
@pytest.mark.parametrize("B", [1, 33, 100])
def test_energy_integer_exact(name, maker, B):
    inst = maker()
    X = W.random_states(100 + B, B, inst.N)
    _check_int(inst, X)


def test_energy_dense_int_forced_dense():
    inst = W.random_sparse(40, 64, 3, 0.5, "int")
    X = W.random_states(41, 77, inst.N)
    _check_int(inst, X, flags=4)   # HOBO_FORCE_DENSE


def test_energy_dense_entries_below_diagonal():
    """hobo_create folds every entry of a full dense tensor (not only the
    upper part) onto its distinct index set."""
    import paper_2407_19987_gb300 as H
    rng = np.random.default_rng(5)
    N, k = 9, 3
    T = rng.integers(-5, 6, size=(N,) * k).astype(np.float32)
    grid = np.stack(np.meshgrid(*[np.arange(N)] * k, indexing="ij"), -1).reshape(-1, k).astype(np.int32)
    inst = W.Instance(N, k, grid, T.reshape(-1), integer=True)
    h = H.Instance.from_dense(T)
    X = W.random_states(6, 40, N)
    E, dE = h.energy(gpuh.to_dev(X))
    np.testing.assert_array_equal(E.cpu().numpy(), O.energy_int(inst, X).astype(np.float32))
    for b in range(40):
        np.testing.assert_array_equal(dE[b].cpu().numpy(), ((1.0 - 2.0 * X[b]) * O.fields(inst, X[b])).astype(np.float32))


FLOAT_CASES = [
    ("order3_sparse", lambda: W.random_sparse(50, 90, 3, 0.1, "normal")),
    ("order4_sparse", lambda: W.random_sparse(51, 48, 4, 0.05, "normal")),
    ("order3_dense_N48", lambda: W.dense_float(52, 48)),
    ("order2_N200", lambda: W.random_sparse(53, 200, 2, 0.5, "normal")),
]


@pytest.mark.parametrize("name,maker", FLOAT_CASES, ids=[c[0] for c in FLOAT_CASES])
@pytest.mark.parametrize("path", [0, 1])
def test_energy_float_within_tolerance(name, maker, path):
    inst = maker()
    h = gpuh.make(inst)
    X = W.random_states(60, 70, inst.N)
    E, dE = h.energy(gpuh.to_dev(X), path=path)
    E = E.cpu().numpy().astype(np.float64)
    dE = dE.cpu().numpy().astype(np.float64)
    absi = gpuh.abs_instance(inst)
    refE = O.energy(inst, X)
    assert gpuh.rel_err(E, refE, O.energy(absi, X)).max() <= gpuh.FLOAT_RTOL
    for b in range(X.shape[0]):
        g = O.fields(inst, X[b])
        ga = O.fields(absi, X[b])
        assert gpuh.rel_err(dE[b], (1.0 - 2.0 * X[b]) * g, ga).max() <= gpuh.FLOAT_RTOL
    E64 = h.energy_fp64(gpuh.to_dev(X)).cpu().numpy()
    np.testing.assert_allclose(E64, refE, rtol=1e-12, atol=1e-9)


def test_energy_dense_float_full_size_sampled():
    """Dense order-3 N=256 float instance (every i<=j<=k entry N(0,1)),
    B=4096 states in one call.  On 64 sampled states, every energy and all
    256 flip deltas of each: the tensor-core path (exact fixed-point limbs)
    and the term-list path are equal bit for bit, and each value is the
    oracle's float64 value rounded once to float32 up to the fixed-point
    rounding of the coefficients (at most 2^-(S+1) per term): |got - ref| <=
    2^-24 |ref| + M 2^-S, M the number of monomials.  That meets the
    relative bar with the floor A/1024.  The true relative error
    |got - ref| / |ref| over the values above that floor is printed, with
    the same figures for the float32-accumulating tensor-core kernel."""
    import paper_2407_19987_gb300 as H
    inst = W.dense_float(2)
    h = gpuh.make(inst)
    info = h.info()
    S = gpuh.fix_shift(info["abs_sum"])
    M = int(sum(info["terms"]))
    B = 4096
    X = W.random_states(61, B, inst.N)
    Xd = gpuh.to_dev(X)
    out = {}
    for path in (H.PATH_TENSOR_CORE, H.PATH_TERMS, H.PATH_TENSOR_CORE_F32ACC):
        E, dE = h.energy(Xd, path=path)
        out[path] = (E.cpu().numpy().astype(np.float64), dE.cpu().numpy().astype(np.float64))
    np.testing.assert_array_equal(out[H.PATH_TENSOR_CORE][0], out[H.PATH_TERMS][0])
    np.testing.assert_array_equal(out[H.PATH_TENSOR_CORE][1], out[H.PATH_TERMS][1])
    absi = gpuh.abs_instance(inst)
    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([[0, 1, 127, 128, B - 1], rng.choice(B, 59, replace=False)]))
    refE, AE = O.energy(inst, X[rows]), O.energy(absi, X[rows])
    refD = np.stack([(1.0 - 2.0 * X[b]) * O.fields(inst, X[b]) for b in rows])
    AD = np.stack([O.fields(absi, X[b]) for b in rows])
    quant = M * 2.0 ** -S
    report = {}
    for path, name in ((H.PATH_TENSOR_CORE, "tensor_core_exact"), (H.PATH_TERMS, "term_list"),
                       (H.PATH_TENSOR_CORE_F32ACC, "tensor_core_f32acc")):
        E, dE = out[path][0][rows], out[path][1][rows]
        for what, got, ref, A in (("E", E, refE, AE), ("dE", dE, refD, AD)):
            err = np.abs(got - ref)
            above = np.abs(ref) >= A / gpuh.COND_MAX
            true_rel = (err[above] / np.abs(ref[above])).max() if above.any() else 0.0
            report[f"{name}.{what}"] = {"max_true_rel_above_floor": float(true_rel),
                                        "share_above_floor": float(above.mean()),
                                        "max_bar_err": float(gpuh.rel_err(got, ref, A).max())}
            if path == H.PATH_TENSOR_CORE_F32ACC:
                assert gpuh.rel_err(got, ref, A, gpuh.COND_MAX_F32ACC).max() <= gpuh.FLOAT_RTOL
            else:
                assert np.all(err <= 2.0 ** -24 * np.abs(ref) + quant), (name, what)
                assert gpuh.rel_err(got, ref, A).max() <= gpuh.FLOAT_RTOL
                assert true_rel <= gpuh.FLOAT_RTOL
    print("relative error, dense N=256 float, 64 states:", report)
    h.close()


def test_energy_wide_instance_N1024():
    inst = W.random_sparse(70, 1024, 2, 0.002, "int")
    X = W.random_states(71, 5, inst.N)
    _check_int(inst, X)


def test_energy_empty_batch_and_no_delta():
    import torch
    inst = W.tiny_dense(1)
    h = gpuh.make(inst)
    X = torch.zeros((0, 1), dtype=torch.int32, device="cuda")
    E, dE = h.energy(X)
    assert E.numel() == 0
    Xs = W.random_states(3, 10, inst.N)
    E, dE = h.energy(gpuh.to_dev(Xs), with_delta=False)
    assert dE is None
    np.testing.assert_array_equal(E.cpu().numpy(), O.energy_int(inst, Xs).astype(np.float32))


def test_energy_ignores_bits_beyond_N():
    inst = W.random_sparse(80, 37, 3, 0.1, "int")
    X = W.random_states(81, 20, inst.N)
    P = W.pack_bits(X)
    P[:, -1] |= np.uint32(0xFFFFFFFF) << np.uint32(37 - 32)
    import torch
    h = gpuh.make(inst)
    E, dE = h.energy(torch.from_numpy(P.view(np.int32)).cuda())
    np.testing.assert_array_equal(E.cpu().numpy(), O.energy_int(inst, X).astype(np.float32))


TC_CASES = [(12, 1), (12, 129), (33, 100), (64, 128), (64, 300), (200, 77), (256, 129)]


@pytest.mark.parametrize("N,B", TC_CASES, ids=[f"N{n}_B{b}" for n, b in TC_CASES])
def test_tensor_core_path_integer_exact(N, B):
    """tcgen05 contraction (path 2) on dense order-3 integer instances:
    ragged state tiles (B not a multiple of 128) and ragged N (not a
    multiple of 16/64) give exact energies and flip deltas."""
    inst = W.random_sparse(90 + N, N, 3, 0.6, "int")
    X = W.random_states(91 + B, B, N)
    _check_int(inst, X, flags=4, path=2)


def test_tensor_core_three_plane_split_large_integers():
    """Coefficients >= 2^16 need the hi+mid+lo split to stay exact."""
    inst = W.random_sparse(95, 10, 3, 1.0, "int", imax=100000)
    assert np.abs(inst.coef).max() >= 2 ** 16
    X = W.random_states(96, 50, inst.N)
    _check_int(inst, X, flags=4, path=2)


@pytest.mark.parametrize("N,B", [(96, 200), (33, 129), (200, 300), (256, 129), (7, 5)])
def test_tensor_core_matches_term_path_float(N, B):
    """Both paths sum the same fixed-point integers exactly and round them
    once: equal energies and flip deltas, bit for bit, on ragged sizes (N
    not a multiple of 64, B not a multiple of 128), with and without the
    deltas."""
    inst = W.dense_float(97 + N, N)
    h = gpuh.make(inst)
    X = gpuh.to_dev(W.random_states(98, B, inst.N))
    E2, d2 = h.energy(X, path=2)
    E1, d1 = h.energy(X, path=1)
    np.testing.assert_array_equal(E2.cpu().numpy(), E1.cpu().numpy())
    np.testing.assert_array_equal(d2.cpu().numpy(), d1.cpu().numpy())
    E2o, _ = h.energy(X, with_delta=False, path=2)
    np.testing.assert_array_equal(E2o.cpu().numpy(), E1.cpu().numpy())
    h.check()
    h.close()


def test_tensor_core_path_refused_for_sparse_instance():
    import paper_2407_19987_gb300 as H
    inst = W.random_sparse(99, 40, 3, 0.05, "int")
    h = gpuh.make(inst)
    with pytest.raises(H.HoboError) as ei:
        h.energy(gpuh.to_dev(W.random_states(1, 4, inst.N)), path=2)
    assert ei.value.code == -7


def test_check_reports_no_timeout_after_normal_work():
    inst = W.dense_float(100, 64)
    h = gpuh.make(inst)
    h.energy(gpuh.to_dev(W.random_states(2, 64, inst.N)))
    h.check()


def test_bounded_wait_timeout_is_reported_and_context_survives():
    """A bounded device wait on a barrier nothing completes gives up after
    its limit; hobo_check reports HOBO_ERR_TIMEOUT once, and the context
    keeps working (the contraction afterwards matches the oracle)."""
    import paper_2407_19987_gb300 as H
    inst = W.dense_float(100, 64)
    h = gpuh.make(inst)
    h.selftest_timeout(20_000_000)
    with pytest.raises(H.HoboError) as ei:
        h.check()
    assert ei.value.code == H.HOBO_ERR_TIMEOUT
    h.check()                                   # status cleared
    X = W.random_states(3, 16, inst.N)
    E, _ = h.energy(gpuh.to_dev(X))
    ref = O.energy(inst, X)
    assert np.all(gpuh.rel_err(E.cpu().numpy().astype(np.float64), ref, O.energy(gpuh.abs_instance(inst), X))
                  <= gpuh.FLOAT_RTOL)
    with pytest.raises(H.HoboError):
        h.selftest_timeout(0)


@pytest.mark.parametrize("N,B,integer", [(12, 300, True), (33, 129, False), (64, 300, True), (200, 257, False),
                                         (256, 4096, False)])
def test_exact_tensor_core_rescore_equals_cuda_core_rescore(N, B, integer):
    """The float64 re-score on the tensor cores (8-bit limb planes of the
    fixed-point coefficients) gives exactly the CUDA-core re-score's
    values: both round the same exact integer once; integer instances also
    equal the oracle's int64 energies."""
    import paper_2407_19987_gb300 as H
    inst = W.random_sparse(70 + N, N, 3, 0.6, "int") if integer else W.dense_float(71, N)
    X = W.random_states(72, B, N)
    Xd = gpuh.to_dev(X)
    flags = H.HOBO_FORCE_DENSE
    h_tc = gpuh.make(inst, flags)
    h_cc = gpuh.make(inst, flags | H.HOBO_RESCORE_CUDA_CORES)
    assert h_tc.info()["dense"] and h_cc.info()["dense"]
    e_tc = h_tc.energy_fp64(Xd).cpu().numpy()
    e_cc = h_cc.energy_fp64(Xd).cpu().numpy()
    np.testing.assert_array_equal(e_tc, e_cc)
    if integer:
        np.testing.assert_array_equal(e_tc, O.energy_int(inst, X).astype(np.float64))
    else:
        rows = np.arange(0, B, max(1, B // 64))
        np.testing.assert_allclose(e_tc[rows], O.energy(inst, X[rows]), rtol=1e-12, atol=1e-9)
    h_tc.check()
    h_tc.close()
    h_cc.close()


def test_dense_rescore_above_tensor_core_size():
    """Dense layout with N > 256 (no tensor-core planes): the CUDA-core
    exact re-score against the oracle's int64 energies."""
    import paper_2407_19987_gb300 as H
    inst = W.random_sparse(80, 300, 3, 0.3, "int")
    h = gpuh.make(inst, H.HOBO_FORCE_DENSE)
    assert h.info()["dense"]
    X = W.random_states(81, 40, inst.N)
    np.testing.assert_array_equal(h.energy_fp64(gpuh.to_dev(X)).cpu().numpy(),
                                  O.energy_int(inst, X).astype(np.float64))
    h.close()
