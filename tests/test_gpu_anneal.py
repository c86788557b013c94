"""GPU parity of the batched Metropolis annealer (hobo_anneal) against the
CPU oracle: integer instances follow the oracle's trajectories bit for bit;
the tuned and plain kernels agree bit for bit on every instance."""
import numpy as np
import pytest

import gpuh
import polyexp
import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu

TUNED, PLAIN = 0, 1


def _run(h, seed, B, betas, mode, **kw):
    return h.anneal(seed, B, betas, mode=mode, want_final=True, want_accepts=True, **kw)


def _compare_oracle(inst, r, ref, N):
    np.testing.assert_array_equal(gpuh.to_host_bits(r["bestX"], N), ref["bestX"])
    np.testing.assert_array_equal(r["bestE"].cpu().numpy(), ref["bestE"])
    np.testing.assert_array_equal(gpuh.to_host_bits(r["X"], N), ref["X"])
    np.testing.assert_array_equal(r["E"].cpu().numpy().astype(np.float64), ref["E"])
    np.testing.assert_array_equal(r["accepts"].cpu().numpy(), ref["accepts"])


INT_CASES = [
    ("tiny_dense", lambda: W.tiny_dense(1), 0, 64, (5.0, 0.05, 100)),
    ("dense_int_N64", lambda: W.random_sparse(40, 64, 3, 0.5, "int"), 4, 24, (30.0, 0.1, 12)),
    ("order2_N50", lambda: W.random_sparse(41, 50, 2, 0.3, "int"), 0, 40, (10.0, 0.1, 20)),
    ("order3_N45", lambda: W.random_sparse(42, 45, 3, 0.05, "int"), 0, 40, (10.0, 0.1, 20)),
    ("order4_N40", lambda: W.random_sparse(43, 40, 4, 0.02, "int"), 0, 33, (10.0, 0.1, 15)),
    ("order5_N24", lambda: W.random_sparse(44, 24, 5, 0.03, "int"), 0, 20, (10.0, 0.1, 15)),
    ("order6_N20", lambda: W.random_sparse(45, 20, 6, 0.02, "int"), 0, 20, (10.0, 0.1, 15)),
    ("order7_N16", lambda: W.random_sparse(46, 16, 7, 0.03, "int"), 0, 20, (10.0, 0.1, 15)),
    ("order8_N14", lambda: W.random_sparse(47, 14, 8, 0.05, "int"), 0, 20, (10.0, 0.1, 15)),
    ("pythagorean", polyexp.pythagorean, 0, 64, (400.0, 0.05, 60)),
    ("tsp", polyexp.tsp_intenc, 0, 64, (400.0, 0.05, 60)),
    ("int_encoded", lambda: W.int_encoded(3), 0, 48, (2000.0, 0.5, 40)),
]


@pytest.mark.parametrize("name,maker,flags,B,sched", INT_CASES, ids=[c[0] for c in INT_CASES])
@pytest.mark.parametrize("mode", [TUNED, PLAIN])
def test_anneal_integer_matches_oracle(name, maker, flags, B, sched, mode):
    inst = maker()
    betas = W.geometric_betas(*sched)
    h = gpuh.make(inst, flags)
    r = _run(h, 1234, B, betas, mode)
    ref = O.anneal(inst, 1234, B, betas)
    _compare_oracle(inst, r, ref, inst.N)
    h.close()


def _reheat(T0, T1, S):
    """Two geometric legs, the second starting hotter than the first ends."""
    return np.concatenate([W.geometric_betas(T0, T1, S // 2), W.geometric_betas(T0 / 10, T1, S - S // 2)])


LATE_CASES = [
    # long dense anneals: after the first tenth of the sweeps the dense sweep
    # visits only the bits it did not find frozen in the last sweep without
    # flips; these schedules give many such sweeps with more than 32
    # candidates, sweeps where every bit is frozen, and flips found among
    # the candidates (then every later bit of the sweep is visited)
    ("dense_int_N64_cold", lambda: W.random_sparse(40, 64, 3, 0.5, "int"), 4, 32,
     lambda: W.geometric_betas(30.0, 0.05, 300)),
    ("dense_int_N64_warm_end", lambda: W.random_sparse(40, 64, 3, 0.5, "int"), 4, 32,
     lambda: W.geometric_betas(100.0, 0.3, 300)),
    # beta falls at the second leg: the frozen bits must be visited again
    ("dense_int_N64_reheat", lambda: W.random_sparse(40, 64, 3, 0.5, "int"), 4, 32, lambda: _reheat(30.0, 0.05, 300)),
    ("tiny_dense_long", lambda: W.tiny_dense(1), 0, 64, lambda: W.geometric_betas(5.0, 0.02, 400)),
    # ten words per state (N = 300)
    ("dense_int_N300", lambda: W.random_sparse(61, 300, 3, 0.3, "int", imax=2), 4, 8,
     lambda: W.geometric_betas(200.0, 0.5, 120)),
    # odd N: the last bit has no pair partner (N = 45, and N = 289 over ten words)
    ("dense_int_N45_odd", lambda: W.random_sparse(63, 45, 3, 0.5, "int"), 4, 48,
     lambda: W.geometric_betas(30.0, 0.05, 200)),
    ("dense_int_N289_odd", lambda: W.random_sparse(64, 289, 3, 0.3, "int", imax=2), 4, 8,
     lambda: W.geometric_betas(200.0, 0.5, 60)),
]


@pytest.mark.parametrize("name,maker,flags,B,sched", LATE_CASES, ids=[c[0] for c in LATE_CASES])
def test_long_dense_anneal_matches_oracle(name, maker, flags, B, sched):
    inst = maker()
    betas = sched()
    h = gpuh.make(inst, flags)
    r = _run(h, 77, B, betas, TUNED)
    ref = O.anneal(inst, 77, B, betas)
    _compare_oracle(inst, r, ref, inst.N)
    h.close()


@pytest.mark.parametrize("N", [96, 97])
@pytest.mark.parametrize("sched", [lambda: W.geometric_betas(10.0, 0.01, 400), lambda: _reheat(10.0, 0.01, 400)],
                         ids=["geometric", "reheat"])
def test_long_dense_float_anneal_tuned_equals_plain(sched, N):
    inst = W.dense_float(52, N)
    betas = sched()
    h = gpuh.make(inst)
    a = _run(h, 98, 32, betas, TUNED)
    b = _run(h, 98, 32, betas, PLAIN)
    for k in ("bestX", "X", "accepts", "bestE", "E"):
        np.testing.assert_array_equal(a[k].cpu().numpy(), b[k].cpu().numpy())
    h.close()


def test_long_dense_anneal_many_states_match_oracle():
    """A long dense anneal of more states than SMs: trajectories of the
    integer instance follow the oracle for every state."""
    inst = W.random_sparse(62, 72, 3, 0.3, "int", imax=2)
    betas = W.geometric_betas(100.0, 0.1, 100)
    h = gpuh.make(inst, 4)
    r = _run(h, 78, 320, betas, TUNED)
    ref = O.anneal(inst, 78, 320, betas)
    _compare_oracle(inst, r, ref, inst.N)
    h.close()


@pytest.mark.parametrize("N", [128, 256])
def test_long_dense_float_many_states_equal_plain(N):
    """4096 states of a dense float instance (27 per SM) against the plain
    kernel on a slice of 32 of them (their global state indices via
    state0)."""
    inst = W.dense_float(54, N)
    betas = W.geometric_betas(10.0, 0.01, 300)
    h = gpuh.make(inst)
    a = _run(h, 97, 4096, betas, TUNED)
    b = _run(h, 97, 32, betas, PLAIN, state0=1000)
    for k in ("bestX", "X", "accepts", "bestE", "E"):
        np.testing.assert_array_equal(a[k][1000:1032].cpu().numpy(), b[k].cpu().numpy())
    h.check()
    h.close()


WIDE_CASES = [
    # N = 1000: the widest sparse sweep (32 words per state, 8 bits in the last word)
    ("sparse_N1000", lambda: W.random_sparse(60, 1000, 3, 2e-5, "int"), 8, (20.0, 0.5, 4)),
    # N = 300 with the cubic part 30 % full: the dense layout at 10 words per state
    # (12 bits in the last word), wider than the bench instance
    ("dense_N300", lambda: W.random_sparse(61, 300, 3, 0.3, "int", imax=2), 4, (200.0, 1.0, 2)),
]


@pytest.mark.parametrize("name,maker,B,sched", WIDE_CASES, ids=[c[0] for c in WIDE_CASES])
@pytest.mark.parametrize("mode", [TUNED, PLAIN])
def test_anneal_wide_integer_matches_oracle(name, maker, B, sched, mode):
    inst = maker()
    betas = W.geometric_betas(*sched)
    h = gpuh.make(inst, 0)
    if name.startswith("dense"):
        assert h.info()["dense"], "expected the dense layout"
    r = _run(h, 77, B, betas, mode)
    ref = O.anneal(inst, 77, B, betas)
    _compare_oracle(inst, r, ref, inst.N)
    h.close()


def test_paper_examples_reach_printed_ground_energies():
    """Sec. V.B / V.C: the annealer finds the printed ground energies
    (objective = energy + offset = 0)."""
    for inst, ground in ((polyexp.pythagorean(), -30.0), (polyexp.tsp_intenc(), -360.0),
                         (polyexp.seating(), -17.0)):
        h = gpuh.make(inst)
        r = h.anneal(7, 1024, W.geometric_betas(float(np.abs(inst.coef).max()), 0.05, 200))
        assert r["bestE"].min().item() == ground
        assert (r["bestE"].cpu().numpy() >= ground).all()


def test_tiny_reaches_bruteforce_ground_state():
    inst = W.tiny_dense(1)
    Emin = O.bruteforce(inst).min()
    h = gpuh.make(inst)
    T0, T1, S, B = W.SCHEDULES["tiny_dense"]
    r = h.anneal(1, B, W.geometric_betas(T0, T1, S))
    assert r["bestE"].min().item() == Emin


FLOAT_CASES = [
    ("sparse3", lambda: W.random_sparse(50, 90, 3, 0.1, "normal"), 0, 40, (5.0, 0.05, 20)),
    ("sparse4", lambda: W.random_sparse(51, 48, 4, 0.05, "normal"), 0, 40, (5.0, 0.05, 20)),
    ("dense_N64", lambda: W.dense_float(52, 64), 0, 40, (10.0, 0.01, 10)),
    ("dense_N256", lambda: W.dense_float(2), 0, 16, (10.0, 0.01, 3)),
]


@pytest.mark.parametrize("name,maker,flags,B,sched", FLOAT_CASES, ids=[c[0] for c in FLOAT_CASES])
def test_anneal_tuned_equals_plain(name, maker, flags, B, sched):
    inst = maker()
    betas = W.geometric_betas(*sched)
    h = gpuh.make(inst, flags)
    a = _run(h, 99, B, betas, TUNED, want_bytes=True)
    b = _run(h, 99, B, betas, PLAIN, want_bytes=True)
    for k in ("bestX", "X", "accepts", "bestE", "coef_bytes"):
        np.testing.assert_array_equal(a[k].cpu().numpy(), b[k].cpu().numpy())
    np.testing.assert_array_equal(a["E"].cpu().numpy(), b["E"].cpu().numpy())
    # the reported best energies are the float64 energies of the best states
    bx = gpuh.to_host_bits(a["bestX"], inst.N)
    np.testing.assert_allclose(a["bestE"].cpu().numpy(), O.energy(inst, bx), rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("maker", [lambda: W.random_sparse(60, 70, 3, 0.08, "int"),
                                   lambda: W.dense_float(61, 64)])
@pytest.mark.parametrize("mode", [TUNED, PLAIN])
def test_anneal_resume_equals_uninterrupted(maker, mode):
    inst = maker()
    betas = W.geometric_betas(8.0, 0.05, 30)
    h = gpuh.make(inst)
    full = h.anneal(5, 40, betas, mode=mode, want_fields=True, want_accepts=True, want_final=True)
    part = h.anneal(5, 40, betas[:10], mode=mode, want_fields=True, want_accepts=True, want_final=True)
    rest = h.anneal(5, 40, betas[10:], mode=mode, sweep0=10, resume=True, X=part["X"],
                    bestX=part["bestX"], bestE32=part["bestE32"], E=part["E"], g=part["g"],
                    want_final=True, want_accepts=True)
    for k in ("bestX", "X", "bestE", "E", "bestE32", "g"):
        np.testing.assert_array_equal(full[k].cpu().numpy(), rest[k].cpu().numpy())
    np.testing.assert_array_equal(full["accepts"].cpu().numpy(),
                                  part["accepts"].cpu().numpy() + rest["accepts"].cpu().numpy())


def test_anneal_independent_of_batch_size():
    inst = W.random_sparse(62, 100, 3, 0.05, "normal")
    betas = W.geometric_betas(5.0, 0.05, 15)
    h = gpuh.make(inst)
    a = _run(h, 8, 100, betas, TUNED)
    b = _run(h, 8, 37, betas, TUNED)
    np.testing.assert_array_equal(a["bestX"][:37].cpu().numpy(), b["bestX"].cpu().numpy())
    np.testing.assert_array_equal(a["E"][:37].cpu().numpy(), b["E"].cpu().numpy())


@pytest.mark.parametrize("mode", [TUNED, PLAIN])
def test_anneal_resume_from_states_only_integer(mode):
    """Integer instance: resuming from the states alone (fields and
    energies recomputed) continues bit for bit."""
    inst = W.random_sparse(64, 60, 4, 0.03, "int")
    betas = W.geometric_betas(8.0, 0.05, 24)
    h = gpuh.make(inst)
    full = _run(h, 9, 33, betas, mode)
    part = _run(h, 9, 33, betas[:7], mode)
    rest = h.anneal(9, 33, betas[7:], mode=mode, sweep0=7, resume=True, X=part["X"],
                    bestX=part["bestX"], bestE32=part["bestE32"], want_final=True)
    for k in ("bestX", "X", "bestE", "E"):
        np.testing.assert_array_equal(full[k].cpu().numpy(), rest[k].cpu().numpy())


def test_anneal_zero_sweeps_returns_initial_states():
    inst = W.random_sparse(63, 30, 3, 0.1, "int")
    h = gpuh.make(inst)
    r = h.anneal(11, 10, np.zeros(0, np.float32), want_final=True)
    X0 = O.init_states(11, inst.N, 10)
    np.testing.assert_array_equal(gpuh.to_host_bits(r["bestX"], inst.N), X0)
    np.testing.assert_array_equal(r["bestE"].cpu().numpy(), O.energy(inst, X0))


def test_int_encoded_full_size_sampled_states():
    """Integer-encoded workload at full size (B=8192, 2000 sweeps); sampled
    states follow the oracle bit for bit."""
    inst = W.int_encoded(3)
    T0, T1, S, B = W.SCHEDULES["int_encoded"]
    betas = W.geometric_betas(T0, T1, S)
    h = gpuh.make(inst)
    r = _run(h, 3, B, betas, TUNED)
    for b in (0, 4097, B - 1):
        ref = O.anneal(inst, 3, 1, betas, state0=b)
        np.testing.assert_array_equal(gpuh.to_host_bits(r["bestX"][b:b + 1], inst.N), ref["bestX"])
        np.testing.assert_array_equal(r["bestE"][b:b + 1].cpu().numpy(), ref["bestE"])
        np.testing.assert_array_equal(r["accepts"][b:b + 1].cpu().numpy(), ref["accepts"])


def test_sparse_order4_full_size_sampled_states():
    """Order-4 workload (N=96, 2% density) at the size the learned-proposal
    measurement anneals (B=4096, 500 sweeps); sampled states follow the
    oracle bit for bit, and their re-scored energies are the oracle's."""
    inst = W.sparse_order4(5000)
    T0, T1, S, B = W.SCHEDULES["sparse_order4"]
    betas = W.geometric_betas(T0, T1, S)
    h = gpuh.make(inst)
    r = _run(h, 11, B, betas, TUNED)
    for b in (0, 1777, B - 1):
        ref = O.anneal(inst, 11, 1, betas, state0=b)
        np.testing.assert_array_equal(gpuh.to_host_bits(r["bestX"][b:b + 1], inst.N), ref["bestX"])
        np.testing.assert_array_equal(r["bestE"][b:b + 1].cpu().numpy(), ref["bestE"])
        np.testing.assert_array_equal(gpuh.to_host_bits(r["X"][b:b + 1], inst.N), ref["X"])
        np.testing.assert_array_equal(r["accepts"][b:b + 1].cpu().numpy(), ref["accepts"])
    h.close()


def test_dense_float_full_size_best_energies():
    """Dense order-3 N=256 float workload at full size (B=4096, 1000
    sweeps): the float64 re-scored best energies equal the oracle energies
    of the returned states, and improve on the initial states."""
    inst = W.dense_float(2)
    T0, T1, S, B = W.SCHEDULES["dense_float"]
    betas = W.geometric_betas(T0, T1, S)
    h = gpuh.make(inst)
    r = h.anneal(2, B, betas, want_final=True)
    bestE = r["bestE"].cpu().numpy()
    sample = np.array([0, 1, 2047, 4095])
    bx = gpuh.to_host_bits(r["bestX"][sample], inst.N)
    np.testing.assert_allclose(bestE[sample], O.energy(inst, bx), rtol=1e-12, atol=1e-9)
    E0 = O.energy(inst, O.init_states(2, inst.N, 4))
    assert (bestE[:4] < E0).all()
    # the float32 energy tracked along the trajectory (float32 sums of every
    # accepted flip's delta) stays within 1e-4 at the float32-sum floor A / 64
    e32 = r["bestE32"].cpu().numpy().astype(np.float64)
    absi = gpuh.abs_instance(inst)
    assert gpuh.rel_err(e32[sample], bestE[sample], O.energy(absi, bx), gpuh.COND_MAX_F32ACC).max() <= 1e-4


@pytest.mark.parametrize("maker,flags", [(lambda: W.tiny_dense(1), 0), (lambda: W.dense_float(2, N=64), 0),
                                         (lambda: W.sparse_order4(5003), 0)], ids=["tiny", "dense64", "order4"])
@pytest.mark.parametrize("mode", [TUNED, PLAIN])
def test_state_offset_shards_reproduce_one_call(maker, flags, mode):
    """Shards of the state range, each with its global offset, give the
    results of one call on the whole range (the multi-GPU split)."""
    inst = maker()
    betas = W.geometric_betas(5.0, 0.05, 25)
    h = gpuh.make(inst, flags)
    full = _run(h, 9, 70, betas, mode)
    T = gpuh.torch()
    parts = [_run(h, 9, hi - lo, betas, mode, state0=lo) for lo, hi in ((0, 33), (33, 70))]
    for k in ("bestX", "bestE", "X", "E", "accepts"):
        assert T.equal(T.cat([p[k] for p in parts]), full[k]), k
    if inst.integer:
        ref = O.anneal(inst, 9, 37, betas, state0=33)
        np.testing.assert_array_equal(parts[1]["bestE"].cpu().numpy(), ref["bestE"])
    h.close()


DEGENERATE = [
    ("N1_order1", lambda: W.random_sparse(80, 1, 1, 0.0, "int")),           # one variable, E = a x
    ("order1_N40", lambda: W.random_sparse(81, 40, 1, 0.0, "int")),         # no interactions: fields constant
    ("complete_N2_order2", lambda: W.dense_all_degrees(82, 2, 2, "int")),
    ("complete_N3_order3", lambda: W.dense_all_degrees(83, 3, 3, "int")),
]


@pytest.mark.parametrize("name,maker", DEGENERATE, ids=[c[0] for c in DEGENERATE])
@pytest.mark.parametrize("mode", [TUNED, PLAIN])
def test_anneal_degenerate_instances_match_oracle(name, maker, mode):
    """The smallest instances the method has: trajectories bit-exact against
    the oracle (33 states: one full warp and a ragged one), and energies and
    flip deltas of every state of the small ones against brute force."""
    inst = maker()
    betas = W.geometric_betas(5.0, 0.05, 20)
    h = gpuh.make(inst, 0)
    r = _run(h, 5, 33, betas, mode)
    ref = O.anneal(inst, 5, 33, betas)
    _compare_oracle(inst, r, ref, inst.N)
    if inst.N <= 3:
        T = gpuh.torch()
        X = np.array([[(s >> i) & 1 for i in range(inst.N)] for s in range(1 << inst.N)], np.uint8)
        E, dE = h.energy(T.from_numpy(W.pack_bits(X).view(np.int32)).cuda())
        np.testing.assert_array_equal(E.cpu().numpy().astype(np.int64), O.energy_int(inst, X))
        for s in range(1 << inst.N):
            np.testing.assert_array_equal(dE[s].cpu().numpy().astype(np.float64), O.flip_delta(inst, X[s]))
    h.close()
