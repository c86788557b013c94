"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(not against a retyping of its own formulas).  CPU only."""
import json
import math
import os
import struct

import numpy as np
import pytest

import polyexp
import workloads as W
from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")


def gold():
    with open(GOLD) as f:
        return json.load(f)


# ---------------------------------------------------------------- energy

def test_energy_qubo_closed_form():
    """Order 2 (Sec. II.B QUBO): E = x^T Q x with the linear terms on the
    diagonal of an upper-triangular Q, evaluated by numpy matmul."""
    rng = np.random.default_rng(11)
    N = 20
    Q = np.triu(rng.integers(-9, 10, size=(N, N))).astype(np.float64)
    iu = np.array([(i, j) for i in range(N) for j in range(i, N) if Q[i, j] != 0], np.int32)
    inst = W.Instance(N, 2, iu, Q[iu[:, 0], iu[:, 1]].astype(np.float32), integer=True)
    X = W.random_states(5, 64, N)
    ref = np.einsum("bi,ij,bj->b", X.astype(np.float64), Q, X.astype(np.float64))
    np.testing.assert_array_equal(O.energy(inst, X), ref)
    np.testing.assert_array_equal(O.energy_int(inst, X), ref.astype(np.int64))


def test_energy_matches_dense_einsum():
    """Sec. IV.C batched contraction E_b = sum_ijk H_ijk X_bi X_bj X_bk,
    evaluated by numpy einsum over the dense tensor, equals the oracle's
    entry-by-entry sum (integers: exact)."""
    inst = W.tiny_dense(1)
    T = inst.dense().astype(np.float64)
    X = W.random_states(7, 200, inst.N).astype(np.float64)
    ref = np.einsum("ijk,bi,bj,bk->b", T, X, X, X)
    np.testing.assert_array_equal(O.energy(inst, X.astype(np.uint8)), ref)


def test_energy_order4_random_float_einsum():
    inst = W.random_sparse(21, 14, 4, 0.3, "normal")
    T = inst.dense().astype(np.float64)
    X = W.random_states(8, 50, inst.N).astype(np.float64)
    ref = np.einsum("ijkl,bi,bj,bk,bl->b", T, X, X, X, X)
    # oracle adds the float32 entries in float64; dense() rounds entries that
    # share a tuple (none here) -> both sums agree to fp64 rounding
    np.testing.assert_allclose(O.energy(inst, X.astype(np.uint8)), ref, rtol=1e-12, atol=1e-9)


def test_bruteforce_tiny_dense_ground_state():
    """All 4096 energies of the N=12 order-3 instance; the minimum is the
    ground state (the tiny workload's target)."""
    inst = W.tiny_dense(1)
    E = O.bruteforce(inst)
    s = np.arange(1 << inst.N)
    X = ((s[:, None] >> np.arange(inst.N)) & 1).astype(np.uint8)
    np.testing.assert_array_equal(E, O.energy_int(inst, X).astype(np.float64))
    T = inst.dense().astype(np.float64)
    Xf = X.astype(np.float64)
    ref = np.einsum("ijk,bi,bj,bk->b", T, Xf, Xf, Xf)
    np.testing.assert_array_equal(E, ref)


def test_batched_equals_single():
    inst = W.random_sparse(3, 30, 3, 0.2, "normal")
    X = W.random_states(3, 10, inst.N)
    Eb = O.energy(inst, X)
    for b in range(10):
        assert O.lib().orc_energy(*(O._p(a) for a in O._terms(inst)[:2]), inst.nnz, inst.order,
                                  O._p(np.ascontiguousarray(X[b]))) == Eb[b]


# ---------------------------------------------------------------- deltas / fields

@pytest.mark.parametrize("maker", [lambda: W.tiny_dense(1), lambda: W.random_sparse(4, 25, 4, 0.2, "int"),
                                   lambda: W.random_sparse(5, 18, 5, 0.1, "normal")])
def test_flip_identity(maker):
    """E(x with bit i flipped) - E(x) = (1 - 2 x_i) g_i (multilinearity)."""
    inst = maker()
    for x in W.random_states(9, 8, inst.N):
        d = O.flip_delta(inst, x)
        g = O.fields(inst, x)
        np.testing.assert_allclose(d, (1.0 - 2.0 * x) * g, rtol=1e-12, atol=1e-9)


def test_euler_identity_per_degree():
    """For the degree-d part E_d of a multilinear polynomial,
    sum_i x_i g_i(E_d) = d * E_d(x)."""
    inst = W.random_sparse(6, 22, 4, 0.25, "int")
    deg = np.array([len(set(r)) for r in inst.idx.tolist()])
    for d in range(1, 5):
        sub = W.Instance(inst.N, inst.order, inst.idx[deg == d], inst.coef[deg == d], integer=True)
        for x in W.random_states(10 + d, 6, inst.N):
            g = O.fields(sub, x)
            assert float(np.dot(x, g)) == d * O.energy(sub, x[None])[0]


def test_replicate_smallest_storage_is_energy_preserving():
    """Sec. III.C: c_ijk stored as c_iiijk in an order-5 tensor gives the
    same energies for binary x."""
    inst = W.random_sparse(7, 15, 3, 0.3, "int")
    idx5 = np.array([W.pad_smallest(tuple(sorted(set(r))), 5) for r in inst.idx.tolist()], np.int32)
    inst5 = W.Instance(inst.N, 5, idx5, inst.coef, integer=True)
    X = W.random_states(12, 100, inst.N)
    np.testing.assert_array_equal(O.energy_int(inst, X), O.energy_int(inst5, X))


# ---------------------------------------------------------------- paper examples

def _ground(inst):
    E = O.bruteforce(inst)
    m = E.min()
    return m, set(np.nonzero(E == m)[0].tolist())


@pytest.mark.slow
def test_paper_seating():
    g = gold()["seating5x5"]
    inst = polyexp.seating()
    assert inst.offset == g["offset"]
    m, states = _ground(inst)
    assert m == g["energy"]
    for grid in g["states_rowmajor_5x5"]:
        bits = np.array(grid, np.uint8).reshape(-1)
        s = int(sum(int(b) << i for i, b in enumerate(bits)))
        assert s in states
        assert O.energy(inst, bits[None])[0] == g["energy"]
    # 17 seats with no three in a line: the five grids found by enumeration
    assert len(states) == 5


def test_paper_pythagorean():
    g = gold()["pythagorean"]
    inst = polyexp.pythagorean()
    assert inst.order == 4 and inst.N == 12
    assert inst.offset == g["offset"]
    m, states = _ground(inst)
    assert m == g["energy"]
    assert len(states) == g["solutions_stated"]

    def enc(x, y, z):
        return sum(((v >> b) & 1) << (4 * a + b) for a, v in enumerate((x, y, z)) for b in range(4))

    for xyz in g["xyz"]:
        assert enc(*xyz) in states
    # closed form: the ground states are exactly the Pythagorean triples
    # with all three entries in 1..15
    trip = {enc(x, y, z) for x in range(1, 16) for y in range(1, 16) for z in range(1, 16)
            if x * x + y * y == z * z}
    assert trip == states


def test_paper_tsp_integer_encoding():
    g = gold()["tsp_intenc"]
    inst = polyexp.tsp_intenc()
    assert inst.order == 6 and inst.N == 6
    assert inst.offset == g["offset"]
    m, states = _ground(inst)
    assert m == g["energy"]

    def enc(b, c, d):
        bits = []
        for v in (b, c, d):
            bits += [(v >> 1) & 1, v & 1]   # most significant bit first
        return sum(bit << i for i, bit in enumerate(bits))

    for xbcd in g["xBCD"]:
        assert enc(*xbcd) in states
    # closed form: xB*xC*xD = 6 with entries in 0..3 <=> a permutation of 1,2,3
    perms = {enc(a, b, c) for a in range(4) for b in range(4) for c in range(4) if a * b * c == 6}
    assert perms == states and len(states) == 6


def test_tsp_einsum_path_flops():
    """Sec. VI.F: the printed einsum-path report for the (6,)^6 tensor is
    numpy's default (greedy) path, which contracts the tensor with one
    vector at a time: the (N^(k-1) x N) . x order the contraction kernels use."""
    g = gold()["tsp_einsum_path"]
    x = np.ones(6)
    T = np.ones((6,) * 6)
    path, report = np.einsum_path("i,j,k,l,m,n,ijklmn->", x, x, x, x, x, x, T, optimize="greedy")
    lines = {l.split(":")[0].strip(): l.split(":")[1].strip() for l in report.splitlines() if ":" in l}
    assert float(lines["Naive FLOP count"]) == g["naive_flops"]
    assert float(lines["Optimized FLOP count"]) == g["optimized_flops"]
    assert float(lines["Largest intermediate"].split()[0]) == g["largest_intermediate"]
    # every step contracts the big tensor with one vector
    assert all(len(step) == 2 for step in path[1:])


# ---------------------------------------------------------------- integer encoding

def test_integer_encoding_round_trip():
    """Sec. IV.B: the bit-level tensor of the integer-encoded workload gives
    the integer objective (evaluated directly on y) minus its offset."""
    inst = W.int_encoded(3)
    m = inst.meta
    X = W.random_states(13, 40, inst.N)
    y = (X.reshape(40, m["n_ints"], m["bits"]) * (1 << np.arange(m["bits"]))).sum(axis=2).astype(np.int64)
    obj = np.zeros(40, np.int64)
    for (a, b, c), w in zip(m["trip"], m["w"]):
        obj += int(w) * y[:, a] * y[:, b] * y[:, c]
    obj += m["penalty"] * (y.sum(axis=1) - m["target"]) ** 2
    np.testing.assert_array_equal(O.energy_int(inst, X), obj - int(inst.offset))
    # the exactness bound the float32 path relies on: sum |folded coef| < 2^24
    folded = {}
    for r, c in zip(inst.idx.tolist(), inst.coef.tolist()):
        k = tuple(sorted(set(r)))
        folded[k] = folded.get(k, 0) + c
    assert sum(abs(v) for v in folded.values()) < 2 ** 24


# ---------------------------------------------------------------- RNG / exp2 / acceptance

def test_philox_known_answers():
    """Philox4x32-10 known-answer vectors published with the generator
    (Salmon et al., SC'11, Random123 distribution)."""
    kat = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for ctr, key, out in kat:
        assert O.philox(ctr, key).tolist() == out


def test_philox_uniformity():
    """Sanity: top bits of many words are balanced."""
    w = np.array([O.philox([i, 0, 0, 0], [1, 2]) for i in range(4096)], dtype=np.uint64).ravel()
    frac = float(((w >> 31) & 1).mean())
    assert abs(frac - 0.5) < 0.02


def test_exp2_constants_are_nearest_floats():
    """The polynomial coefficients in hobo_oracle.c are the float32 values
    nearest to (ln 2)^k / k!, and the log2(e) constant nearest to 1/ln 2."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    src = open(os.path.join(os.path.dirname(O.__file__), "hobo_oracle.c")).read()
    want = {}
    for k in range(7):
        want[k] = mpmath.log(2) ** k / mpmath.factorial(k)

    def nearest(v):
        f = np.float32(float(v))
        c = [np.nextafter(f, np.float32(-1)), f, np.nextafter(f, np.float32(2))]
        return min(c, key=lambda q: abs(mpmath.mpf(float(q)) - v))

    for k in range(1, 7):
        h = "0x%08X" % struct.unpack("<I", struct.pack("<f", nearest(want[k])))[0]
        assert h + "u" in src, (k, h)
    h = "0x%08X" % struct.unpack("<I", struct.pack("<f", nearest(1 / mpmath.log(2))))[0]
    assert h + "u" in src


def test_exp2_error_bound():
    """|exp2own(t) - 2^t| <= 4e-7 * 2^t on [-125, 0]; 0 below -125."""
    ts = np.concatenate([np.linspace(-125, 0, 20011), -np.logspace(-8, 2, 2000),
                         np.arange(-125, 1, 0.5)]).astype(np.float32)
    got = np.array([O.exp2(t) for t in ts], dtype=np.float64)
    ref = np.exp2(ts.astype(np.float64))
    rel = np.abs(got - ref) / ref
    assert rel.max() <= 4e-7, rel.max()
    assert O.exp2(0.0) == 1.0
    assert O.exp2(-125.5) == 0.0 and O.exp2(-1e30) == 0.0


def test_metropolis_rule():
    assert O.metropolis(-3.0, 1.0, 0xFFFFFFFF)         # downhill always
    assert O.metropolis(0.0, 100.0, 0xFFFFFFFF)        # flat always
    assert O.metropolis(5.0, 0.0, 0xFFFFFFFF)          # infinite temperature
    assert not O.metropolis(1000.0, 10.0, 0)           # u=0 < p=0 is false
    # acceptance frequency matches exp(-beta dE) over uniform words
    rng = np.random.default_rng(0)
    ws = rng.integers(0, 2 ** 32, size=20000, dtype=np.uint64)
    f = np.mean([O.metropolis(1.0, 0.7, int(w)) for w in ws])
    assert abs(f - math.exp(-0.7)) < 0.01


# ---------------------------------------------------------------- annealer

def test_anneal_incremental_equals_reevaluation():
    """The incremental-field annealer makes exactly the decisions of the
    annealer that re-evaluates E for every trial flip (integer instance)."""
    inst = W.tiny_dense(1)
    betas = W.geometric_betas(5.0, 0.05, 40)
    a = O.anneal(inst, 123, 32, betas)
    b = O.anneal(inst, 123, 32, betas, naive=True)
    for k in ("X", "E", "bestX", "bestE", "accepts"):
        np.testing.assert_array_equal(a[k], b[k])
    np.testing.assert_array_equal(O.energy(inst, a["X"]), a["E"])
    np.testing.assert_array_equal(O.energy(inst, a["bestX"]), a["bestE"])


def test_anneal_order4_incremental_equals_reevaluation():
    inst = W.random_sparse(8, 16, 4, 0.15, "int")
    betas = W.geometric_betas(6.0, 0.1, 20)
    a = O.anneal(inst, 7, 8, betas)
    b = O.anneal(inst, 7, 8, betas, naive=True)
    for k in ("X", "E", "bestX", "bestE", "accepts"):
        np.testing.assert_array_equal(a[k], b[k])


def test_anneal_reaches_ground_state_tiny():
    inst = W.tiny_dense(1)
    E = O.bruteforce(inst)
    betas = W.geometric_betas(5.0, 0.05, 100)
    r = O.anneal(inst, 1, 64, betas)
    assert r["bestE"].min() == E.min()
    assert (r["bestE"] >= E.min()).all()


def test_anneal_paper_examples_reach_ground():
    for inst, ground in ((polyexp.pythagorean(), -30.0), (polyexp.tsp_intenc(), -360.0)):
        scale = float(np.abs(inst.coef).max())
        betas = W.geometric_betas(scale, 0.05, 200)
        r = O.anneal(inst, 5, 64, betas)
        assert r["bestE"].min() == ground


def test_init_states_layout():
    X = O.init_states(99, 70, 3)
    for b in range(3):
        for i in (0, 1, 5, 69):
            w = O.philox([i >> 2, 0, b, 1], [99, 0])[i & 3]
            assert X[b, i] == (w >> 31)


def test_anneal_recording_and_offset_states():
    inst = W.random_sparse(9, 20, 3, 0.3, "int")
    betas = W.geometric_betas(4.0, 0.1, 10)
    full = O.anneal(inst, 3, 6, betas, rec_B=6)
    part = O.anneal(inst, 3, 3, betas, state0=3)
    np.testing.assert_array_equal(full["bestX"][3:], part["bestX"])
    np.testing.assert_array_equal(full["rec"][-1], full["X"])


def test_aggregate_hand_example():
    """Result table: distinct states by energy, ties by first index, with
    occurrence counts (the sampler output of Sec. V)."""
    a, b, c = [1, 0, 1], [0, 1, 1], [1, 1, 0]
    X = np.array([a, b, a, c, b, a], np.uint8)
    E = np.array([1.0, 0.0, 1.0, 0.0, 0.0, 1.0])
    S, UE, cnt, first = O.aggregate(X, E)
    np.testing.assert_array_equal(S, np.array([b, c, a], np.uint8))
    np.testing.assert_array_equal(UE, [0.0, 0.0, 1.0])
    np.testing.assert_array_equal(cnt, [2, 1, 3])
    np.testing.assert_array_equal(first, [1, 3, 0])


def test_aggregate_properties():
    rng = np.random.default_rng(5)
    pool = rng.integers(0, 2, size=(15, 9)).astype(np.uint8)
    pick = rng.integers(0, 15, size=400)
    X = pool[pick]
    E = (X.astype(np.int64) * np.arange(9)).sum(1).astype(np.float64) % 5
    S, UE, cnt, first = O.aggregate(X, E)
    assert cnt.sum() == 400 and len({s.tobytes() for s in S}) == len(S)
    for s, f, k in zip(S, first, cnt):
        rows = np.nonzero((X == s).all(1))[0]
        assert rows[0] == f and len(rows) == k
    keys = list(zip(UE, first))
    assert keys == sorted(keys)


def test_tt_decomposition_of_the_tsp_tensor_has_the_printed_bond_dimensions():
    """Sec. VI.F: the order-6 (6,...,6) TSP tensor decomposes exactly into
    cores (6,2), (2,6,3), (3,6,4), (4,6,4), (4,6,2), (2,6); the train
    reproduces the tensor and its energies on all 64 states."""
    inst = polyexp.tsp_intenc()
    T = inst.dense().astype(np.float64)
    cores = O.tt_svd(T)
    assert [G.shape for G in cores] == [(1, 6, 2), (2, 6, 3), (3, 6, 4), (4, 6, 4), (4, 6, 2), (2, 6, 1)]
    np.testing.assert_allclose(O.tt_full(cores), T, atol=1e-9 * np.abs(T).max())
    X = np.array([[(s >> i) & 1 for i in range(6)] for s in range(64)], np.uint8)
    np.testing.assert_allclose(O.tt_energy(cores, X), O.energy(inst, X), atol=1e-7)


def test_tt_network_einsum_path_matches_report():
    """Sec. VI.F: numpy's path for x contracted with the six cores costs 701
    flops with a largest intermediate of 16 elements."""
    shapes = [(6, 2), (2, 6, 3), (3, 6, 4), (4, 6, 4), (4, 6, 2), (2, 6)]
    ops = [np.ones(6)] * 6 + [np.ones(s) for s in shapes]
    _, info = np.einsum_path("i,j,k,l,m,n,iA,AjB,BkC,ClD,DmE,En->", *ops, optimize="greedy")
    assert "7.010e+02" in info and "1.600e+01" in info


def test_tt_energy_closed_forms():
    """A rank-1 train is an outer product: E = prod_c (g_c . x); a random
    train equals the energy of its full tensor by brute force."""
    rng = np.random.default_rng(9)
    gs = [rng.standard_normal(7) for _ in range(3)]
    cores = [g.reshape(1, 7, 1) for g in gs]
    X = rng.integers(0, 2, size=(20, 7))
    np.testing.assert_allclose(O.tt_energy(cores, X), np.prod([X @ g for g in gs], axis=0), rtol=1e-12)
    cores = [rng.standard_normal((1, 5, 3)), rng.standard_normal((3, 5, 2)), rng.standard_normal((2, 5, 1))]
    A = O.tt_full(cores)
    X = np.array([[(s >> i) & 1 for i in range(5)] for s in range(32)], np.float64)
    want = np.einsum("ijk,bi,bj,bk->b", A, X, X, X)
    np.testing.assert_allclose(O.tt_energy(cores, X), want, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(O.tt_full(O.tt_svd(A)), A, atol=1e-10)
