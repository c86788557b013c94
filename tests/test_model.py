"""Host front end (paper_2407_19987_gb300.model): polynomials over binary
variables with x*x = x, integer encodings (Sec. IV.B), compilation to
tensor entries with the smallest index repeated (Sec. III.C).  Checked
against the test-side expansion of the paper's examples and the printed
offsets and ground energies."""
import json
import os

import numpy as np
import pytest

import paper_models as PM
import polyexp
import workloads as W
from oracle import oracle as O
from paper_2407_19987_gb300.model import Model, Poly

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def _as_instance(c, name=""):
    return W.Instance(c.N, c.order, c.idx, c.coef, c.offset, True, name)


@pytest.mark.parametrize("front,ref,gold", [(PM.seating, polyexp.seating, "seating5x5"),
                                            (PM.pythagorean, polyexp.pythagorean, "pythagorean"),
                                            (PM.tsp, polyexp.tsp_intenc, "tsp_intenc")])
def test_examples_compile_to_the_same_objective(front, ref, gold):
    m, c = front()
    r = ref()
    assert c.N == r.N and c.offset == GOLD[gold]["offset"] == r.offset
    X = W.random_states(5, 3000, c.N) if c.N > 16 else np.array(
        [[(s >> i) & 1 for i in range(c.N)] for s in range(1 << c.N)], np.uint8)
    np.testing.assert_array_equal(O.energy(_as_instance(c), X), O.energy(r, X))
    assert np.all(np.diff(c.idx, axis=1) >= 0)


def test_small_examples_ground_energies_by_enumeration():
    for front, gold in ((PM.pythagorean, "pythagorean"), (PM.tsp, "tsp_intenc")):
        m, c = front()
        E = O.bruteforce(_as_instance(c))
        assert E.min() == GOLD[gold]["energy"]
        # every ground state decodes to a valid solution
        for s in np.nonzero(E == E.min())[0]:
            v = c.decode(np.array([(s >> i) & 1 for i in range(c.N)]))
            if gold == "pythagorean":
                assert v["x"] ** 2 + v["y"] ** 2 == v["z"] ** 2 and min(v["x"], v["y"], v["z"]) > 0
            else:
                assert v["xB"] * v["xC"] * v["xD"] == 6


def test_binary_algebra_and_encoding():
    m = Model()
    q = m.binary("q", (2, 3))
    a = m.binary("a")
    assert m.names == ["q0_0", "q0_1", "q0_2", "q1_0", "q1_1", "q1_2", "a"]
    assert q[0, 1] * q[0, 1] == q[0, 1]                      # x * x = x
    assert (q[0, 0] + a) ** 2 == q[0, 0] + a + 2 * q[0, 0] * a
    y = m.integer("y", 3, lower=1)
    c = m.compile((y - 4) ** 2 + a)
    assert c.order == 2 and c.offset == 9
    bits = np.zeros(c.N, np.int64)
    bits[c.integers["y"][0][0]] = 1
    bits[c.integers["y"][0][2]] = 1                          # y = 1 + 1 + 4
    assert c.decode(bits)["y"] == 6
    words = W.pack_bits(bits[None, :].astype(np.uint8))[0]
    assert c.decode(words)["y"] == 6
    assert m.compile(q[0, 0] * q[1, 2] * a).idx.tolist() == [[0, 5, 6]]
    assert sorted(m.compile(3 * q[1, 1] + q[0, 0] * a).idx.tolist()) == [[0, 6], [4, 4]]


def test_compile_refuses_inexact_coefficients():
    m = Model()
    x = m.binary("x")
    with pytest.raises(ValueError):
        m.compile((2 ** 25 + 1) * x)
    assert m.compile((2 ** 25 + 1) * x, exact=False).coef[0] == np.float32(2 ** 25)
    with pytest.raises(TypeError):
        x + "a"


def test_msb_first_encoding_dense_form_and_refusals():
    m = Model()
    y = m.integer("y", 3, msb_first=True)                    # y = 4 b0 + 2 b1 + b2
    x = m.binary("x")
    c = m.compile(y * x - 2 * y + 7)
    assert c.offset == 7 and c.order == 2
    ids, weights, lower = c.integers["y"]
    assert weights == [4, 2, 1] and lower == 0
    bits = np.zeros(c.N, np.int64)
    bits[ids[0]] = bits[ids[2]] = 1
    assert c.decode(bits)["y"] == 5
    # the dense upper-triangular tensor holds the same energy as the entries
    X = np.array([[(s >> i) & 1 for i in range(c.N)] for s in range(1 << c.N)], np.uint8)
    T = c.dense()
    dense_E = np.einsum("ij,bi,bj->b", T, X.astype(np.float64), X.astype(np.float64))
    np.testing.assert_array_equal(dense_E, O.energy(_as_instance(c), X))
    # objective value = energy + offset, checked against direct evaluation
    Xi = X.astype(np.int64)
    yv = 4 * Xi[:, ids[0]] + 2 * Xi[:, ids[1]] + Xi[:, ids[2]]
    np.testing.assert_array_equal(dense_E + c.offset, yv * Xi[:, c.groups["x"]] - 2 * yv + 7)
    assert x ** 0 == 1 and (x ** 3) == x
    with pytest.raises(ValueError):
        m.binary("x")                                          # name already declared
    other = Model()
    other.binary("u", (5,))
    w = other.binary("w")
    with pytest.raises(ValueError):
        m.compile(w)                                           # index beyond this model's variables
