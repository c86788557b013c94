"""Tiny polynomial expander over binary symbols (test helper only).

Used to build the paper's three worked examples (Sec. V) as HOBO tensors.
A polynomial is a dict mapping a sorted tuple of distinct symbol indices to
an integer coefficient; multiplying two monomials takes the union of their
index sets, which is x*x = x for binary variables (Sec. II.B).  The empty
tuple carries the constant, which the tensor form returns separately as the
offset (Sec. V listings print it).
"""
from __future__ import annotations

import numpy as np

from workloads import Instance, pad_smallest


class P:
    def __init__(self, terms=None):
        self.t = {}
        for k, v in (terms or {}).items():
            if v != 0:
                self.t[k] = self.t.get(k, 0) + v

    @staticmethod
    def var(i: int) -> "P":
        return P({(i,): 1})

    @staticmethod
    def const(c) -> "P":
        return P({(): c})

    def _lift(self, o):
        return o if isinstance(o, P) else P.const(o)

    def __add__(self, o):
        o = self._lift(o)
        r = dict(self.t)
        for k, v in o.t.items():
            r[k] = r.get(k, 0) + v
        return P({k: v for k, v in r.items() if v != 0})

    __radd__ = __add__

    def __neg__(self):
        return P({k: -v for k, v in self.t.items()})

    def __sub__(self, o):
        return self + (-self._lift(o))

    def __rsub__(self, o):
        return self._lift(o) - self

    def __mul__(self, o):
        o = self._lift(o)
        r = {}
        for ka, va in self.t.items():
            for kb, vb in o.t.items():
                k = tuple(sorted(set(ka) | set(kb)))
                r[k] = r.get(k, 0) + va * vb
        return P({k: v for k, v in r.items() if v != 0})

    __rmul__ = __mul__

    def __pow__(self, n: int):
        r = P.const(1)
        for _ in range(n):
            r = r * self
        return r

    def to_instance(self, N: int, name: str = "") -> Instance:
        """Tensor-entry form: order = highest degree, lower-degree monomials
        padded by repeating the smallest index (Sec. III.C)."""
        mons = [(k, v) for k, v in self.t.items() if k]
        order = max(len(k) for k, _ in mons)
        idx = np.array([pad_smallest(k, order) for k, _ in mons], dtype=np.int32)
        coef = np.array([v for _, v in mons], dtype=np.float32)
        return Instance(N, order, idx, coef, float(self.t.get((), 0)), True, name)


def seating():
    """Sec. V.A: 5x5 seats, reward each occupied seat, penalty 10 for three
    consecutive occupied seats in a row or a column."""
    q = [[P.var(5 * i + j) for j in range(5)] for i in range(5)]
    H1 = P()
    for i in range(5):
        for j in range(5):
            H1 = H1 - q[i][j]
    H2 = P()
    for i in range(5):
        for j in range(3):
            H2 = H2 + q[i][j] * q[i][j + 1] * q[i][j + 2]
    for j in range(5):
        for i in range(3):
            H2 = H2 + q[i][j] * q[i + 1][j] * q[i + 2][j]
    return (H1 + 10 * H2).to_instance(25, "seating5x5")


def pythagorean():
    """Sec. V.B: three 4-bit integers (least significant bit first),
    (x^2 + y^2 - z^2)^2 plus 10 for each integer that is zero."""
    q = [[P.var(4 * a + b) for b in range(4)] for a in range(3)]
    x = sum((2 ** b) * q[0][b] for b in range(4))
    y = sum((2 ** b) * q[1][b] for b in range(4))
    z = sum((2 ** b) * q[2][b] for b in range(4))
    H1 = (x * x + y * y - z * z) ** 2
    H2 = P()
    for a in range(3):
        prod = P.const(1)
        for b in range(4):
            prod = prod * (1 - q[a][b])
        H2 = H2 + prod
    return (H1 + 10 * H2).to_instance(12, "pythagorean")


def tsp_intenc():
    """Sec. V.C: three 2-bit integers (most significant bit first),
    10*(xB*xC*xD - 6)^2.  The fourth symbol row q3_* is unused; the tensor
    covers the six bits of rows 0..2."""
    q = [[P.var(2 * a + b) for b in range(2)] for a in range(3)]
    xB = 2 * q[0][0] + q[0][1]
    xC = 2 * q[1][0] + q[1][1]
    xD = 2 * q[2][0] + q[2][1]
    return (10 * (xB * xC * xD - 6) ** 2).to_instance(6, "tsp_intenc")
