"""Host front end: polynomials over binary variables compiled to HOBO
tensor entries.

A model declares named binary variables (arrays of them, named like
``q{}_{}``), builds an objective from them with +, -, * and integer powers
(binary variables satisfy x*x = x, Sec. II.B, so a product of monomials is
the union of their variable sets), encodes integers in binary (Sec. IV.B),
and compiles the objective to the tensor-entry form the library takes
(Sec. III.C): one entry per monomial of degree >= 1, the tensor order being
the highest degree, a lower-degree monomial stored with its smallest index
repeated in front; the constant term is returned apart as the offset.
``Compiled.instance()`` hands the entries to ``hobo_create_terms``;
``Compiled.decode()`` maps a state back to named arrays and integers.

Coefficients stay exact Python numbers during expansion; the library takes
float32, and ``compile(..., exact=True)`` refuses coefficients that float32
cannot hold exactly.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np


class Poly:
    """Polynomial over binary variables: {sorted tuple of distinct variable
    indices: coefficient}; the empty tuple holds the constant."""

    __slots__ = ("t",)

    def __init__(self, terms=None):
        self.t = {}
        for k, v in (terms or {}).items():
            if v != 0:
                self.t[k] = self.t.get(k, 0) + v

    @staticmethod
    def lift(o) -> "Poly":
        if isinstance(o, Poly):
            return o
        if isinstance(o, (int, float, np.integer, np.floating)):
            return Poly({(): o.item() if isinstance(o, np.generic) else o})
        raise TypeError(f"cannot use {type(o).__name__} in a polynomial")

    def __add__(self, o):
        o = Poly.lift(o)
        r = dict(self.t)
        for k, v in o.t.items():
            r[k] = r.get(k, 0) + v
        return Poly({k: v for k, v in r.items() if v != 0})

    __radd__ = __add__

    def __neg__(self):
        return Poly({k: -v for k, v in self.t.items()})

    def __sub__(self, o):
        return self + (-Poly.lift(o))

    def __rsub__(self, o):
        return Poly.lift(o) - self

    def __mul__(self, o):
        o = Poly.lift(o)
        r = {}
        for ka, va in self.t.items():
            for kb, vb in o.t.items():
                k = tuple(sorted(set(ka).union(kb)))       # x * x = x
                r[k] = r.get(k, 0) + va * vb
        return Poly({k: v for k, v in r.items() if v != 0})

    __rmul__ = __mul__

    def __pow__(self, n: int):
        if not isinstance(n, (int, np.integer)) or n < 0:
            raise ValueError("power must be a non-negative integer")
        r, base, n = Poly({(): 1}), self, int(n)
        while n:
            if n & 1:
                r = r * base
            base = base * base
            n >>= 1
        return r

    def __eq__(self, o):
        return isinstance(o, (Poly, int, float)) and self.t == Poly.lift(o).t

    def __hash__(self):
        return hash(frozenset(self.t.items()))

    @property
    def degree(self) -> int:
        return max((len(k) for k in self.t), default=0)

    @property
    def constant(self):
        return self.t.get((), 0)

    def terms(self):
        return dict(self.t)

    def __repr__(self):
        return f"Poly({len(self.t)} terms, degree {self.degree})"


@dataclass
class Compiled:
    """Tensor-entry form of an objective: idx int32 [nnz, order] (rows
    non-decreasing, smallest index repeated for lower degrees), coef float32
    [nnz], offset = constant term; energy + offset = objective."""
    N: int
    order: int
    idx: np.ndarray
    coef: np.ndarray
    offset: float
    names: list
    groups: dict = field(default_factory=dict)
    integers: dict = field(default_factory=dict)

    def instance(self, flags: int = 0):
        from .binding import Instance
        return Instance.from_terms(self.idx, self.coef, self.N, flags)

    def dense(self) -> np.ndarray:
        """The upper-triangular tensor (N,)*order with each entry at its
        stored index tuple (small N only)."""
        T = np.zeros((self.N,) * self.order, dtype=np.float64)
        np.add.at(T, tuple(self.idx[:, d] for d in range(self.order)), self.coef.astype(np.float64))
        return T

    def decode(self, bits) -> dict:
        """Named values of a state (0/1 array [N] or packed uint32/int32
        words): every declared array as an int array, every integer as an int."""
        b = np.asarray(bits)
        if b.size != self.N:                                  # packed words
            words = b.astype(np.int64).reshape(-1) & 0xFFFFFFFF
            b = np.array([(int(words[i >> 5]) >> (i & 31)) & 1 for i in range(self.N)], dtype=np.int64)
        b = b.reshape(-1).astype(np.int64)
        out = {}
        for name, ids in self.groups.items():
            out[name] = b[np.asarray(ids)]
        for name, (ids, weights, lower) in self.integers.items():
            out[name] = int(lower + sum(w * int(b[i]) for i, w in zip(ids, weights)))
        return out


class Model:
    """Declares binary variables and compiles objectives over them."""

    def __init__(self):
        self.names: list = []
        self.groups: dict = {}
        self.integers: dict = {}

    def _new(self, name: str) -> Poly:
        i = len(self.names)
        self.names.append(name)
        return Poly({(i,): 1})

    def binary(self, name: str, shape=()):
        """A binary variable (shape ()) or an array of them named by
        position, e.g. binary('q', (3, 4)) -> q0_0 .. q2_3."""
        shape = tuple(shape) if isinstance(shape, (tuple, list)) else (int(shape),)
        if name in self.groups or name in self.integers:
            raise ValueError(f"{name} already declared")
        if not shape:
            v = self._new(name)
            self.groups[name] = np.array(len(self.names) - 1)
            return v
        arr = np.empty(shape, dtype=object)
        ids = np.empty(shape, dtype=np.int64)
        for pos in itertools.product(*(range(s) for s in shape)):
            arr[pos] = self._new(name + "_".join(str(p) for p in pos))
            ids[pos] = len(self.names) - 1
        self.groups[name] = ids
        return arr

    def integer(self, name: str, bits: int, msb_first: bool = False, lower: int = 0) -> Poly:
        """An integer lower + sum_k w_k x_k over `bits` new binary variables
        (Sec. IV.B): w_k = 2^k, least significant bit first, or 2^(bits-1-k)
        with msb_first."""
        if bits < 1:
            raise ValueError("bits must be >= 1")
        xs = self.binary(name, (bits,))
        ids = self.groups.pop(name).reshape(-1).tolist()
        weights = [2 ** (bits - 1 - k) if msb_first else 2 ** k for k in range(bits)]
        self.integers[name] = (ids, weights, lower)
        y = Poly({(): lower})
        for w, x in zip(weights, xs):
            y = y + w * x
        return y

    def bits(self, name: str) -> list:
        """The binary variables of a declared integer, in encoding order."""
        return [Poly({(i,): 1}) for i in self.integers[name][0]]

    def compile(self, H, exact: bool = True) -> Compiled:
        H = Poly.lift(H)
        mons = [(k, v) for k, v in H.t.items() if k]
        order = max((len(k) for k, _ in mons), default=1)
        idx = np.zeros((len(mons), order), dtype=np.int32)
        coef = np.zeros(len(mons), dtype=np.float32)
        for r, (k, v) in enumerate(mons):
            idx[r] = [k[0]] * (order - len(k)) + list(k)         # Sec. III.C storage
            coef[r] = np.float32(v)
            if exact and float(coef[r]) != v:
                raise ValueError(f"coefficient {v} of {k} is not exactly a float32")
        N = len(self.names)
        if mons and int(idx.max()) >= N:
            raise ValueError("objective uses a variable of another model")
        return Compiled(N, order, idx, coef, float(H.constant), list(self.names),
                        {k: np.asarray(v) for k, v in self.groups.items()}, dict(self.integers))
