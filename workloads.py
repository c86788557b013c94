"""Seeded synthetic HOBO instances and annealing schedules.

This module only draws random numbers and lays out inputs; it holds none of
the solver's arithmetic (no folding of repeated indices, no energies, no
fields).  Both the CPU oracle and the CUDA path consume exactly what it
returns, so the two sides see identical inputs.

An instance is a list of index tuples of a fixed length ``order`` with one
coefficient each.  A monomial of lower degree is stored the way Sec. III.C /
Sec. IV.A of the paper store it: the smallest index is repeated in front
until the tuple reaches the tensor's order (c_ijk -> c_iiijk).  Tuples are
sorted ascending, i.e. they address the upper (non-decreasing) part of the
order-k HOBO tensor of Sec. II.C.

Workloads (shapes follow the paper's examples and the benchmark table):
  tiny_dense      order 3, N=12, every i<=j<=k entry, integers U{-10..10}
  dense_float     order 3, N=256, every i<=j<=k entry, N(0,1) float32
  int_encoded     32 four-bit integers (N=128), 200 random cubic monomials
                  y_i y_j y_k with weights U{-3..3} plus 4*(sum y - 240)^2,
                  expanded over the binary encoding of Sec. IV.B
  uneven_batch    512 order-3 instances, N~U[16,192], 5% term density
  sparse_order4   order 4, N=96, 2% term density, integers in [-8,8]\\{0}
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Instance:
    """One HOBO instance in tensor-entry form.

    idx:    int32 [nnz, order], each row non-decreasing, values in [0, N)
    coef:   float32 [nnz], the tensor entry at that index tuple
    offset: constant term of the objective (not part of the tensor)
    integer: True if every coefficient is an integer
    """
    N: int
    order: int
    idx: np.ndarray
    coef: np.ndarray
    offset: float = 0.0
    integer: bool = False
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.idx.shape[0])

    def dense(self) -> np.ndarray:
        """Dense float32 tensor of shape (N,)*order with the entries placed at
        their index tuples (entries sharing a tuple are added)."""
        T = np.zeros((self.N,) * self.order, dtype=np.float64)
        np.add.at(T, tuple(self.idx[:, d] for d in range(self.order)), self.coef.astype(np.float64))
        return T.astype(np.float32)


def pad_smallest(tup, order: int) -> tuple:
    """Sort a monomial's indices and repeat the smallest one in front until
    the tuple has ``order`` entries (Sec. III.C storage rule)."""
    s = sorted(tup)
    if len(s) > order:
        raise ValueError("monomial degree exceeds tensor order")
    return tuple([s[0]] * (order - len(s)) + s)


def _all_nondecreasing(N: int, order: int) -> np.ndarray:
    """All index tuples i1<=i2<=...<=ik over range(N), lexicographic."""
    if order == 1:
        return np.arange(N, dtype=np.int32)[:, None]
    rows = []
    prev = _all_nondecreasing(N, order - 1)
    for i in range(N):
        tail = prev[prev[:, 0] >= i]
        rows.append(np.concatenate([np.full((tail.shape[0], 1), i, np.int32), tail], axis=1))
    return np.concatenate(rows, axis=0).astype(np.int32)


def tiny_dense(seed: int = 1, N: int = 12, order: int = 3) -> Instance:
    """Order-3, N=12, all non-decreasing entries, integer coefficients
    uniform in [-10, 10]."""
    rng = np.random.default_rng(seed)
    idx = _all_nondecreasing(N, order)
    coef = rng.integers(-10, 11, size=idx.shape[0]).astype(np.float32)
    return Instance(N, order, idx, coef, 0.0, True, f"tiny_dense_N{N}_k{order}_s{seed}")


def dense_float(seed: int = 2, N: int = 256, order: int = 3) -> Instance:
    """Order-3 dense instance, all non-decreasing entries ~ N(0,1) float32."""
    rng = np.random.default_rng(seed)
    idx = _all_nondecreasing(N, order)
    coef = rng.standard_normal(idx.shape[0], dtype=np.float32)
    return Instance(N, order, idx, coef, 0.0, False, f"dense_float_N{N}_k{order}_s{seed}")


def int_encoded(seed: int = 3, n_ints: int = 32, bits: int = 4, n_cubic: int = 200,
                wmax: int = 3, target: int = 240, penalty: int = 4) -> Instance:
    """Binary-encoded integers y_i = sum_b 2^b x_{bits*i+b} (Sec. IV.B,
    least significant bit first).  Objective:
        sum_{t<n_cubic} w_t y_{a_t} y_{b_t} y_{c_t} + penalty*(sum_i y_i - target)^2
    with a,b,c drawn with replacement and w_t ~ U{-wmax..wmax}.  Each product
    of encodings is multiplied out term by term into bit tuples; repeated
    bits are left as repeats (x*x is not reduced here).  The constant
    penalty*target^2 becomes the offset."""
    rng = np.random.default_rng(seed)
    N = n_ints * bits
    order = 3
    pw = [1 << b for b in range(bits)]
    tuples, coefs = [], []
    trip = rng.integers(0, n_ints, size=(n_cubic, 3))
    w = rng.integers(-wmax, wmax + 1, size=n_cubic)
    for t in range(n_cubic):
        if w[t] == 0:
            continue
        a, b, c = (int(v) for v in trip[t])
        for ba in range(bits):
            for bb in range(bits):
                for bc in range(bits):
                    tuples.append(pad_smallest((bits * a + ba, bits * b + bb, bits * c + bc), order))
                    coefs.append(float(w[t]) * pw[ba] * pw[bb] * pw[bc])
    # penalty*(S - target)^2 = penalty*S^2 - 2*penalty*target*S + penalty*target^2
    wbit = np.array([pw[p % bits] for p in range(N)], dtype=np.int64)
    for p in range(N):
        for q in range(N):
            tuples.append(pad_smallest((p, q), order))
            coefs.append(float(penalty * wbit[p] * wbit[q]))
    for p in range(N):
        tuples.append(pad_smallest((p,), order))
        coefs.append(float(-2 * penalty * target * wbit[p]))
    idx = np.array(tuples, dtype=np.int32)
    coef = np.array(coefs, dtype=np.float32)
    inst = Instance(N, order, idx, coef, float(penalty * target * target), True,
                    f"int_encoded_{n_ints}x{bits}_s{seed}")
    inst.meta.update(dict(n_ints=n_ints, bits=bits, trip=trip, w=w, target=target, penalty=penalty))
    return inst


def _sample_subsets(rng, N: int, d: int, count: int) -> np.ndarray:
    """``count`` distinct d-subsets of range(N), uniformly, as sorted rows."""
    if count == 0:
        return np.zeros((0, d), np.int32)
    have = np.zeros((0, d), np.int64)
    while have.shape[0] < count:
        need = count - have.shape[0]
        draw = np.sort(rng.integers(0, N, size=(2 * need + 64, d)), axis=1)
        ok = np.all(np.diff(draw, axis=1) > 0, axis=1) if d > 1 else np.ones(draw.shape[0], bool)
        draw = draw[ok]
        # keep first occurrences, in draw order, of subsets not seen before
        allrows = np.concatenate([have, draw], axis=0)
        key = np.zeros(allrows.shape[0], np.int64)
        for c in range(d):
            key = key * N + allrows[:, c]
        _, first = np.unique(key, return_index=True)
        first.sort()
        have = allrows[first][:count]
    return have.astype(np.int32)


def random_sparse(seed: int, N: int, order: int, density: float, coef: str = "normal",
                  imax: int = 8) -> Instance:
    """Random instance with every linear term present and every monomial of
    degree 2..order over distinct variables present independently with
    probability ``density``.  coef='normal': N(0,1) float32;
    coef='int': uniform in [-imax, imax] without 0."""
    rng = np.random.default_rng(seed)
    rows = [np.arange(N, dtype=np.int32)[:, None]]
    for d in range(2, order + 1):
        total = math.comb(N, d)
        cnt = int(rng.binomial(total, density))
        rows.append(_sample_subsets(rng, N, d, cnt))
    # pad each monomial with its smallest index in front (Sec. III.C)
    padded = [np.concatenate([np.repeat(r[:, :1], order - r.shape[1], axis=1), r], axis=1)
              for r in rows if r.shape[0] > 0]
    idx = np.concatenate(padded, axis=0).astype(np.int32).reshape(-1, order)
    if coef == "normal":
        c = rng.standard_normal(idx.shape[0], dtype=np.float32)
        integer = False
    else:
        mag = rng.integers(1, imax + 1, size=idx.shape[0])
        sgn = rng.integers(0, 2, size=idx.shape[0]) * 2 - 1
        c = (mag * sgn).astype(np.float32)
        integer = True
    return Instance(N, order, idx, c, 0.0, integer, f"sparse_N{N}_k{order}_p{density}_s{seed}")


def dense_all_degrees(seed: int, N: int, order: int, coef: str = "normal", imax: int = 3,
                      top_only: bool = False) -> Instance:
    """Every monomial over distinct variables of degree 1..order (or of
    degree `order` only) with a coefficient: N(0,1) float32 or uniform in
    [-imax, imax] without 0.  Lower degrees padded with the smallest index."""
    import itertools
    rng = np.random.default_rng(seed)
    rows = []
    for d in ([order] if top_only else range(1, order + 1)):
        comb = np.array(list(itertools.combinations(range(N), d)), dtype=np.int32).reshape(-1, d)
        rows.append(np.concatenate([np.repeat(comb[:, :1], order - d, axis=1), comb], axis=1))
    idx = np.concatenate(rows, axis=0)
    if coef == "normal":
        c = rng.standard_normal(idx.shape[0], dtype=np.float32)
    else:
        c = (rng.integers(1, imax + 1, size=idx.shape[0]) * (rng.integers(0, 2, size=idx.shape[0]) * 2 - 1)).astype(np.float32)
    return Instance(N, order, idx, c, 0.0, coef != "normal", f"dense{order}_N{N}_s{seed}")


def uneven_batch(seed: int = 4000, count: int = 512, nmin: int = 16, nmax: int = 192,
                 density: float = 0.05) -> list:
    """``count`` order-3 instances with N ~ U[nmin, nmax] and N(0,1)
    coefficients; instance t uses seed ``seed + t``."""
    out = []
    for t in range(count):
        rng = np.random.default_rng(seed + t)
        n = int(rng.integers(nmin, nmax + 1))
        out.append(random_sparse(seed + t, n, 3, density, "normal"))
    return out


def sparse_order4(seed: int = 5000, N: int = 96, density: float = 0.02) -> Instance:
    """Order-4, N=96, 2% term density, integer coefficients in [-8,8]\\{0}."""
    return random_sparse(seed, N, 4, density, "int", 8)


def geometric_betas(T0: float, T1: float, sweeps: int) -> np.ndarray:
    """Inverse temperatures of a geometric schedule T_s = T0*(T1/T0)^(s/(S-1)),
    evaluated in float64 and rounded once to float32."""
    if sweeps == 1:
        T = np.array([T0], dtype=np.float64)
    else:
        s = np.arange(sweeps, dtype=np.float64)
        T = T0 * (T1 / T0) ** (s / (sweeps - 1))
    return (1.0 / T).astype(np.float32)


def random_states(seed: int, B: int, N: int) -> np.ndarray:
    """B random binary states, uint8 [B, N]."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2, size=(B, N), dtype=np.uint8)


def pack_bits(X: np.ndarray) -> np.ndarray:
    """uint8 [B, N] 0/1 -> uint32 [B, ceil(N/32)], bit i of a state in word
    i//32 at position i%32."""
    B, N = X.shape
    W = (N + 31) // 32
    Xp = np.zeros((B, W * 32), dtype=np.uint64)
    Xp[:, :N] = X
    Xp = Xp.reshape(B, W, 32)
    sh = np.arange(32, dtype=np.uint64)
    return (Xp << sh).sum(axis=2).astype(np.uint32)


def unpack_bits(P: np.ndarray, N: int) -> np.ndarray:
    """Inverse of pack_bits."""
    B, W = P.shape
    sh = np.arange(32, dtype=np.uint32)
    bits = ((P[:, :, None] >> sh) & 1).astype(np.uint8).reshape(B, W * 32)
    return bits[:, :N]


# Schedules used for each workload: (T0, T1, sweeps, B).
SCHEDULES = {
    "tiny_dense": (5.0, 0.05, 100, 256),
    "dense_float": (10.0, 0.01, 1000, 4096),
    "int_encoded": (2000.0, 0.5, 2000, 8192),
    "uneven_batch": (5.0, 0.02, 500, 1024),
    "sparse_order4": (8.0, 0.05, 500, 4096),
}
