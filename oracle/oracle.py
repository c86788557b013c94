"""The CPU oracle: a ctypes wrapper of hobo_oracle.c plus the result table
and tensor-train routines in numpy.

Test infrastructure only: the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this module; the product path never
does.  The energy, field, random-number, annealing and network routines are
thin marshalling over the C code, which states their arithmetic and
sources.  Written here in numpy, each citing its passage:
  aggregate            the result table of a run (Sec. V: states by energy
                       with occurrence counts); pinned by a hand example and
                       by direct scans on random pools.
  tt_svd, tt_full,     tensor-train decomposition and contraction (Sec. VI);
  tt_energy            pinned by the TSP tensor's printed bond dimensions,
                       the printed einsum path cost, rank-1 closed forms and
                       brute force against the full tensor.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hobo_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fno-strict-aliasing",
           "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        i64, i32, u64, dbl, flt = C.c_int64, C.c_int, C.c_uint64, C.c_double, C.c_float
        _lib.orc_energy.restype = dbl
        _lib.orc_energy.argtypes = [P, P, i64, i32, P]
        _lib.orc_energy_batch.argtypes = [P, P, i64, i32, i32, P, i64, P]
        _lib.orc_energy_batch_i64.argtypes = [P, P, i64, i32, i32, P, i64, P]
        _lib.orc_bruteforce.argtypes = [P, P, i64, i32, i32, P]
        _lib.orc_flip_delta.argtypes = [P, P, i64, i32, i32, P, P]
        _lib.orc_fields.argtypes = [P, P, i64, i32, i32, P, P]
        _lib.orc_philox4x32_10.argtypes = [P, P, P]
        _lib.orc_exp2.restype = flt
        _lib.orc_exp2.argtypes = [flt]
        _lib.orc_metropolis.restype = i32
        _lib.orc_metropolis.argtypes = [flt, flt, C.c_uint32]
        _lib.orc_init_states.argtypes = [u64, i32, i64, P]
        _lib.orc_anneal.argtypes = [P, P, i64, i32, i32, u64, i64, i64, P, i32,
                                    P, P, P, P, P, i64, P]
        _lib.orc_anneal_naive.argtypes = [P, P, i64, i32, i32, u64, i64, i64, P, i32,
                                          P, P, P, P, P]
        _lib.orc_anneal_learned.argtypes = [P, P, i64, i32, i32, u64, i64, P, i32,
                                            i32, P, P, P, P, P, dbl, i32, i32, flt, dbl, flt,
                                            P, P, P, P, P, i32, i64, P, P]
        _lib.orc_mlp_forward.argtypes = [i32, P, P, P, P, P, dbl, P, i64, P]
        _lib.orc_mlp_loss_grad.restype = dbl
        _lib.orc_mlp_loss_grad.argtypes = [i32, P, P, P, P, P, dbl, P, P, i64, P, P, P, P, P, P]
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _terms(inst):
    idx = np.ascontiguousarray(inst.idx, dtype=np.int32)
    coef = np.ascontiguousarray(inst.coef, dtype=np.float64)
    return idx, coef


def energy(inst, X: np.ndarray) -> np.ndarray:
    """Energies (float64) of the 0/1 states in rows of X (uint8 [B, N])."""
    idx, coef = _terms(inst)
    X = np.ascontiguousarray(X, dtype=np.uint8)
    E = np.zeros(X.shape[0], dtype=np.float64)
    lib().orc_energy_batch(_p(idx), _p(coef), idx.shape[0], inst.order, inst.N, _p(X), X.shape[0], _p(E))
    return E


def energy_int(inst, X: np.ndarray) -> np.ndarray:
    """Exact int64 energies for integer-coefficient instances."""
    idx, coef = _terms(inst)
    ci = np.ascontiguousarray(np.rint(coef).astype(np.int64))
    if not np.array_equal(ci.astype(np.float64), coef):
        raise ValueError("instance has non-integer coefficients")
    X = np.ascontiguousarray(X, dtype=np.uint8)
    E = np.zeros(X.shape[0], dtype=np.int64)
    lib().orc_energy_batch_i64(_p(idx), _p(ci), idx.shape[0], inst.order, inst.N, _p(X), X.shape[0], _p(E))
    return E


def bruteforce(inst) -> np.ndarray:
    """Energy of every state s in [0, 2^N), x_i = bit i of s."""
    if inst.N > 30:
        raise ValueError("N too large for enumeration")
    idx, coef = _terms(inst)
    E = np.zeros(1 << inst.N, dtype=np.float64)
    lib().orc_bruteforce(_p(idx), _p(coef), idx.shape[0], inst.order, inst.N, _p(E))
    return E


def flip_delta(inst, x: np.ndarray) -> np.ndarray:
    idx, coef = _terms(inst)
    x = np.ascontiguousarray(x, dtype=np.uint8)
    d = np.zeros(inst.N, dtype=np.float64)
    lib().orc_flip_delta(_p(idx), _p(coef), idx.shape[0], inst.order, inst.N, _p(x), _p(d))
    return d


def fields(inst, x: np.ndarray) -> np.ndarray:
    idx, coef = _terms(inst)
    x = np.ascontiguousarray(x, dtype=np.uint8)
    g = np.zeros(inst.N, dtype=np.float64)
    lib().orc_fields(_p(idx), _p(coef), idx.shape[0], inst.order, inst.N, _p(x), _p(g))
    return g


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.array(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.array(key, dtype=np.uint32))
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def exp2(t: float) -> np.float32:
    return np.float32(lib().orc_exp2(float(np.float32(t))))


def metropolis(dE: float, beta: float, w: int) -> bool:
    return bool(lib().orc_metropolis(float(np.float32(dE)), float(np.float32(beta)), int(w) & 0xFFFFFFFF))


def init_states(seed: int, N: int, B: int) -> np.ndarray:
    X = np.zeros((B, N), dtype=np.uint8)
    lib().orc_init_states(seed, N, B, _p(X))
    return X


def anneal(inst, seed: int, B: int, betas: np.ndarray, state0: int = 0, rec_B: int = 0,
           naive: bool = False) -> dict:
    """Run the oracle annealer on states state0 .. state0+B-1."""
    idx, coef = _terms(inst)
    betas = np.ascontiguousarray(betas, dtype=np.float32)
    S = betas.shape[0]
    N = inst.N
    Xf = np.zeros((B, N), np.uint8)
    Xb = np.zeros((B, N), np.uint8)
    Ef = np.zeros(B, np.float64)
    Eb = np.zeros(B, np.float64)
    acc = np.zeros(B, np.int64)
    if naive:
        lib().orc_anneal_naive(_p(idx), _p(coef), idx.shape[0], inst.order, N, seed, state0, B,
                               _p(betas), S, _p(Xf), _p(Ef), _p(Xb), _p(Eb), _p(acc))
        return dict(X=Xf, E=Ef, bestX=Xb, bestE=Eb, accepts=acc)
    rec = np.zeros((S, rec_B, N), np.uint8) if rec_B > 0 else None
    lib().orc_anneal(_p(idx), _p(coef), idx.shape[0], inst.order, N, seed, state0, B,
                     _p(betas), S, _p(Xf), _p(Ef), _p(Xb), _p(Eb), _p(acc), rec_B,
                     _p(rec) if rec is not None else None)
    return dict(X=Xf, E=Ef, bestX=Xb, bestE=Eb, accepts=acc, rec=rec)


def _mlp_args(w):
    H = w["b1"].shape[0]
    arrs = [np.ascontiguousarray(w[k], dtype=np.float64) for k in ("W1", "b1", "W2", "b2", "w3")]
    return H, arrs, float(np.asarray(w["b3"]).reshape(-1)[0])


def mlp_forward(w: dict, F: np.ndarray) -> np.ndarray:
    """Logits of the MLP (weights dict W1 [H,3], b1, W2 [H,H], b2, w3, b3) on rows F [n,3]."""
    H, (W1, b1, W2, b2, w3), b3 = _mlp_args(w)
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(F.shape[0], np.float64)
    lib().orc_mlp_forward(H, _p(W1), _p(b1), _p(W2), _p(b2), _p(w3), b3, _p(F), F.shape[0], _p(out))
    return out


def mlp_loss_grad(w: dict, F: np.ndarray, y: np.ndarray):
    """Mean binary cross-entropy and its gradients (dict like w)."""
    H, (W1, b1, W2, b2, w3), b3 = _mlp_args(w)
    F = np.ascontiguousarray(F, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    g = {"W1": np.zeros((H, 3)), "b1": np.zeros(H), "W2": np.zeros((H, H)), "b2": np.zeros(H),
         "w3": np.zeros(H)}
    gb3 = np.zeros(1)
    loss = lib().orc_mlp_loss_grad(H, _p(W1), _p(b1), _p(W2), _p(b2), _p(w3), b3, _p(F), _p(y), F.shape[0],
                                   _p(g["W1"]), _p(g["b1"]), _p(g["W2"]), _p(g["b2"]), _p(g["w3"]), _p(gb3))
    g["b3"] = gb3
    return loss, g


def anneal_learned(inst, seed: int, B: int, betas: np.ndarray, w: dict | None, plain_every: int = 4,
                   top_frac: float = 1.0, vmax: float = 32.0, rec_every: int = 0, rec_B: int = 0,
                   select: int = 0, threshold: float = 0.0) -> dict:
    """Oracle annealer with the learned proposal (network weights ``w`` as
    in mlp_forward, or None for plain sweeps only).  With recording, returns
    rec_F [rows, 3], rec_x (0xFF where a bit was not attempted) and the
    labels rec_y: 1 if the recorded bit differs from the state's final best
    bit, 0 if not, -1 if not attempted."""
    idx, coef = _terms(inst)
    betas = np.ascontiguousarray(betas, dtype=np.float32)
    S = betas.shape[0]
    N = inst.N
    Xf = np.zeros((B, N), np.uint8)
    Xb = np.zeros((B, N), np.uint8)
    Ef = np.zeros(B, np.float64)
    Eb = np.zeros(B, np.float64)
    acc = np.zeros(B, np.int64)
    if w is not None:
        H, (W1, b1, W2, b2, w3), b3 = _mlp_args(w)
        wp = [_p(a) for a in (W1, b1, W2, b2, w3)]
    else:
        H, wp, b3 = 0, [None] * 5, 0.0
    rec = rec_every > 0 and rec_B > 0
    rB = min(rec_B, B) if rec else 0
    nrows = ((S + rec_every - 1) // rec_every) * rB * N if rec else 0
    recF = np.zeros((max(nrows, 1), 3), np.float32)
    recx = np.full(max(nrows, 1), 0xFF, np.uint8)
    lib().orc_anneal_learned(_p(idx), _p(coef), idx.shape[0], inst.order, N, seed, B, _p(betas), S,
                             H, *wp, b3, plain_every, int(select), float(top_frac), float(threshold), float(vmax),
                             _p(Xf), _p(Ef), _p(Xb), _p(Eb), _p(acc),
                             max(rec_every, 1), rB, _p(recF) if rec else None, _p(recx) if rec else None)
    out = dict(X=Xf, E=Ef, bestX=Xb, bestE=Eb, accepts=acc)
    if rec:
        recF, recx = recF[:nrows], recx[:nrows]
        b_of_row = (np.arange(nrows) // N) % rB
        best = Xb[b_of_row, np.arange(nrows) % N]
        y = np.where(recx == 0xFF, -1.0, (recx != best).astype(np.float64)).astype(np.float32)
        out.update(rec_F=recF, rec_x=recx, rec_y=y)
    return out


def aggregate(X: np.ndarray, E: np.ndarray):
    """Result table of a run: the distinct rows of X (uint8 [B, N]) with
    their energy (that of the first occurrence), occurrence count and first
    index, sorted by energy then first index.  Returns (states [K, N],
    energy [K], count [K], first [K])."""
    X = np.ascontiguousarray(X, dtype=np.uint8)
    E = np.asarray(E, dtype=np.float64)
    seen = {}
    for b in range(X.shape[0]):
        key = X[b].tobytes()
        if key in seen:
            seen[key][1] += 1
        else:
            seen[key] = [b, 1]
    rows = sorted(seen.values(), key=lambda t: (E[t[0]], t[0]))
    first = np.array([r[0] for r in rows], dtype=np.int64)
    count = np.array([r[1] for r in rows], dtype=np.int64)
    return X[first], E[first], count, first


def tt_svd(T: np.ndarray, rel_tol: float = 1e-10) -> list:
    """Tensor-train decomposition by successive SVDs (Sec. VI): reshape the
    remainder to (r_{c-1} n_c) x rest, SVD it, keep the singular values above
    rel_tol times the largest as core c, carry Sigma V* on.  Cores
    G_c [r_{c-1}, n_c, r_c], r_0 = r_d = 1."""
    T = np.asarray(T, dtype=np.float64)
    d, n = T.ndim, T.shape
    cores, r, C = [], 1, T.reshape(1, -1)
    for c in range(d - 1):
        C = C.reshape(r * n[c], -1)
        U, s, Vt = np.linalg.svd(C, full_matrices=False)
        rk = max(1, int((s > rel_tol * s[0]).sum())) if s.size and s[0] > 0 else 1
        cores.append(U[:, :rk].reshape(r, n[c], rk))
        C = s[:rk, None] * Vt[:rk]
        r = rk
    cores.append(C.reshape(r, n[d - 1], 1))
    return cores


def tt_full(cores) -> np.ndarray:
    """The tensor a train represents: A[i1..id] = G1[:, i1, :] ... Gd[:, id, :]."""
    A = cores[0]
    for G in cores[1:]:
        A = np.tensordot(A, G, axes=([A.ndim - 1], [0]))
    return A.reshape(A.shape[1:-1])


def tt_energy(cores, X: np.ndarray) -> np.ndarray:
    """E(x) = sum over all index tuples of A[i1..id] x_i1 ... x_id for each
    row x of X, by contracting every core with x: the product of the
    matrices M_c = sum_i x_i G_c[:, i, :], in float64."""
    X = np.asarray(X, dtype=np.float64)
    out = np.zeros(X.shape[0])
    for b in range(X.shape[0]):
        v = np.ones((1,))
        for G in cores:
            v = v @ np.einsum("i,aib->ab", X[b], np.asarray(G, dtype=np.float64))
        out[b] = v[0]
    return out
