"""Helpers shared by the GPU parity tests: moving seeded inputs to the
device, reading results back, and the float tolerance of the parity bar."""
from __future__ import annotations

import numpy as np

import workloads as W

FLOAT_RTOL = 1e-5   # relative error bar of the float instances


def torch():
    import torch as T
    return T


def make(inst, flags: int = 0):
    import paper_2407_19987_gb300 as H
    return H.Instance.from_terms(inst.idx, inst.coef, inst.N, flags)


def to_dev(X_u8: np.ndarray):
    T = torch()
    packed = W.pack_bits(np.ascontiguousarray(X_u8, dtype=np.uint8)).view(np.int32)
    return T.from_numpy(np.ascontiguousarray(packed)).cuda()


def to_host_bits(Xt, N: int) -> np.ndarray:
    P = np.ascontiguousarray(Xt.cpu().numpy()).view(np.uint32)
    return W.unpack_bits(P, N)


def abs_instance(inst):
    return W.Instance(inst.N, inst.order, inst.idx, np.abs(inst.coef), inst.offset, inst.integer)


# Values whose cancellation condition number scale/|ref| exceeds 64 are held
# to the absolute bound 1e-5 * scale / 64 (about 2.6 float32 ulps of the sum
# of magnitudes): no float32 summation of float32 terms can promise a
# relative error on a result that cancels more deeply than that.
COND_MAX = 64.0


def rel_err(got: np.ndarray, ref: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """|got - ref| / max(|ref|, scale / COND_MAX), scale = sum of
    |coefficient| over the terms active in that quantity."""
    den = np.maximum(np.abs(ref), scale / COND_MAX)
    den = np.where(den == 0, 1.0, den)
    return np.abs(got - ref) / den
