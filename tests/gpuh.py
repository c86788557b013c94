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


# The float bar: err = |got - ref| / max(|ref|, A / COND_MAX) <= 1e-5, with
# A the sum of |coefficient| over the terms active in that quantity (the
# floor 2^-10 A of the scope's reading of the relative-error bar).  The
# exact fixed-point paths (term list, tensor-core limb planes) round each
# result once, so they meet it with a wide margin.  The kernels that
# accumulate bf16-split products in float32 (the order-4 tensor-core path,
# the float32-accumulating order-3 path kept for comparison) carry float32
# summation error relative to A: they are held to the floor A / 64 (1e-5 of
# it is 2.6 float32 ulps of A), COND_MAX_F32ACC.
COND_MAX = 1024.0
COND_MAX_F32ACC = 64.0


def rel_err(got: np.ndarray, ref: np.ndarray, scale: np.ndarray, cond_max: float = COND_MAX) -> np.ndarray:
    """|got - ref| / max(|ref|, scale / cond_max), scale = sum of
    |coefficient| over the terms active in that quantity."""
    den = np.maximum(np.abs(ref), scale / cond_max)
    den = np.where(den == 0, 1.0, den)
    return np.abs(got - ref) / den


def fix_shift(abs_sum: float) -> int:
    """The library's fixed-point scale S: the sum of all |coefficients|
    times 2^S stays below 2^62."""
    import math
    if abs_sum <= 0:
        return 0
    return 62 - math.frexp(abs_sum)[1]
