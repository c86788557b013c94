"""Pins of the oracle's learned-proposal routines (network and annealer).

The network has no counterpart in the paper; what pins it here is
independent of the oracle's own code: finite differences of its loss,
networks built by hand to compute a known function, and the closed form of
the binary cross-entropy at constant logits.  The learned annealer is tied
to the plain annealer (no network, constant network) and to a directly
computed top-k set of scores.
"""
import math

import numpy as np
import pytest

import workloads as WL
from oracle import oracle as O


def _random_net(rng, H):
    return {"W1": rng.standard_normal((H, 3)) * 0.8, "b1": rng.standard_normal(H) * 0.3,
            "W2": rng.standard_normal((H, H)) * (1.5 / math.sqrt(H)), "b2": rng.standard_normal(H) * 0.3,
            "w3": rng.standard_normal(H) * (1.0 / math.sqrt(H)), "b3": np.array([0.1])}


def _zero_net(H, b3=0.0):
    return {"W1": np.zeros((H, 3)), "b1": np.zeros(H), "W2": np.zeros((H, H)), "b2": np.zeros(H),
            "w3": np.zeros(H), "b3": np.array([b3])}


def identity_net(H=32):
    """logit = f0: h1 = (relu(f0), relu(-f0), relu(f1), 0...), layer 2 a
    cyclic shift of the first three units (not symmetric, so a transposed
    W2 is caught), w3 picks +relu(f0) - relu(-f0)."""
    w = _zero_net(H)
    w["W1"][0, 0] = 1.0
    w["W1"][1, 0] = -1.0
    w["W1"][2, 1] = 1.0
    # z2[0] = h1[1], z2[1] = h1[2], z2[2] = h1[0]
    w["W2"][0, 1] = 1.0
    w["W2"][1, 2] = 1.0
    w["W2"][2, 0] = 1.0
    w["w3"][0] = -1.0
    w["w3"][2] = 1.0
    return w


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(11)
    H, n = 8, 24
    w = _random_net(rng, H)
    F = rng.standard_normal((n, 3))
    y = (rng.random(n) < 0.4).astype(np.float64)
    loss, g = O.mlp_loss_grad(w, F, y)
    h = 1e-6
    for k in ("W1", "b1", "W2", "b2", "w3", "b3"):
        flat = w[k].reshape(-1)
        for j in range(flat.size):
            wp = {kk: vv.copy() for kk, vv in w.items()}
            wm = {kk: vv.copy() for kk, vv in w.items()}
            wp[k].reshape(-1)[j] += h
            wm[k].reshape(-1)[j] -= h
            fd = (O.mlp_loss_grad(wp, F, y)[0] - O.mlp_loss_grad(wm, F, y)[0]) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[j]) < 1e-7 + 1e-5 * abs(fd), (k, j)


def test_mlp_loss_equals_mean_of_forward_cross_entropy():
    rng = np.random.default_rng(12)
    w = _random_net(rng, 6)
    F = rng.standard_normal((10, 3))
    y = (rng.random(10) < 0.5).astype(np.float64)
    z = O.mlp_forward(w, F)
    want = np.mean(np.log1p(np.exp(-np.abs(z))) + np.maximum(z, 0) - y * z)
    assert O.mlp_loss_grad(w, F, y)[0] == pytest.approx(want, rel=1e-12)


def test_identity_network_computes_first_feature():
    rng = np.random.default_rng(13)
    F = rng.standard_normal((50, 3)) * 3
    assert np.array_equal(O.mlp_forward(identity_net(), F), F[:, 0])
    w = identity_net()
    w["W2"] = w["W2"].T.copy()
    assert not np.allclose(O.mlp_forward(w, F), F[:, 0])


def test_constant_logit_closed_forms():
    # all weights zero, b3 = c: logit c everywhere; loss = softplus(c) - mean(y) c,
    # d/d b3 = sigmoid(c) - mean(y); every other gradient is zero
    rng = np.random.default_rng(14)
    F = rng.standard_normal((9, 3))
    y = np.array([1, 0, 0, 1, 1, 0, 1, 1, 0], np.float64)
    for c in (0.0, 2.0, -3.5):
        w = _zero_net(4, c)
        assert np.all(O.mlp_forward(w, F) == c)
        loss, g = O.mlp_loss_grad(w, F, y)
        assert loss == pytest.approx(math.log1p(math.exp(c)) - y.mean() * c, rel=1e-14, abs=1e-15)
        assert g["b3"][0] == pytest.approx(1 / (1 + math.exp(-c)) - y.mean(), rel=1e-14, abs=1e-15)
        for k in ("W1", "b1", "W2", "b2", "w3"):
            assert not np.any(g[k])
    # at logit 0 the loss is ln 2 whatever the labels
    assert O.mlp_loss_grad(_zero_net(4), F, y)[0] == pytest.approx(math.log(2), rel=1e-15)
    # with b2 = 1 (so h2 = 1) the w3 gradient is the b3 gradient per unit
    w = _zero_net(4, 0.5)
    w["b2"][:] = 1.0
    _, g = O.mlp_loss_grad(w, F, y)
    assert np.allclose(g["w3"], g["b3"][0], rtol=1e-14)


def _sched(inst, sweeps):
    return WL.geometric_betas(5.0, 0.05, sweeps)


def test_learned_anneal_without_network_is_plain_anneal():
    inst = WL.sparse_order4(seed=5001, N=40, density=0.05)
    b = _sched(inst, 30)
    a = O.anneal(inst, 3, 8, b)
    l = O.anneal_learned(inst, 3, 8, b, None, plain_every=4)
    for k in ("X", "E", "bestX", "bestE", "accepts"):
        assert np.array_equal(a[k], l[k]), k


def test_learned_anneal_with_constant_network_is_plain_anneal():
    # equal scores everywhere: ties go by index, which is the plain order
    inst = WL.tiny_dense()
    b = _sched(inst, 40)
    a = O.anneal(inst, 9, 8, b)
    l = O.anneal_learned(inst, 9, 8, b, _zero_net(32, 0.7), plain_every=3, top_frac=1.0)
    for k in ("X", "E", "bestX", "bestE", "accepts"):
        assert np.array_equal(a[k], l[k]), k


def test_learned_sweep_attempts_top_scores_of_start_state():
    # one learned sweep (plain_every = 2 makes sweep 0 learned): the recorded
    # (attempted) bits are the ceil(top_frac N) largest clamp(beta g)/8 of
    # the initial state, ties to the lower index
    inst = WL.tiny_dense()
    N, B = inst.N, 6
    beta = np.array([0.7], np.float32)
    X0 = O.init_states(21, N, B)
    for top_frac in (0.25, 0.5, 1.0):
        r = O.anneal_learned(inst, 21, B, beta, identity_net(), plain_every=2, top_frac=top_frac,
                             vmax=6.0, rec_every=1, rec_B=B)
        k = math.ceil(top_frac * N)
        for b in range(B):
            g = O.fields(inst, X0[b]).astype(np.float32)
            v = np.clip(beta[0] * g, -6.0, 6.0) / 8
            order = sorted(range(N), key=lambda i: (-v[i], i))
            got = set(np.nonzero(r["rec_x"][b * N:(b + 1) * N] != 0xFF)[0])
            assert got == set(order[:k])
        # at most one flip per attempted bit
        assert np.all(r["accepts"] <= k)


def test_learned_anneal_energies_are_consistent():
    inst = WL.sparse_order4(seed=5002, N=48, density=0.04)
    b = WL.geometric_betas(8.0, 0.05, 40)
    r = O.anneal_learned(inst, 5, 6, b, identity_net(), plain_every=4, top_frac=0.5)
    assert np.array_equal(r["E"], O.energy(inst, r["X"]))
    assert np.array_equal(r["bestE"], O.energy(inst, r["bestX"]))
    assert np.all(r["bestE"] <= r["E"])


def test_threshold_sweep_attempts_bits_at_or_above_threshold():
    # select 1: one learned sweep attempts exactly the bits whose score
    # (here clamp(beta g)/8) is >= threshold at the start state
    inst = WL.sparse_order4(seed=5005, N=40, density=0.05)
    N, B = inst.N, 5
    beta = np.array([0.3], np.float32)
    X0 = O.init_states(8, N, B)
    for thr in (-0.2, 0.0, 0.4):
        r = O.anneal_learned(inst, 8, B, beta, identity_net(), plain_every=2, select=1, threshold=thr,
                             vmax=20.0, rec_every=1, rec_B=B)
        for b in range(B):
            g = O.fields(inst, X0[b]).astype(np.float32)
            v = np.clip(beta[0] * g, -20.0, 20.0) / 8
            got = set(np.nonzero(r["rec_x"][b * N:(b + 1) * N] != 0xFF)[0])
            assert got == set(np.nonzero(v >= thr)[0])


def test_threshold_below_every_score_is_plain_anneal():
    inst = WL.tiny_dense()
    b = _sched(inst, 30)
    a = O.anneal(inst, 4, 6, b)
    l = O.anneal_learned(inst, 4, 6, b, identity_net(), plain_every=3, select=1, threshold=-1e9)
    for k in ("X", "E", "bestX", "bestE", "accepts"):
        assert np.array_equal(a[k], l[k]), k
