"""GPU parity of the learned proposal: the network's forward and backward
passes against the oracle's float64 network on the same bf16-rounded
weights, the optimiser's first step against its closed form, and the
learned sweep (hobo_anneal_learned) against the oracle's learned annealer
on integer instances, trajectory for trajectory."""
import math

import numpy as np
import pytest

import gpuh
import workloads as W
from oracle import oracle as O
from test_oracle_mlp import identity_net

pytestmark = pytest.mark.gpu


def _H():
    import paper_2407_19987_gb300 as H
    return H


def _flat(w, H):
    return np.concatenate([w["W1"].reshape(-1), w["b1"], w["W2"].reshape(-1), w["b2"], w["w3"],
                           np.asarray(w["b3"]).reshape(-1)]).astype(np.float32)


def _features(rng, n):
    F = np.empty((n, 3), np.float32)
    F[:, 0] = np.clip(rng.standard_normal(n) * 2.0, -4, 4)
    F[:, 1] = rng.integers(0, 2, n) * 2 - 1
    F[:, 2] = rng.uniform(-1.0, 0.6, n)
    return F


def _abs_net(w):
    return {k: np.abs(v) for k, v in w.items()}


def tol_cuda_cores(H):
    """Bound on |logit - oracle| relative to the network run on magnitudes:
    layer 1, the H x H layer and the head each sum at most H + 4 float32
    terms (error <= (H + 4) 2^-24 of the sum of magnitudes; layer 1's error
    is far smaller), and ReLU and the next layer's weights carry an error
    on by at most its magnitude-network value."""
    return (2 * H + 8) * 2.0 ** -24


def tol_tensor_cores(H):
    """The same plus the two-plane split: bf16 keeps 8 significant bits, so
    |h1 - hi| <= 2^-8 |h1| and |h1 - hi - lo| <= 2^-16 |h1|; the products of
    the planes with the bf16 weights are exact."""
    return 2.0 ** -16 + tol_cuda_cores(H)


def test_mlp_forward_matches_oracle():
    T = gpuh.torch()
    m = _H().MLP(hidden=256, seed=3)
    w = m.unpack(m.params(rounded=True))
    rng = np.random.default_rng(1)
    F = _features(rng, 1000)   # 7 full 128-row tensor-core tiles and a ragged one
    got = m.forward(T.from_numpy(F).cuda()).cpu().numpy().astype(np.float64)
    ref = O.mlp_forward(w, F)
    # width 256: the tensor-core pass (bounds derived above)
    scale = O.mlp_forward(_abs_net(w), np.abs(F))
    assert np.all(np.abs(got - ref) <= tol_tensor_cores(256) * scale)
    assert m.forward(T.zeros((0, 3), device="cuda")).numel() == 0
    m.close()


def test_mlp_loss_and_gradients_match_oracle():
    T = gpuh.torch()
    m = _H().MLP(hidden=64, seed=4)
    w = m.unpack(m.params(rounded=True))
    rng = np.random.default_rng(2)
    n = 777
    F = _features(rng, n)
    y = (rng.random(n) < 0.3).astype(np.float32)
    loss, g = m.loss_grad(T.from_numpy(F).cuda(), T.from_numpy(y).cuda())
    rl, rg = O.mlp_loss_grad(w, F, y)
    assert abs(float(loss.item()) - rl) <= 1e-5 * abs(rl)
    got = m.unpack(g.cpu().numpy())
    for k in ("W1", "b1", "W2", "b2", "w3", "b3"):
        ref = rg[k].reshape(got[k].shape)
        tol = 2e-4 * np.max(np.abs(ref)) + 1e-7
        assert np.max(np.abs(got[k] - ref)) <= tol, k
    m.close()


def test_adam_first_step_moves_each_weight_by_lr():
    # from zero moments, Adam's first update is lr * g / (|g| + eps)
    T = gpuh.torch()
    m = _H().MLP(hidden=32, seed=5)
    rng = np.random.default_rng(3)
    F = T.from_numpy(_features(rng, 300)).cuda()
    y = T.from_numpy((rng.random(300) < 0.5).astype(np.float32)).cuda()
    w0 = m.params(rounded=False)
    _, g = m.loss_grad(F, y)
    g = g.cpu().numpy()
    lr = 1e-3
    m.train_step(F, y, lr)
    T.cuda.synchronize()
    w1 = m.params(rounded=False)
    big = np.abs(g) > 1e-5
    step = (w0 - w1)[big]
    np.testing.assert_allclose(step, lr * np.sign(g[big]), rtol=1e-4, atol=1e-6 * np.max(np.abs(w0)))
    assert np.array_equal(w1[g == 0], w0[g == 0])
    # rounded copies follow the masters
    r = m.params(rounded=True)
    assert np.array_equal(r, T.from_numpy(w1).bfloat16().float().numpy())
    m.close()


def test_training_reduces_loss():
    T = gpuh.torch()
    m = _H().MLP(hidden=128, seed=6)
    rng = np.random.default_rng(4)
    Fn = _features(rng, 4096)
    yn = ((Fn[:, 0] * Fn[:, 1]) < 0).astype(np.float32)
    F, y = T.from_numpy(Fn).cuda(), T.from_numpy(yn).cuda()
    loss = T.zeros(1, device="cuda")
    l0, _ = m.loss_grad(F, y)
    l0 = float(l0.item())
    for _ in range(200):
        m.train_step(F, y, 3e-3, loss)
    l1, _ = m.loss_grad(F, y)
    assert float(l1.item()) < 0.5 * l0


def test_save_load_roundtrip(tmp_path):
    T = gpuh.torch()
    m = _H().MLP(hidden=96, seed=7)
    p = str(tmp_path / "net.bin")
    m.save(p)
    m2 = _H().MLP.load(p)
    assert m2.hidden == 96
    assert np.array_equal(m.params(rounded=True), m2.params(rounded=True))
    F = T.from_numpy(_features(np.random.default_rng(5), 130)).cuda()
    assert T.equal(m.forward(F), m2.forward(F))
    with open(p, "r+b") as f:
        f.write(b"{\"format\": \"other\"}\n")
    with pytest.raises(_H().HoboError):
        _H().MLP.load(p)


def _set_net(w, H=32):
    m = _H().MLP(hidden=H, seed=0)
    m.set_params(_flat(w, H))
    return m


def _compare(r, ref, N):
    np.testing.assert_array_equal(gpuh.to_host_bits(r["bestX"], N), ref["bestX"])
    np.testing.assert_array_equal(r["bestE"].cpu().numpy(), ref["bestE"])
    np.testing.assert_array_equal(gpuh.to_host_bits(r["X"], N), ref["X"])
    np.testing.assert_array_equal(r["E"].cpu().numpy().astype(np.float64), ref["E"])
    np.testing.assert_array_equal(r["accepts"].cpu().numpy(), ref["accepts"])


CASES = [
    ("tiny_dense", lambda: W.tiny_dense(1), 0, 40, (5.0, 0.05, 60)),
    ("dense_int_N64", lambda: W.random_sparse(40, 64, 3, 0.5, "int"), 4, 24, (30.0, 0.1, 12)),
    ("order3_N45", lambda: W.random_sparse(42, 45, 3, 0.05, "int"), 0, 40, (10.0, 0.1, 20)),
    ("order4_N96", lambda: W.sparse_order4(5003), 0, 24, (8.0, 0.05, 16)),
    ("order6_N20", lambda: W.random_sparse(45, 20, 6, 0.02, "int"), 0, 20, (10.0, 0.1, 15)),
]


# (plain_every, select, top_frac, threshold).  With the identity network the
# score is clamp(beta g)/8; on integer instances distinct scores differ by
# at least beta/8, far above the table interpolation's rounding, and no
# score lies within that rounding of the thresholds -1e-3 and 0.3, so the
# interpolated scores order and select exactly as the oracle's.
SELECTS = [(3, 0, 1.0, 0.0), (4, 0, 0.6, 0.0), (2, 0, 0.1, 0.0), (3, 1, 1.0, -1e-3), (2, 1, 1.0, 0.3)]


@pytest.mark.parametrize("name,maker,flags,B,sched", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("plain_every,select,top_frac,threshold", SELECTS)
def test_learned_anneal_matches_oracle(name, maker, flags, B, sched, plain_every, select, top_frac, threshold):
    inst = maker()
    betas = W.geometric_betas(*sched)
    h = gpuh.make(inst, flags)
    w = identity_net()
    m = _set_net(w)
    r = _H().anneal_learned(h, m, 77, B, betas, plain_every=plain_every, select=select, top_frac=top_frac,
                            threshold=threshold, want_final=True, want_accepts=True)
    ref = O.anneal_learned(inst, 77, B, betas, w, plain_every=plain_every, select=select, top_frac=top_frac,
                           threshold=threshold)
    _compare(r, ref, inst.N)
    h.close()


@pytest.mark.parametrize("net", ["none", "constant", "plain_every_1"])
def test_learned_anneal_reduces_to_tuned_anneal(net):
    inst = W.random_sparse(46, 70, 3, 0.1, "normal")
    betas = W.geometric_betas(5.0, 0.05, 30)
    h = gpuh.make(inst)
    m, pe = None, 4
    if net == "constant":
        w = identity_net()
        w = {k: np.zeros_like(v) for k, v in w.items()}
        w["b3"] = np.array([0.25])
        m = _set_net(w)
    elif net == "plain_every_1":
        m, pe = _H().MLP(hidden=64, seed=8), 1
    r = _H().anneal_learned(h, m, 5, 50, betas, plain_every=pe, want_final=True, want_accepts=True)
    t = h.anneal(5, 50, betas, mode=0, want_final=True, want_accepts=True)
    for k in ("bestX", "bestE", "X", "E", "accepts"):
        assert gpuh.torch().equal(r[k], t[k]), k
    h.close()


def test_recorded_features_and_labels_match_oracle():
    inst = W.sparse_order4(5004, N=64, density=0.03)
    betas = W.geometric_betas(8.0, 0.05, 24)
    h = gpuh.make(inst)
    w = identity_net()
    m = _set_net(w)
    for net, sel in ((None, 0), (m, 0), (m, 1)):
        r = _H().anneal_learned(h, net, 31, 40, betas, plain_every=3, select=sel, top_frac=0.5, threshold=-1e-3,
                                rec_every=5, rec_states=7)
        ref = O.anneal_learned(inst, 31, 40, betas, w if net is not None else None, plain_every=3,
                               select=sel, top_frac=0.5, threshold=-1e-3, rec_every=5, rec_B=7)
        F = r["rec_F"].cpu().numpy()
        np.testing.assert_array_equal(r["rec_y"].cpu().numpy(), ref["rec_y"])
        np.testing.assert_array_equal(F[:, :2], ref["rec_F"][:, :2])
        np.testing.assert_allclose(F[:, 2], ref["rec_F"][:, 2], rtol=2.5e-7, atol=0)
        if net is None:
            assert np.all(ref["rec_y"] >= 0)
        else:
            assert np.any(ref["rec_y"] < 0)
    h.close()


def test_learned_anneal_arguments():
    inst = W.random_sparse(47, 300, 3, 0.01, "normal")
    h = gpuh.make(inst)
    with pytest.raises(_H().HoboError):
        _H().anneal_learned(h, None, 1, 8, W.geometric_betas(5, .1, 4))   # N > 256
    h.close()
    h = gpuh.make(W.tiny_dense(1))
    with pytest.raises(_H().HoboError):
        _H().anneal_learned(h, None, 1, 8, W.geometric_betas(5, .1, 4), select=2)
    r = _H().anneal_learned(h, None, 1, 0, W.geometric_betas(5, .1, 4))
    assert r["bestE"].numel() == 0
    r = _H().anneal_learned(h, None, 1, 16, np.zeros(0, np.float32), want_final=True)
    X0 = O.init_states(1, 12, 16)
    np.testing.assert_array_equal(gpuh.to_host_bits(r["bestX"], 12), X0)
    h.close()


def test_trained_network_gain_over_the_sweep_without_it():
    """What the trained network gains in wall time: train it on recorded
    plain-annealer trajectories of seeded order-4 instances (N=96, 2%
    density), then on held-out instances compare the time to reach a
    target (lowest energy of 64 runs x 2000 sweeps + 0.5%) with 99%
    confidence, TTS99 = call time / B * ln 0.01 / ln(1 - p), minimised over
    schedule lengths, with and without the network.  Measured outcome,
    asserted: training lowers the loss by an order of magnitude; both forms
    reach the target; a learned sweep costs at least 1.2x a plain one (it
    sorts the N scores every sweep); and the learned form's best TTS99 is
    no better than the tuned sweep's (geomean ratio >= 0.9, measured about
    1.2 on the bench's instances): on wall time the network gains nothing
    on this workload."""
    import bench
    import paper_2407_19987_gb300 as H
    from paper_2407_19987_gb300 import learned as LP
    train = [W.sparse_order4(10 ** 6 + k) for k in range(16)]
    hs = [gpuh.make(i) for i in train]
    betas = W.geometric_betas(8.0, 0.05, 200)
    F, y = LP.record(hs, seed=10 ** 6, B=128, betas=betas, rec_every=4, rec_states=16)
    for h in hs:
        h.close()
    net = H.MLP(256, seed=1)
    loss0 = LP.full_loss(net, F, y)
    LP.train(net, F, y, steps=600, batch=8192, lr=1e-3, seed=1)
    loss1 = LP.full_loss(net, F, y)
    assert loss1 < 0.1 * loss0
    B = 2048
    ratios, cost = [], []
    for seed in (5000, 5001):
        inst = W.sparse_order4(seed)
        h = gpuh.make(inst)
        r = h.anneal(99, 64, W.geometric_betas(8.0, 0.05, 2000))
        best = float(r["bestE"].min().item())
        target = best + 0.005 * abs(best)

        def tuned(S):
            E, ms = LP.run_schedule(h, None, seed=11, B=B, betas=W.geometric_betas(8.0, 0.05, S))
            return E, ms

        def learned(S):
            E, ms = LP.run_schedule(h, net, seed=11, B=B, betas=W.geometric_betas(8.0, 0.05, S), plain_every=4)
            return E, ms

        for fn in (tuned, learned):
            fn(20)                                       # warm-up
        ladder = (20, 50, 100, 200)
        t = bench.tts_ladder(tuned, target, B, ladder)
        l = bench.tts_ladder(learned, target, B, ladder)
        assert t["best"] is not None and l["best"] is not None
        ratios.append(l["best"]["tts99_ms"] / t["best"]["tts99_ms"])
        cost.append(l["rungs"][-1]["ms"] / t["rungs"][-1]["ms"])
        print(f"seed {seed}: TTS99 tuned {t['best']['tts99_ms']:.4f} ms at {t['best']['sweeps']} sweeps, "
              f"learned {l['best']['tts99_ms']:.4f} ms at {l['best']['sweeps']}; 200-sweep call "
              f"{t['rungs'][-1]['ms']:.2f} vs {l['rungs'][-1]['ms']:.2f} ms")
        h.close()
    net.close()
    assert min(cost) >= 1.2, cost
    assert float(np.exp(np.mean(np.log(ratios)))) >= 0.9, ratios


@pytest.mark.parametrize("name,maker", [("N1_order1", lambda: W.random_sparse(80, 1, 1, 0.0, "int")),
                                        ("complete_N3_order3", lambda: W.dense_all_degrees(83, 3, 3, "int"))],
                         ids=["N1_order1", "complete_N3_order3"])
@pytest.mark.parametrize("select", [0, 1])
def test_learned_anneal_degenerate_instances_match_oracle(name, maker, select):
    """One variable, and a complete three-variable instance: the learned
    sweep sorts or filters keys of which all but one or three are padding."""
    inst = maker()
    betas = W.geometric_betas(5.0, 0.05, 12)
    h = gpuh.make(inst)
    w = identity_net()
    m = _set_net(w)
    r = _H().anneal_learned(h, m, 5, 33, betas, plain_every=3, select=select, top_frac=1.0, threshold=-1e-3,
                            want_final=True, want_accepts=True)
    ref = O.anneal_learned(inst, 5, 33, betas, w, plain_every=3, select=select, top_frac=1.0, threshold=-1e-3)
    _compare(r, ref, inst.N)
    h.close()
    m.close()
