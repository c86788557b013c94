"""GPU parity of the batched annealer over instances of uneven size
(hobo_batch_*): every state of every instance is annealed exactly as the
per-instance hobo_anneal with the same seed anneals it."""
import numpy as np
import pytest

import gpuh
import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _mixed_instances():
    rng = np.random.default_rng(77)
    insts = []
    for t in range(10):
        N = int(rng.integers(16, 121))
        insts.append(W.random_sparse(700 + t, N, 3, 0.05, "normal"))
    insts.append(W.dense_float(720, 48))                    # dense layout group
    insts.append(W.random_sparse(721, 40, 4, 0.03, "normal"))   # order-4 group
    insts.append(W.random_sparse(722, 30, 5, 0.02, "int"))      # order 5..8 group
    return insts


@pytest.mark.parametrize("mode", [0, 1, 2], ids=["graph", "per_instance_tuned", "per_instance_plain"])
def test_batch_equals_per_instance_anneal(mode):
    import paper_2407_19987_gb300 as H
    insts = _mixed_instances()
    hs = [gpuh.make(i) for i in insts]
    B = [17 + 5 * t for t in range(len(hs))]               # uneven batch sizes
    seeds = [1000 + 3 * t for t in range(len(hs))]
    betas = W.geometric_betas(5.0, 0.05, 12)
    bt = H.Batch(hs, B)
    r = bt.anneal(seeds, betas, mode=mode, want_final=True, want_accepts=True)
    for t, h in enumerate(hs):
        ref = h.anneal(seeds[t], B[t], betas, want_final=True, want_accepts=True,
                       mode=H.HOBO_ANNEAL_PLAIN if mode == 2 else H.HOBO_ANNEAL_TUNED)
        np.testing.assert_array_equal(bt.rows(r["bestX"], t).cpu().numpy(), ref["bestX"].cpu().numpy())
        np.testing.assert_array_equal(bt.rows(r["bestE"], t).cpu().numpy(), ref["bestE"].cpu().numpy())
        np.testing.assert_array_equal(bt.rows(r["X"], t).cpu().numpy(), ref["X"].cpu().numpy())
        np.testing.assert_array_equal(bt.rows(r["E"], t).cpu().numpy(), ref["E"].cpu().numpy())
        np.testing.assert_array_equal(bt.rows(r["accepts"], t).cpu().numpy(), ref["accepts"].cpu().numpy())


def test_batch_integer_instances_match_oracle():
    import paper_2407_19987_gb300 as H
    insts = [W.random_sparse(800 + t, 20 + 7 * t, 3, 0.1, "int") for t in range(4)]
    hs = [gpuh.make(i) for i in insts]
    B = [8, 3, 11, 6]
    seeds = [5, 6, 7, 8]
    betas = W.geometric_betas(8.0, 0.1, 10)
    bt = H.Batch(hs, B)
    r = bt.anneal(seeds, betas, want_accepts=True)
    for t, inst in enumerate(insts):
        ref = O.anneal(inst, seeds[t], B[t], betas)
        np.testing.assert_array_equal(gpuh.to_host_bits(bt.rows(r["bestX"], t), inst.N), ref["bestX"])
        np.testing.assert_array_equal(bt.rows(r["bestE"], t).cpu().numpy(), ref["bestE"])
        np.testing.assert_array_equal(bt.rows(r["accepts"], t).cpu().numpy(), ref["accepts"])


def test_batch_graph_replay_with_new_seeds_and_schedule():
    """The captured graph is replayed; seeds and schedule are inputs of each
    call, not baked into the graph."""
    import paper_2407_19987_gb300 as H
    insts = [W.random_sparse(900 + t, 25 + 9 * t, 3, 0.08, "normal") for t in range(5)]
    hs = [gpuh.make(i) for i in insts]
    B = [10, 20, 5, 15, 12]
    bt = H.Batch(hs, B)
    for call, (seed0, T0) in enumerate(((1, 5.0), (50, 2.0), (77, 9.0))):
        seeds = [seed0 + t for t in range(5)]
        betas = W.geometric_betas(T0, 0.05, 9)
        r = bt.anneal(seeds, betas)
        for t, h in enumerate(hs):
            ref = h.anneal(seeds[t], B[t], betas)
            np.testing.assert_array_equal(bt.rows(r["bestX"], t).cpu().numpy(), ref["bestX"].cpu().numpy())
            np.testing.assert_array_equal(bt.rows(r["bestE"], t).cpu().numpy(), ref["bestE"].cpu().numpy())
    w, c = bt.launch_shape(0)
    assert 1 <= w <= 8 and c > 0


def test_batch_forced_launch_shapes_agree():
    import paper_2407_19987_gb300 as H
    insts = [W.random_sparse(950 + t, 30 + 11 * t, 3, 0.06, "normal") for t in range(4)]
    hs = [gpuh.make(i) for i in insts]
    B = [33, 7, 64, 21]
    seeds = [9, 8, 7, 6]
    betas = W.geometric_betas(4.0, 0.1, 8)
    bt = H.Batch(hs, B)
    outs = [bt.anneal(seeds, betas, no_autotune=True, warps_per_cta=w, ctas_per_sm=c)
            for w, c in ((1, 1), (4, 2), (8, 16))]
    for o in outs[1:]:
        np.testing.assert_array_equal(o["bestX"].cpu().numpy(), outs[0]["bestX"].cpu().numpy())
        np.testing.assert_array_equal(o["bestE"].cpu().numpy(), outs[0]["bestE"].cpu().numpy())


def test_uneven_batch_full_size_sampled():
    """512 order-3 instances, N ~ U[16,192], 5% density, B=1024 each, 500
    sweeps, in one graph launch; three sampled instances equal their
    per-instance anneals."""
    import paper_2407_19987_gb300 as H
    insts = W.uneven_batch(4000, 512)
    T0, T1, S, B = W.SCHEDULES["uneven_batch"]
    betas = W.geometric_betas(T0, T1, S)
    hs = [gpuh.make(i) for i in insts]
    bt = H.Batch(hs, [B] * len(hs))
    seeds = [4000 + t for t in range(len(hs))]
    r = bt.anneal(seeds, betas)
    for t in (0, 257, 511):
        ref = hs[t].anneal(seeds[t], B, betas)
        np.testing.assert_array_equal(bt.rows(r["bestX"], t).cpu().numpy(), ref["bestX"].cpu().numpy())
        np.testing.assert_array_equal(bt.rows(r["bestE"], t).cpu().numpy(), ref["bestE"].cpu().numpy())
