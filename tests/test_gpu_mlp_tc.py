"""Tensor-core forward pass of the proposal network (hidden widths 64..256):
logits against the oracle's float64 network on the same bf16-rounded
weights (and the CUDA-core pass beside it), the learned sweep's score
tables against the oracle network on the table's features, and learned
anneals whose tables come from this pass against the oracle's learned
annealer, trajectory for trajectory."""
import numpy as np
import pytest

import gpuh
import workloads as W
from oracle import oracle as O
from test_gpu_learned import CASES, _abs_net, _compare, _features, _set_net, tol_cuda_cores, tol_tensor_cores
from test_oracle_mlp import identity_net

pytestmark = pytest.mark.gpu


def _H():
    import paper_2407_19987_gb300 as H
    return H


@pytest.mark.parametrize("H", [64, 128, 192, 256])
@pytest.mark.parametrize("n", [1, 127, 1000, 40000])
def test_tensor_core_forward_matches_oracle(H, n):
    if n == 40000 and H in (128, 192):
        pytest.skip("the large case runs at the smallest and largest width")
    T = gpuh.torch()
    m = _H().MLP(hidden=H, seed=10 + H)
    w = m.unpack(m.params(rounded=True))
    rng = np.random.default_rng(H * 7 + n)
    F = _features(rng, n)          # n = 1000: 7 full 128-row tiles and a ragged one;
    Fd = T.from_numpy(F).cuda()    # n = 40000: 313 tiles, several per CTA
    got = m.forward(Fd).cpu().numpy().astype(np.float64)
    m.check()
    ref = O.mlp_forward(w, F)
    scale = O.mlp_forward(_abs_net(w), np.abs(F))
    assert np.all(np.abs(got - ref) <= tol_tensor_cores(H) * scale)
    m.set_tensor_cores(False)
    cc = m.forward(Fd).cpu().numpy().astype(np.float64)
    assert np.all(np.abs(cc - ref) <= tol_cuda_cores(H) * scale)
    m.close()


def test_tensor_core_forward_of_special_networks():
    """The identity network gives logit = f0 up to the two-plane split (2^-16);
    a network with W2 = 0 gives b3 + sum w3 relu(b2) exactly on every row."""
    T = gpuh.torch()
    rng = np.random.default_rng(3)
    F = _features(rng, 300)
    m = _set_net(identity_net(64), 64)
    got = m.forward(T.from_numpy(F).cuda()).cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, F[:, 0].astype(np.float64), rtol=2.0 ** -16, atol=0)
    m.close()
    w = identity_net(128)
    w["W2"][:] = 0.0
    w["b2"][:] = np.linspace(-1, 1, 128)
    w["w3"][:] = np.linspace(0.5, -0.25, 128)
    w["b3"] = np.array([0.125])
    m = _set_net(w, 128)
    got = m.forward(T.from_numpy(F).cuda()).cpu().numpy()
    wr = m.unpack(m.params(rounded=True))
    ref = O.mlp_forward(wr, F)
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-5)
    assert np.all(got == got[0])
    m.close()


@pytest.mark.parametrize("H,G", [(256, 256), (64, 33)])
def test_score_tables_match_oracle_network(H, G):
    T = gpuh.torch()
    m = _H().MLP(hidden=H, seed=21)
    w = m.unpack(m.params(rounded=True))
    betas = W.geometric_betas(8.0, 0.05, 37)
    vmax = 32.0
    tab = m.score_tables(T.from_numpy(betas).cuda(), G, vmax).cpu().numpy().astype(np.float64)
    m.check()
    assert tab.shape == (37, 2, G)
    # features of row (s, x, k): (v_k / 8, 2x - 1, -ln(beta_s) / 4)
    k = np.arange(G, dtype=np.float64)
    v = -vmax + 2 * vmax * k / (G - 1)
    S = len(betas)
    F = np.empty((S, 2, G, 3))
    F[..., 0] = v / 8
    F[:, 0, :, 1], F[:, 1, :, 1] = -1.0, 1.0
    F[..., 2] = (-np.log(betas.astype(np.float64)) / 4)[:, None, None]
    F = F.reshape(-1, 3)
    ref = O.mlp_forward(w, F).reshape(S, 2, G)
    scale = O.mlp_forward(_abs_net(w), np.abs(F)).reshape(S, 2, G)
    # (+1e-6: the kernel forms -ln(beta)/4 in float32 from the float32 beta)
    assert np.all(np.abs(tab - ref) <= tol_tensor_cores(H) * scale + 1e-6)
    m.set_tensor_cores(False)
    cc = m.score_tables(T.from_numpy(betas).cuda(), G, vmax).cpu().numpy().astype(np.float64)
    assert np.all(np.abs(cc - ref) <= tol_cuda_cores(H) * scale + 1e-6)
    m.close()


def test_tensor_core_path_selection_and_arguments():
    T = gpuh.torch()
    H = _H()
    for width in (32, 96, 320):
        m = H.MLP(hidden=width, seed=1)
        with pytest.raises(H.HoboError):
            m.set_tensor_cores(True)
        m.set_tensor_cores(False)
        m.close()
    m = H.MLP(hidden=64, seed=1)
    b = T.ones(4, device="cuda")
    with pytest.raises(H.HoboError):
        m.score_tables(b, G=1)
    with pytest.raises(H.HoboError):
        m.score_tables(b, G=16, vmax=0.0)
    assert m.score_tables(T.ones(0, device="cuda"), G=16).shape == (0, 2, 16)
    m.check()
    m.close()


SELECTS_TC = [(3, 0, 1.0, 0.0), (2, 0, 0.1, 0.0), (3, 1, 1.0, -1e-3)]


@pytest.mark.parametrize("name,maker,flags,B,sched", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("plain_every,select,top_frac,threshold", SELECTS_TC)
def test_learned_anneal_with_tensor_core_tables_matches_oracle(name, maker, flags, B, sched, plain_every, select,
                                                               top_frac, threshold):
    """Identity network of width 64 (tables from the tensor-core pass): the
    two-plane residual (<= 2^-16 of a score) is far below the beta/8 gap
    between distinct scores on integer instances and below the distance of
    every score to the threshold -1e-3, so selections equal the oracle's."""
    inst = maker()
    betas = W.geometric_betas(*sched)
    h = gpuh.make(inst, flags)
    w = identity_net(64)
    m = _set_net(w, 64)
    r = _H().anneal_learned(h, m, 77, B, betas, plain_every=plain_every, select=select, top_frac=top_frac,
                            threshold=threshold, want_final=True, want_accepts=True)
    h.check()
    ref = O.anneal_learned(inst, 77, B, betas, w, plain_every=plain_every, select=select, top_frac=top_frac,
                           threshold=threshold)
    _compare(r, ref, inst.N)
    h.close()
    m.close()


@pytest.mark.parametrize("H", [32, 1024])
def test_cuda_core_forward_at_the_smallest_and_largest_width(H):
    """Widths the tensor-core pass does not take run the float32 passes."""
    T = gpuh.torch()
    m = _H().MLP(hidden=H, seed=H)
    with pytest.raises(_H().HoboError):
        m.set_tensor_cores(True)
    w = m.unpack(m.params(rounded=True))
    F = _features(np.random.default_rng(H), 300)
    got = m.forward(T.from_numpy(F).cuda()).cpu().numpy().astype(np.float64)
    ref = O.mlp_forward(w, F)
    scale = O.mlp_forward(_abs_net(w), np.abs(F))
    assert np.all(np.abs(got - ref) <= tol_cuda_cores(H) * scale)
    m.close()
