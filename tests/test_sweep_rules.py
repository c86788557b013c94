"""The facts the late-phase sweep's shortcuts rest on, checked on the CPU
against the oracle's Metropolis test (the definition every kernel follows):

- an uphill move whose exponent t = -(beta*dE)*log2(e) (float32 roundings)
  is below -125 is rejected whatever its draw, since the fixed exp2 is 0
  there and positive from -125 up;
- for t < -25 every draw other than u = 0 rejects (exp2(t) < 2^-24);
- t is non-increasing in beta for a fixed dE > 0, so a bit found frozen
  stays frozen at every larger beta until its field changes.
"""
import numpy as np

from oracle import oracle as O

LOG2E = np.frombuffer(np.uint32(0x3FB8AA3B).tobytes(), dtype=np.float32)[0]


def _t(beta, dE):
    a = np.float32(beta) * np.float32(dE)          # float32 products, round to nearest
    return -(np.float32(a) * LOG2E)


def test_exp2_is_zero_exactly_below_minus_125():
    ts = np.concatenate([np.linspace(-130.0, -120.0, 4001, dtype=np.float32),
                         np.array([np.nextafter(np.float32(-125.0), np.float32(-200.0)), np.float32(-125.0),
                                   np.nextafter(np.float32(-125.0), np.float32(0.0))], dtype=np.float32)])
    for t in ts:
        assert (O.exp2(float(t)) > 0.0) == (t >= np.float32(-125.0)), t


def test_exp2_below_minus_25_is_smaller_than_every_nonzero_draw():
    rng = np.random.default_rng(5)
    ts = np.concatenate([rng.uniform(-125.0, -25.0, 20000).astype(np.float32),
                         np.array([np.nextafter(np.float32(-25.0), np.float32(-200.0))], dtype=np.float32)])
    ts = ts[ts < np.float32(-25.0)]
    p = np.array([O.exp2(float(t)) for t in ts])
    assert (p < 2.0 ** -24).all()


def test_metropolis_decisions_the_shortcuts_assume():
    rng = np.random.default_rng(6)
    for _ in range(3000):
        dE = np.float32(rng.uniform(0.01, 50.0))
        beta = np.float32(rng.uniform(0.0, 30.0))
        t = _t(beta, dE)
        w_zero = int(rng.integers(0, 256))                 # u = 0
        w_any = int(rng.integers(256, 2 ** 32))            # u >= 2^-24
        assert O.metropolis(float(dE), float(beta), w_zero) == bool(t >= np.float32(-125.0))
        if t < np.float32(-25.0):
            assert not O.metropolis(float(dE), float(beta), w_any)
    # downhill and level moves are accepted without a draw
    assert O.metropolis(-1.0, 3.0, 2 ** 32 - 1) and O.metropolis(0.0, 3.0, 2 ** 32 - 1)


def test_exponent_is_non_increasing_in_beta():
    rng = np.random.default_rng(7)
    n = 200000
    dE = rng.uniform(1e-3, 300.0, n).astype(np.float32)
    b = np.sort(rng.uniform(0.0, 120.0, (n, 2)).astype(np.float32), axis=1)
    t1 = -((b[:, 0] * dE).astype(np.float32) * LOG2E).astype(np.float32)
    t2 = -((b[:, 1] * dE).astype(np.float32) * LOG2E).astype(np.float32)
    assert (t2 <= t1).all()
    # so "frozen at beta1" implies "frozen at beta2"
    assert not ((t1 < -125.0) & ~(t2 < -125.0)).any()
