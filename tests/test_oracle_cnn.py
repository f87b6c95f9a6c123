"""Pins of the oracle's convolutional network.

  * conv against scipy.signal.correlate2d (zero padding), channel by channel;
  * backward against central finite differences of the loss;
  * Adam: first step moves each parameter by lr * sign(grad).
"""
import numpy as np
import pytest
import scipy.signal

from oracle import cnn
from paper_2404_17542_gb300 import inputs


def small_net(seed, c_in=3, width=4, layers=3):
    ws, bs = inputs.cnn_weights(seed, c_in=c_in, width=width, layers=layers)
    rng = np.random.default_rng(seed + 1)
    bs = [rng.normal(0, 0.1, size=b.shape) for b in bs]
    return ws, bs


def test_conv_matches_library_correlation():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 7, 9))
    w = rng.normal(size=(2, 3, 3, 3))
    b = rng.normal(size=2)
    y = cnn.conv(x, w, b)
    for o in range(2):
        want = b[o] + sum(scipy.signal.correlate2d(x[c], w[o, c], mode="same", boundary="fill")
                          for c in range(3))
        assert np.allclose(y[o], want, atol=1e-12)


def test_backward_matches_finite_differences():
    ws, bs = small_net(3)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(3, 6, 5))
    target = rng.normal(size=(1, 6, 5))
    weight = (rng.uniform(size=(1, 6, 5)) > 0.3).astype(float)

    def L():
        return cnn.loss(cnn.forward(ws, bs, x)[-1], target, weight)[0]

    acts = cnn.forward(ws, bs, x)
    _l, dy = cnn.loss(acts[-1], target, weight)
    dws, dbs = cnn.backward(ws, bs, acts, dy)
    h = 1e-6
    for li in range(len(ws)):
        for idx in [(0, 0, 1, 1), (1, 2, 0, 2), (0, 1, 2, 0)]:
            if any(a >= s for a, s in zip(idx, ws[li].shape)):
                continue
            old = ws[li][idx]
            ws[li][idx] = old + h
            lp = L()
            ws[li][idx] = old - h
            lm = L()
            ws[li][idx] = old
            assert dws[li][idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)
        old = bs[li][0]
        bs[li][0] = old + h
        lp = L()
        bs[li][0] = old - h
        lm = L()
        bs[li][0] = old
        assert dbs[li][0] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)


def test_adam_first_step_is_signed_lr():
    p = [np.array([1.0, -2.0, 0.5])]
    g = [np.array([0.3, -4.0, 1e-3])]
    m = [np.zeros(3)]
    v = [np.zeros(3)]
    cnn.adam(p, g, m, v, 1, lr=0.01, eps=0.0)
    assert np.allclose(p[0], [1.0 - 0.01, -2.0 + 0.01, 0.5 - 0.01])


def test_features_channels():
    pb = inputs.jittered_box(8, 2, seed=2)
    r = np.arange(pb.mesh.N, dtype=float)
    x, (s_r, s_d, s_out) = cnn.features(pb.mesh, r, pb.mask, pb.pos)
    assert x.shape == (8, 8, 8)
    assert np.allclose(x[1] + x[2] + x[3], 1.0)
    assert np.abs(x[4]).max() <= 0.5 + 1e-12 and np.abs(x[5]).max() <= 0.5 + 1e-12
    assert s_r == pytest.approx(np.sqrt(np.mean(r ** 2)))
    assert s_d == 0.0 and s_out == pytest.approx(s_r * pb.mesh.l0 ** 2)
    assert not x[6].any() and not x[7].any()
    d = np.full(pb.mesh.N, -3.0)
    x, (_sr, s_d, s_out) = cnn.features(pb.mesh, r, pb.mask, pb.pos, d)
    assert s_d == s_out == 3.0 and np.allclose(x[6], -1.0)


def test_bf16_round_definition():
    # exactly representable values stay; halfway cases go to the even mantissa
    assert cnn.bf16_round(1.0) == 1.0 and cnn.bf16_round(-0.375) == -0.375
    assert cnn.bf16_round(1.0 + 2.0 ** -8) == 1.0                    # tie -> even (1.0)
    assert cnn.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2 * 2.0 ** -7  # tie -> even
    assert cnn.bf16_round(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    x = (np.random.default_rng(1).normal(size=1000) * 1e3).astype(np.float32)
    y = cnn.bf16_round(x.astype(np.float64))
    assert np.all(np.abs(y - x) <= np.abs(x) * 2.0 ** -8)           # half an ulp
    assert np.array_equal(cnn.bf16_round(y), y)                      # idempotent
    # second definition: round the float32 bit pattern at bit 16, ties to even
    bits = x.view(np.uint32).astype(np.uint64)
    rb = ((bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    assert np.array_equal(rb.view(np.float32).astype(np.float64), y)


def test_warm_start_is_the_residual_minimiser():
    rng = np.random.default_rng(7)
    A = rng.normal(size=(12, 12)) + 12 * np.eye(12)
    b, p, e = rng.normal(size=(3, 12))
    q, s = cnn.warm_start(A, b, p, e)
    res = lambda x: np.linalg.norm(b - A @ x)
    assert res(q) <= res(p)
    for d in (-1e-3, 1e-3):
        assert res(q) <= res(p + (s + d) * e)
    # e = exact correction gives the solution with s = 1
    q, s = cnn.warm_start(A, b, p, np.linalg.solve(A, b) - p)
    assert s == pytest.approx(1.0) and res(q) < 1e-10


def test_flatten_round_trip():
    ws, bs = inputs.cnn_weights(5)
    flat = inputs.cnn_flatten(ws, bs)
    assert flat.size == 7 * 32 * 9 + 32 + 2 * (32 * 32 * 9 + 32) + 32 * 9 + 1
    ws2, bs2 = inputs.cnn_unflatten(flat)
    for a, b in zip(ws + bs, ws2 + bs2):
        assert np.array_equal(a, b)
