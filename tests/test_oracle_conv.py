"""Pins of the FP64 network reference (oracle/conv_ref.py) against things it
does not compute itself: scipy's circular correlation, brute-force loops,
central finite differences, and closed forms of the Adam update."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import conv_ref as cr


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("dil", [1, 2, 3])
def test_conv_matches_scipy_circular_correlation(dil):
    x = _rand((2, 7, 9, 3), 1)
    w = _rand((4, 9, 3), 2)
    b = _rand(4, 3)
    y = cr.conv3x3(x, w, b, dil)
    for bb in range(2):
        for co in range(4):
            ref = np.full((7, 9), b[co])
            for ci in range(3):
                k = np.zeros((2 * dil + 1, 2 * dil + 1))
                for tap in range(9):
                    ky, kx = divmod(tap, 3)
                    k[ky * dil, kx * dil] = w[co, tap, ci]
                ref += ndimage.correlate(x[bb, :, :, ci], k, mode="wrap")
            assert np.allclose(y[bb, :, :, co], ref, rtol=1e-13, atol=1e-13)


def test_conv_matches_brute_force_loops_with_wraparound():
    # dilation larger than the image: offsets wrap more than once
    x = _rand((1, 3, 4, 2), 4)
    w = _rand((2, 9, 2), 5)
    dil = 5
    y = cr.conv3x3(x, w, None, dil)
    H, W = 3, 4
    for i in range(H):
        for j in range(W):
            for co in range(2):
                s = 0.0
                for ky in range(3):
                    for kx in range(3):
                        for ci in range(2):
                            s += x[0, (i + (ky - 1) * dil) % H, (j + (kx - 1) * dil) % W, ci] * w[co, 3 * ky + kx, ci]
                assert abs(y[0, i, j, co] - s) < 1e-13


def _fd(f, a, idx, eps=1e-6):
    a1 = a.copy()
    a1[idx] += eps
    a2 = a.copy()
    a2[idx] -= eps
    return (f(a1) - f(a2)) / (2 * eps)


@pytest.mark.parametrize("dil", [1, 2])
def test_conv_gradients_match_finite_differences(dil):
    x = _rand((2, 4, 5, 3), 6)
    w = _rand((2, 9, 3), 7)
    b = _rand(2, 8)
    g = _rand((2, 4, 5, 2), 9)
    dx, dw, db = cr.conv3x3_backward(x, w, g, dil)
    rng = np.random.default_rng(10)
    for _ in range(12):
        idx = tuple(int(rng.integers(0, n)) for n in x.shape)
        assert abs(_fd(lambda a: np.sum(g * cr.conv3x3(a, w, b, dil)), x, idx) - dx[idx]) < 1e-7
        idw = tuple(int(rng.integers(0, n)) for n in w.shape)
        assert abs(_fd(lambda a: np.sum(g * cr.conv3x3(x, a, b, dil)), w, idw) - dw[idw]) < 1e-7
    for c in range(2):
        assert abs(_fd(lambda a: np.sum(g * cr.conv3x3(x, w, a, dil)), b, (c,)) - db[c]) < 1e-7


@pytest.mark.parametrize("relu", [True, False])
def test_network_gradients_match_finite_differences(relu):
    dils = (1, 2, 1)
    chans = [3, 4, 4, 2]
    rng = np.random.default_rng(11)
    params = [(rng.standard_normal((chans[i + 1], 9, chans[i])) * 0.4, rng.standard_normal(chans[i + 1]) * 0.1)
              for i in range(3)]
    x = rng.standard_normal((1, 5, 6, 3))
    t = rng.standard_normal((1, 5, 6, 2))
    wch = np.array([1.0, 0.25])

    def loss_of(ps):
        return cr.weighted_mse(cr.net_forward(x, ps, dils, relu)[-1], t, wch, 0.5)[0]

    acts = cr.net_forward(x, params, dils, relu)
    _, dy = cr.weighted_mse(acts[-1], t, wch, 0.5)
    grads = cr.net_backward(x, params, dils, acts, dy, relu)
    for li in range(3):
        for k in range(6):
            idx = tuple(int(rng.integers(0, n)) for n in params[li][0].shape)

            def f(a, li=li):
                ps = list(params)
                ps[li] = (a, params[li][1])
                return loss_of(ps)

            assert abs(_fd(f, params[li][0], idx) - grads[li][0][idx]) < 1e-6 * max(1.0, abs(grads[li][0][idx]))
        for c in range(chans[li + 1]):

            def fb(a, li=li):
                ps = list(params)
                ps[li] = (params[li][0], a)
                return loss_of(ps)

            assert abs(_fd(fb, params[li][1], (c,)) - grads[li][1][c]) < 1e-6 * max(1.0, abs(grads[li][1][c]))


def test_weighted_mse_closed_form():
    y = np.array([[1.0, 2.0], [3.0, 5.0]])
    t = np.array([[0.0, 2.0], [1.0, 1.0]])
    loss, dy = cr.weighted_mse(y, t, np.array([2.0, 0.5]), 0.25)
    assert loss == pytest.approx(0.25 * (2 * 1 + 0 + 2 * 4 + 0.5 * 16))
    assert np.allclose(dy, 0.5 * np.array([[2.0, 0.0], [4.0, 2.0]]))


def test_adam_constant_gradient_moves_by_lr_every_step():
    # with m = v = 0 initially and a constant gradient the bias-corrected
    # moments equal g and g^2 at every step: each step is lr * g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3])
    p = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    lr, eps = 0.01, 1e-8
    for t in range(1, 6):
        p, m, v = cr.adam_step(p, g, m, v, lr, 0.9, 0.999, eps, t)
        assert np.allclose(p, -t * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)
