"""Pins of the conv-net oracle: a library correlation and central finite differences (P10)."""
import numpy as np
import pytest
from scipy import signal

from oracle import convnet


def test_conv3d_equals_library_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 5, 6, 7))
    w = rng.standard_normal((2, 3, 3, 3, 3))
    y = convnet.conv3d(x, w)
    for o in range(2):
        ref = sum(signal.correlate(x[i], w[o, i], mode="same", method="direct") for i in range(3))
        assert np.max(np.abs(y[o] - ref)) < 1e-12


def _loss(ws, x, g):
    return float(np.sum(convnet.forward(x, ws)[-1] * g))


@pytest.mark.parametrize("seed", [1, 2])
def test_gradients_vs_finite_differences(seed):
    rng = np.random.default_rng(seed)
    ws = convnet.init_weights(seed)
    x = rng.standard_normal((8, 4, 5, 6))
    g = rng.standard_normal((8, 4, 5, 6))
    acts = convnet.forward(x, ws)
    gws, gx = convnet.backward(acts, ws, g)
    eps = 1e-6
    for l in range(4):
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in ws[l].shape)
            wp = [w.copy() for w in ws]
            wm = [w.copy() for w in ws]
            wp[l][idx] += eps
            wm[l][idx] -= eps
            fd = (_loss(wp, x, g) - _loss(wm, x, g)) / (2 * eps)
            assert abs(fd - gws[l][idx]) <= 1e-6 * max(1.0, abs(fd))
    for _ in range(6):
        idx = tuple(rng.integers(0, s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += eps
        xm[idx] -= eps
        fd = (_loss(ws, xp, g) - _loss(ws, xm, g)) / (2 * eps)
        assert abs(fd - gx[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_positive_homogeneity():
    rng = np.random.default_rng(5)
    ws = convnet.init_weights(5)
    x = rng.standard_normal((8, 3, 4, 5))
    a = convnet.forward(x, ws)[-1]
    b = convnet.forward(3.7 * x, ws)[-1]
    assert np.max(np.abs(b - 3.7 * a)) < 1e-12 * np.max(np.abs(b))
