"""Pins of the FP64 network oracle: hand-written gradients against central
finite differences on a tiny instance, and the layer adjoints against their
definition <A x, y> = <x, A^T y> (no GPU)."""
import numpy as np
import pytest

from oracle import unet as U


def tiny(seed=0):
    P = U.init_params(c=4, cin=3, cout=2, seed=seed)
    r = np.random.default_rng(seed + 10)
    x = r.standard_normal((2, 8, 8, 3))
    t = r.standard_normal((2, 8, 8, 2))
    return P, x, t


def total_loss(P, x, t):
    out, _ = U.forward(P, x)
    return U.loss(out, t)


@pytest.mark.parametrize("name", ["e1a", "e2b", "b1", "d3a", "d2b", "d1a", "head"])
def test_gradients_match_finite_differences(name):
    P, x, t = tiny()
    out, a = U.forward(P, x)
    G = U.backward(P, a, out, t)
    r = np.random.default_rng(3)
    for which in (0, 1):  # weight, bias
        arr = P[name][which]
        for _ in range(4):
            idx = tuple(r.integers(0, s) for s in arr.shape)
            h = 1e-6
            old = arr[idx]
            arr[idx] = old + h
            lp = total_loss(P, x, t)
            arr[idx] = old - h
            lm = total_loss(P, x, t)
            arr[idx] = old
            fd = (lp - lm) / (2 * h)
            an = G[name][which][idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (name, which, idx, fd, an)


def test_layer_adjoints():
    r = np.random.default_rng(1)
    x = r.standard_normal((2, 8, 6, 3))
    # pool / pool_bwd and up / up_bwd are adjoint pairs
    y = r.standard_normal((2, 4, 3, 3))
    assert np.isclose(np.sum(U.pool(x) * y), np.sum(x * U.pool_bwd(y)))
    z = r.standard_normal((2, 8, 6, 3))
    assert np.isclose(np.sum(U.up(y) * z), np.sum(y * U.up_bwd(z)))
    # conv: d/dx of <conv(x), dy> equals conv_bwd's dx
    W = r.standard_normal((5, 3, 3, 3))
    dy = r.standard_normal((2, 8, 6, 5))
    dx, dW, db = U.conv_bwd(x, W, dy)
    lin = lambda xx: np.sum((U.conv(xx, W, np.zeros(5))) * dy)
    assert np.isclose(lin(x), np.sum(x * dx))
    assert np.isclose(np.sum(U.conv(x, W, np.zeros(5)) * dy), np.sum(W * dW))


def test_conv_matches_direct_sum():
    """The shifted-product convolution equals the textbook zero-padded sum."""
    r = np.random.default_rng(2)
    x = r.standard_normal((1, 5, 4, 2))
    W = r.standard_normal((3, 3, 3, 2))
    b = r.standard_normal(3)
    y = U.conv(x, W, b)
    for (h, w, o) in [(0, 0, 0), (2, 3, 1), (4, 1, 2)]:
        s = b[o]
        for kh in range(3):
            for kw in range(3):
                hh, ww = h + kh - 1, w + kw - 1
                if 0 <= hh < 5 and 0 <= ww < 4:
                    s += W[o, kh, kw] @ x[0, hh, ww]
        assert np.isclose(y[0, h, w, o], s)
