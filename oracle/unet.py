"""FP64 CPU oracle of the warm-start surrogate network (a small U-Net).

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): it checks the
GPU network kernels' forward pass and gradients.  Plain numpy in float64:
3x3 convolutions as shifted matrix products, leaky ReLU (slope 0.02), 2x2
average pooling, nearest 2x upsampling, channel concatenation, a 1x1 head and
a mean-squared-error loss; the backward pass is written out by hand, layer by
layer (pinned against central finite differences in the tests).

Architecture (channel widths c, 2c, 4c; ``cin`` input planes, ``cout`` outputs):
  e1a cin->c, e1b c->c | pool | e2a c->2c, e2b 2c->2c | pool | e3a 2c->4c,
  e3b 4c->4c | pool | b1 4c->4c, b2 4c->4c | up, concat e3b | d3a 8c->4c,
  d3b 4c->2c | up, concat e2b | d2a 4c->2c, d2b 2c->c | up, concat e1b |
  d1a 2c->c, d1b c->c | head 1x1 c->cout (no activation)
Weights are W[Co][3][3][Ci] (head: W[Co][Ci]), biases b[Co].
"""
from __future__ import annotations

import numpy as np

SLOPE = 0.02


def layer_specs(c: int, cin: int, cout: int):
    """(name, input channels, output channels) of every convolution in order."""
    return [("e1a", cin, c), ("e1b", c, c), ("e2a", c, 2 * c), ("e2b", 2 * c, 2 * c),
            ("e3a", 2 * c, 4 * c), ("e3b", 4 * c, 4 * c), ("b1", 4 * c, 4 * c),
            ("b2", 4 * c, 4 * c), ("d3a", 8 * c, 4 * c), ("d3b", 4 * c, 2 * c),
            ("d2a", 4 * c, 2 * c), ("d2b", 2 * c, c), ("d1a", 2 * c, c), ("d1b", c, c),
            ("head", c, cout)]


def init_params(c, cin, cout, seed=0):
    r = np.random.default_rng(seed)
    P = {}
    for name, ci, co in layer_specs(c, cin, cout):
        if name == "head":
            P[name] = (r.standard_normal((co, ci)) * np.sqrt(1.0 / ci), np.zeros(co))
        else:
            P[name] = (r.standard_normal((co, 3, 3, ci)) * np.sqrt(2.0 / (9 * ci)),
                       0.01 * r.standard_normal(co))
    return P


# ---------------------------------------------------------------- layers
def conv(x, W, b):
    B, H, Wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((B, H, Wd, W.shape[0])) + b
    for kh in range(3):
        for kw in range(3):
            y += xp[:, kh:kh + H, kw:kw + Wd, :] @ W[:, kh, kw, :].T
    return y


def conv_bwd(x, W, dy):
    B, H, Wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for kh in range(3):
        for kw in range(3):
            dW[:, kh, kw, :] = np.einsum("bhwo,bhwi->oi", dy, xp[:, kh:kh + H, kw:kw + Wd, :])
            dxp[:, kh:kh + H, kw:kw + Wd, :] += dy @ W[:, kh, kw, :]
    return dxp[:, 1:-1, 1:-1, :], dW, dy.sum(axis=(0, 1, 2))


def act(z):
    return np.where(z > 0, z, SLOPE * z)


def act_bwd(dy, y):
    return np.where(y > 0, dy, SLOPE * dy)


def pool(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_bwd(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_bwd(dy):
    B, H, W, C = dy.shape
    return dy.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


# ---------------------------------------------------------------- network
def forward(P, x):
    """Returns (output, cache of activations)."""
    a = {"x": x}
    def cv(name, inp):
        W, b = P[name]
        y = act(conv(inp, W, b))
        a[name] = y
        return y
    e1 = cv("e1b", cv("e1a", x))
    e2 = cv("e2b", cv("e2a", pool(e1)))
    e3 = cv("e3b", cv("e3a", pool(e2)))
    bt = cv("b2", cv("b1", pool(e3)))
    a["cat3"] = np.concatenate([up(bt), e3], axis=-1)
    d3 = cv("d3b", cv("d3a", a["cat3"]))
    a["cat2"] = np.concatenate([up(d3), e2], axis=-1)
    d2 = cv("d2b", cv("d2a", a["cat2"]))
    a["cat1"] = np.concatenate([up(d2), e1], axis=-1)
    d1 = cv("d1b", cv("d1a", a["cat1"]))
    W, b = P["head"]
    out = d1 @ W.T + b
    return out, a


def loss(out, target):
    return float(np.mean((out - target) ** 2))


def backward(P, a, out, target):
    """Gradients of the mean-squared error w.r.t. every parameter."""
    G = {}
    g = 2.0 * (out - target) / out.size
    W, _ = P["head"]
    G["head"] = (np.einsum("bhwo,bhwi->oi", g, a["d1b"]), g.sum(axis=(0, 1, 2)))
    g = g @ W

    def cvb(name, inp, dy):
        W, _ = P[name]
        dz = act_bwd(dy, a[name])
        dx, dW, db = conv_bwd(inp, W, dz)
        G[name] = (dW, db)
        return dx

    g = cvb("d1a", a["cat1"], cvb("d1b", a["d1a"], g))
    c1 = a["e1b"].shape[-1]
    g_up1, g_e1 = g[..., :-c1], g[..., -c1:]
    g = cvb("d2a", a["cat2"], cvb("d2b", a["d2a"], up_bwd(g_up1)))
    c2 = a["e2b"].shape[-1]
    g_up2, g_e2 = g[..., :-c2], g[..., -c2:]
    g = cvb("d3a", a["cat3"], cvb("d3b", a["d3a"], up_bwd(g_up2)))
    c3 = a["e3b"].shape[-1]
    g_up3, g_e3 = g[..., :-c3], g[..., -c3:]
    g = cvb("b1", pool(a["e3b"]), cvb("b2", a["b1"], up_bwd(g_up3)))
    g = cvb("e3a", pool(a["e2b"]), cvb("e3b", a["e3a"], g_e3 + pool_bwd(g)))
    g = cvb("e2a", pool(a["e1b"]), cvb("e2b", a["e2a"], g_e2 + pool_bwd(g)))
    cvb("e1a", a["x"], cvb("e1b", a["e1a"], g_e1 + pool_bwd(g)))
    return G
