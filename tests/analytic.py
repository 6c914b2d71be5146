"""Closed-form solutions the oracle is pinned to (textbook fluid mechanics, not
the lattice Boltzmann method)."""
import math

import numpy as np


def taylor_green(n, u0, nu, t, ny=None):
    """Decaying Taylor-Green vortex (incompressible Navier-Stokes), with the
    initial state of ``inputs.taylor_green``: u decays as exp(-2 nu k^2 t)."""
    ny = n if ny is None else ny
    kx, ky = 2 * math.pi / n, 2 * math.pi / ny
    dec = math.exp(-nu * (kx * kx + ky * ky) * t)
    x = np.arange(n)[None, :].astype(float)
    y = np.arange(ny)[:, None].astype(float)
    cx, sx, cy, sy = np.cos(kx * x), np.sin(kx * x), np.cos(ky * y), np.sin(ky * y)
    ux = -u0 * cx * sy * dec
    uy = u0 * sx * cy * dec
    dxux = u0 * kx * sx * sy * dec
    dyux = -u0 * ky * cx * cy * dec
    dxuy = u0 * kx * cx * cy * dec
    dyuy = -u0 * ky * sx * sy * dec
    return dict(ux=ux, uy=uy, sxx=dxux, syy=dyuy, sxy=0.5 * (dxuy + dyux),
                omega=dxuy - dyux)


def diffusion_sine(n, amp, D, t):
    """phi = 1 + amp sin(kx) sin(ky) exp(-2 D k^2 t) (pure diffusion)."""
    k = 2 * math.pi / n
    x = np.arange(n)[None, :].astype(float)
    y = np.arange(n)[:, None].astype(float)
    return 1.0 + amp * np.sin(k * x) * np.sin(k * y) * math.exp(-2 * D * k * k * t)


def laplace_lid(n, terms=401):
    """Steady diffusion in a square with phi = 1 on the top wall and 0 on the
    other three (separation of variables).  Walls sit half-way between nodes, so
    node (i, j) is at X = i + 1/2, Y = j + 1/2 in a box of side L = n."""
    X = (np.arange(n) + 0.5)[None, :] / n
    Y = (np.arange(n) + 0.5)[:, None] / n
    phi = np.zeros((n, n))
    for m in range(1, terms + 1, 2):
        a = m * math.pi
        # sinh(a Y)/sinh(a) written with exponentials that stay finite
        ratio = np.exp(a * (Y - 1.0)) * (1 - np.exp(-2 * a * Y)) / (1 - math.exp(-2 * a))
        phi += 4.0 / a * np.sin(a * X) * ratio
    return phi


def rel_l2(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))
