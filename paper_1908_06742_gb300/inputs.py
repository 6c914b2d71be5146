"""Seeded synthetic workloads (initial macroscopic fields and parameter draws).

This module holds no arithmetic of the lattice Boltzmann method: it only lays
out the initial velocity, density, scalar and gradient fields of the benchmark
flows, and draws the parameters of batched instances from a seeded generator.
Both the CUDA path and its CPU checker consume what it produces.

Coordinates: node (i, j) sits at x = i, y = j (lattice units).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Fields:
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    phi: np.ndarray
    grads: np.ndarray  # (6, ny, nx): dxux, dyux, dxuy, dyuy, dxphi, dyphi


def taylor_green(n: int, u0: float = 0.01, phi_amp: float = 0.1, rho0: float = 1.0,
                 cs2: float = 1.0 / 3.0, ny: int | None = None, window=None,
                 xp=np, device=None) -> Fields:
    """Decaying Taylor-Green vortex at t = 0 on a periodic n x n grid.

    u_x = -u0 cos(kx) sin(ky), u_y = u0 sin(kx) cos(ky), k = 2 pi / n,
    pressure p = -rho0 u0^2 / 4 (cos 2kx + cos 2ky), rho = rho0 + p / c_s^2,
    scalar phi = 1 + phi_amp sin(kx) sin(ky).  Exact gradients are returned for
    the Chapman-Enskog initialisation of the populations.

    ``window = (x0, y0, w, h)`` returns only that sub-rectangle of the grid
    (indices taken modulo the period); ``xp = torch`` with ``device`` builds the
    fields directly in device memory (float64), for grids too large for the host.
    """
    ny = n if ny is None else ny
    kx = 2.0 * math.pi / n
    ky = 2.0 * math.pi / ny
    x0, y0, w, h = window if window is not None else (0, 0, n, ny)
    if xp is np:
        xs = (np.arange(w, dtype=np.int64) + x0) % n
        ys = (np.arange(h, dtype=np.int64) + y0) % ny
        x = xs.astype(np.float64)[None, :]
        y = ys.astype(np.float64)[:, None]
    else:
        xs = (xp.arange(w, dtype=xp.int64, device=device) + x0) % n
        ys = (xp.arange(h, dtype=xp.int64, device=device) + y0) % ny
        x = xs.to(xp.float64)[None, :]
        y = ys.to(xp.float64)[:, None]
    cx, sx = xp.cos(kx * x), xp.sin(kx * x)
    cy, sy = xp.cos(ky * y), xp.sin(ky * y)
    ux = -u0 * cx * sy
    uy = u0 * sx * cy
    p = -rho0 * u0 * u0 / 4.0 * (xp.cos(2 * kx * x) + xp.cos(2 * ky * y))
    rho = rho0 + p / cs2
    phi = 1.0 + phi_amp * sx * sy
    grads = xp.stack([
        u0 * kx * sx * sy,             # d_x u_x
        -u0 * ky * cx * cy,            # d_y u_x
        u0 * kx * cx * cy,             # d_x u_y
        -u0 * ky * sx * sy,            # d_y u_y
        phi_amp * kx * cx * sy,        # d_x phi
        phi_amp * ky * sx * cy,        # d_y phi
    ])
    if xp is np:
        b = lambda a: np.ascontiguousarray(np.broadcast_to(a, (h, w)), np.float64)
        return Fields(b(rho), b(ux), b(uy), b(phi), np.ascontiguousarray(grads, np.float64))
    b = lambda a: xp.broadcast_to(a, (h, w)).contiguous()
    return Fields(b(rho), b(ux), b(uy), b(phi), grads.contiguous())


def rest(nx: int, ny: int, rho0: float = 1.0, phi: float = 0.0) -> Fields:
    """Fluid at rest with uniform scalar (lid-driven cavity start)."""
    z = np.zeros((ny, nx))
    return Fields(np.full((ny, nx), rho0), z.copy(), z.copy(), np.full((ny, nx), phi),
                  np.zeros((6, ny, nx)))


def uniform_advection(n: int, u: float = 0.02, v: float = 0.0, phi_amp: float = 0.1) -> Fields:
    """Uniform translation (u, v) of a sine scalar on a periodic grid: zero
    velocity gradient, nonzero scalar gradient."""
    k = 2.0 * math.pi / n
    x = np.arange(n, dtype=np.float64)[None, :]
    y = np.arange(n, dtype=np.float64)[:, None]
    phi = 1.0 + phi_amp * np.sin(k * x) * np.sin(k * y)
    grads = np.zeros((6, n, n))
    grads[4] = phi_amp * k * np.cos(k * x) * np.sin(k * y)
    grads[5] = phi_amp * k * np.sin(k * x) * np.cos(k * y)
    return Fields(np.ones((n, n)), np.full((n, n), u), np.full((n, n), v), phi, grads)


def random_state(nx: int, ny: int, seed: int, amp: float = 0.01):
    """Random smooth-free perturbation fields (rho, ux, uy, phi) for parity of
    the raw step on arbitrary data (no physical meaning)."""
    r = np.random.default_rng(seed)
    rho = 1.0 + amp * r.standard_normal((ny, nx))
    ux = amp * r.standard_normal((ny, nx))
    uy = amp * r.standard_normal((ny, nx))
    phi = 1.0 + 10 * amp * r.standard_normal((ny, nx))
    grads = amp * 0.1 * r.standard_normal((6, ny, nx))
    return Fields(rho, ux, uy, phi, grads)


CAVITY_SIZES = (64, 96, 128, 192, 256, 384, 512)


def cavity_batch(n_inst: int = 512, seed: int = 0, re_lo: float = 100.0, re_hi: float = 3200.0,
                 sizes=CAVITY_SIZES):
    """Independent lid-driven cavities: size uniform over ``sizes``, Reynolds
    number log-uniform in [re_lo, re_hi], Peclet = Reynolds."""
    r = np.random.default_rng(seed)
    n = r.choice(np.asarray(sizes), size=n_inst)
    re = np.exp(r.uniform(math.log(re_lo), math.log(re_hi), size=n_inst))
    return [dict(n=int(n[i]), re=float(re[i]), pe=float(re[i])) for i in range(n_inst)]


def sine_waves(n: int, a: float = 0.01, b: float = 0.008, c: float = 0.004, d: float = -0.003,
               phi_amp: float = 0.0) -> Fields:
    """Smooth periodic velocity with every gradient component nonzero:
    u_x = a sin(ky) + c sin(kx), u_y = b sin(kx) + d sin(ky), k = 2 pi / n
    (shear from a, b; divergence from c, d), rho = 1,
    phi = 1 + phi_amp sin(kx) sin(ky), with the exact gradients."""
    k = 2.0 * math.pi / n
    x = np.arange(n, dtype=np.float64)[None, :]
    y = np.arange(n, dtype=np.float64)[:, None]
    sx, cx, sy, cy = np.sin(k * x), np.cos(k * x), np.sin(k * y), np.cos(k * y)
    b2 = lambda v: np.ascontiguousarray(np.broadcast_to(v, (n, n)), np.float64)
    ux = b2(a * sy + c * sx)
    uy = b2(b * sx + d * sy)
    phi = b2(1.0 + phi_amp * sx * sy)
    grads = np.stack([b2(c * k * cx), b2(a * k * cy), b2(b * k * cx), b2(d * k * cy),
                      b2(phi_amp * k * cx * sy), b2(phi_amp * k * sx * cy)])
    return Fields(np.ones((n, n)), ux, uy, phi, grads)
