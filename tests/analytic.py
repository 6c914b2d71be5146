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
                omega=dxuy - dyux, dxux=dxux, dyux=dyux, dxuy=dxuy, dyuy=dyuy)


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


def poiseuille(H, F, nu, rho=1.0):
    """Steady plane Poiseuille flow between half-way walls at y = -1/2 and
    H - 1/2 driven by a body force F: u_x(j), and omega_z = -d u_x / dy."""
    y = np.arange(H) + 0.5
    ux = F / (2 * rho * nu) * y * (H - y)
    om = -F / (2 * rho * nu) * (H - 2 * y)
    return ux, om


def four_rolls(n, u0, nu, rho=1.0):
    """Steady four-rolls mill on a periodic n x n grid (k = 2 pi / n): the body
    force F = 2 rho nu k^2 u0 (sin kx sin ky, cos kx cos ky) sustains
    u = u0 (sin kx sin ky, cos kx cos ky), omega = -2 u0 k sin kx cos ky."""
    k = 2 * math.pi / n
    x = np.arange(n)[None, :].astype(float)
    y = np.arange(n)[:, None].astype(float)
    sx, cx, sy, cy = np.sin(k * x), np.cos(k * x), np.sin(k * y), np.cos(k * y)
    ux, uy = u0 * sx * sy, u0 * cx * cy
    force = np.stack([2 * rho * nu * k * k * ux, 2 * rho * nu * k * k * uy])
    return dict(ux=ux, uy=uy, omega=-2 * u0 * k * sx * cy, force=force)


def womersley(H, Fm, Omega, nu, t, rho=1.0):
    """Channel flow driven by F_x = Fm cos(Omega t) between walls at distance
    H (half-way walls): u = Re{ Fm/(i Omega rho) [1 - cosh(kappa eta)/cosh(kappa L)] e^{i Omega t} },
    kappa = sqrt(i Omega / nu), eta the distance from the centre line, L = H/2;
    omega_z = -du/dy."""
    eta = np.arange(H) + 0.5 - H / 2
    L = H / 2
    kap = np.sqrt(1j * Omega / nu)
    amp = Fm / (1j * Omega * rho)
    e = np.exp(1j * Omega * t)
    u = np.real(amp * (1 - np.cosh(kap * eta) / np.cosh(kap * L)) * e)
    om = np.real(amp * kap * np.sinh(kap * eta) / np.cosh(kap * L) * e)
    return u, om


def rel_l2(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))
