"""The paper's own forced validation flows (Sec. 5.1-5.3), run on the GPU at
the paper's parameters and compared with the analytic solutions, as the paper
does.  These check the method end to end (FP32 CUDA path); the oracle parity
of the same code lives in test_gpu_forcing.py.  Measured values are quoted in
each docstring; bounds leave a margin above them."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1908_06742_gb300 import build as B
from paper_1908_06742_gb300 import ddflb as D
from tests import analytic as A

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    D.load()


def f64(g):
    return {k: v.double().cpu().numpy() for k, v in g.fields().items()}


def channel_config(H, tau, **kw):
    # higher-order rates unity, tau^phi = 0.57, phi = 1 (bottom) / 2 (top) (Sec. 5.1)
    w = 1.0 / tau
    return D.Config(nx=3, ny=H, bc="channel", omega_f=(0, 0, 0, 1.0, w, w, 1.0, 1.0, 1.0),
                    omega_g=(0, 1 / 0.57, 1 / 0.57, 1, 1, 1, 1, 1, 1), phi_wall=1.0,
                    phi_lid=2.0, u_lid=0.0, **kw)


@pytest.mark.parametrize("umax", [0.01, 0.03, 0.05, 0.08])
def test_poiseuille_paper_set(umax):
    """Sec. 5.1: 3 x 151 channel, F_x = 3e-6, U_max set through nu =
    F H^2 / (8 U_max), from rest for 1.5 H^2/nu steps.  The velocity is parabolic
    and omega linear across the channel (interior rows: the first row at each
    wall sits outside the bulk relations)."""
    H, F = 151, 3e-6
    nu = F * H * H / (8 * umax)
    tau = 3 * nu + 0.5
    g = D.Lattice(channel_config(H, tau, fx=F))
    z = np.zeros((H, 3))
    g.init(np.ones((H, 3)), z, z, np.full((H, 3), 1.5))
    g.step(int(1.5 * H * H / nu))
    f = f64(g)
    ua, oa = A.poiseuille(H, F, nu)
    eu = A.rel_l2(f["ux"][:, 1], ua)
    eo = A.rel_l2(f["omega"][1:-1, 1], oa[1:-1])
    print(f"poiseuille U_max {umax}: E_u {eu:.2e} E_omega {eo:.2e}")
    assert abs(ua.max() - umax) < 1e-3 * umax
    assert eu < 2e-3 and eo < 2e-2


def four_rolls_run(N, u0, nu_lb, efolds=14.0, omega_hi=1.0):
    a = A.four_rolls(N, u0, nu_lb)
    w = 1.0 / (3 * nu_lb + 0.5)
    cfg = D.Config(nx=N, ny=N, omega_f=(0, 0, 0, omega_hi, w, w, omega_hi, omega_hi, omega_hi),
                   omega_g=(0, 1 / 0.57, 1 / 0.57) + (omega_hi,) * 6)
    g = D.Lattice(cfg).set_force_field(a["force"])
    z = np.zeros((N, N))
    g.init(np.ones((N, N)), z, z, np.full((N, N), 2.0))
    k = 2 * math.pi / N
    g.step(int(efolds / (2 * nu_lb * k * k)))
    f = f64(g)
    e_om = math.sqrt(np.sum((f["omega"] - a["omega"]) ** 2) / np.sum(a["omega"] ** 2))
    return A.rel_l2(f["ux"], a["ux"]), e_om


def test_four_rolls_mill_re40():
    """Sec. 5.2: 84 x 84, u0 = 0.035, Re = 2 pi u0 / nu = 40 (nu in box units,
    dx = 2 pi / N; lattice nu = u0 N / Re), uniform phi = 2, tau^phi = 0.57,
    started from rest.  Measured E_u, E_omega recorded in the printout."""
    N, u0 = 84, 0.035
    eu, eo = four_rolls_run(N, u0, u0 * N / 40.0)
    print(f"four-rolls Re 40: E_u {eu:.2e} E_omega {eo:.2e}")
    assert eu < 5e-3 and eo < 1e-2


@pytest.mark.parametrize("u0,min_slope", [(0.045, 1.3), (0.0045, 1.8)])
def test_four_rolls_mill_convergence(u0, min_slope):
    """Sec. 5.2.1: fixed nu = 0.00218 (box units, so the lattice nu grows with
    N), N = 24, 48, 96, 192; E_g,omega of Eq. (sca).  The paper reports slope
    -2.0 at u0 = 0.045.  Measured here: at u0 = 0.045, E_omega = 8.2e-2,
    2.7e-2, 1.0e-2, 3.9e-3 (fitted slope -1.46) while E_u stalls at 6e-4 and
    phi varies by 1.2e-2 at every N: with dt = dx the lattice Mach number stays
    fixed, so the O(Ma^2) compressibility error does not shrink, and through
    the scalar gradient terms of Sec. 4 it adds a first-order part to the omega
    error.  At u0 = 0.0045 (Mach number / 10) the same sweep gives E_omega =
    7.6e-2, 1.9e-2, 4.5e-3, 1.4e-3 (slope -1.93)."""
    nu = 0.00218
    errs = []
    for N in (24, 48, 96, 192):
        nu_lb = nu * N / (2 * math.pi)
        eu, eo = four_rolls_run(N, u0, nu_lb)
        errs.append(eo)
        print(f"convergence u0 {u0} N {N}: nu_lb {nu_lb:.4f} E_u {eu:.2e} E_omega {eo:.2e}")
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    slope = -np.polyfit(np.log([24, 48, 96, 192]), np.log(errs), 1)[0]
    print("orders", orders, "fitted slope", -slope)
    assert all(errs[i + 1] < errs[i] for i in range(3))
    assert min_slope <= slope <= 2.5, (errs, orders)


def test_four_rolls_mill_convergence_diffusive_scaling():
    """Sec. 5.2.1 read with diffusive scaling: the study fixes nu = 0.00218 and
    u0 = 0.045 in the 2 pi box but (unlike the Re 40 case) does not state the
    time step; with dt = dx^2 the lattice viscosity is 0.00218 at every N and
    the lattice velocity u0 2 pi / N falls with N, so Re = 2 pi u0 / nu = 130
    as in the dt = dx reading while the Mach number falls with the grid.  This
    reading reproduces the paper's second order: E_omega = 7.2e-2, 1.86e-2,
    4.5e-3, 1.4e-3 over N = 24 ... 192, fitted slope -1.90 (the paper: -2.0).
    The dt = dx reading (test above) keeps the Mach number and stalls at
    -1.46; nu = 0.00218 in lattice units with u0 = 0.045 in lattice units is
    Re 500-4000, where the four-rolls state does not hold (E_u ~ 1 at N = 192)."""
    nu, u0 = 0.00218, 0.045
    errs = []
    for N in (24, 48, 96, 192):
        eu, eo = four_rolls_run(N, u0 * 2 * math.pi / N, nu)
        errs.append(eo)
        print(f"diffusive N {N}: u_lb {u0 * 2 * math.pi / N:.5f} E_u {eu:.2e} E_omega {eo:.2e}")
    slope = -np.polyfit(np.log([24, 48, 96, 192]), np.log(errs), 1)[0]
    print("fitted slope", -slope)
    assert all(errs[i + 1] < errs[i] for i in range(3))
    assert 1.8 <= slope <= 2.2, errs


@pytest.mark.parametrize("tau,bound_om", [(0.781, 4e-2), (0.596, 2e-1)])
def test_womersley_paper_set(tau, bound_om):
    """Sec. 5.3: 3 x 101, F = 1e-5 cos(2 pi t / T), T = 10000, tau = 0.781
    (Wo 4.1) and 0.596 (Wo 7.1).  Started from the analytic profile at t = 0
    (with its Chapman-Enskog gradients; from rest the slowest viscous mode,
    exp(-pi^2 nu t / H^2), would still hold 7% after three periods), one
    period, then 8 phases of the next compared with the analytic u and omega
    (rows away from the walls)."""
    T, Fm, H = 10000, 1e-5, 101
    Om = 2 * math.pi / T
    nu = (tau - 0.5) / 3
    g = D.Lattice(channel_config(H, tau, fx=Fm, force_omega=Om))
    y = np.arange(H) + 0.5
    u0, om0 = A.womersley(H, Fm, Om, nu, 0.0)
    grads = np.zeros((6, H, 3))
    grads[1] = np.repeat(-om0[:, None], 3, axis=1)     # d_y u_x
    grads[5] = 1.0 / H                                 # d_y phi
    g.init(np.ones((H, 3)), np.repeat(u0[:, None], 3, axis=1), np.zeros((H, 3)),
           np.repeat((1.0 + y / H)[:, None], 3, axis=1), grads)
    g.step(T)
    eu, eo = [], []
    for k in range(8):
        f = f64(g)
        ua, oa = A.womersley(H, Fm, Om, nu, T + k * (T // 8))
        eu.append(np.linalg.norm(f["ux"][:, 1] - ua) / np.linalg.norm(ua))
        eo.append(np.linalg.norm(f["omega"][4:-4, 1] - oa[4:-4]) / np.linalg.norm(oa[4:-4]))
        g.step(T // 8)
    print(f"womersley tau {tau}: max E_u {max(eu):.2e} max E_omega {max(eo):.2e}")
    assert max(eu) < 1e-2 and max(eo) < bound_om
