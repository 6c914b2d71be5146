"""Pins of the oracle's time stepping and local kinematics against closed forms,
conservation laws, symmetries and brute force (no GPU).

Measured values at the time of writing are quoted next to each bound.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1908_06742_gb300 import inputs
from tests import analytic as A

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]


def tg_params(n, nu=0.01, D=None, **kw):
    D = nu if D is None else D
    base = dict(nx=n, ny=n, omega_nu=O.omega_from_diffusivity(nu), omega_bulk=1.2, omega_hi=1.2,
                omega_phi=O.omega_from_diffusivity(D), omega_phi_hi=1.2)
    base.update(kw)
    return O.OracleParams(**base)


def run_tg(n, u0, steps, nu=0.01, phi_amp=0.0, **kw):
    F = inputs.taylor_green(n, u0, phi_amp=phi_amp)
    L = O.OracleLattice(tg_params(n, nu, **kw)).init(F.rho, F.ux, F.uy, F.phi, F.grads)
    L.step(steps)
    return L


# ----------------------------------------------------------------- streaming
def test_pure_streaming_is_a_shift():
    """With all rates zero the collision is the identity and one step moves
    population a by e_a with periodic wrap (brute force with np.roll)."""
    r = np.random.default_rng(0)
    n = 7
    p = O.OracleParams(nx=n, ny=5, lam_override=(0,) * 9, lam_phi_override=(0,) * 9)
    f = 0.1 + r.random((9, 5, n)); g = 0.1 + r.random((9, 5, n))
    L = O.OracleLattice(p).set_state(f, g)
    L.step(1)
    for a in range(9):
        np.testing.assert_allclose(L.f[a], np.roll(f[a], (EY[a], EX[a]), axis=(0, 1)), rtol=1e-13)
        np.testing.assert_allclose(L.g[a], np.roll(g[a], (EY[a], EX[a]), axis=(0, 1)), rtol=1e-13)


def test_bounce_back_streaming_is_reversible():
    """Half-way bounce-back streaming is a permutation whose inverse is
    'reverse directions, stream, reverse again' (cavity walls, lid at rest)."""
    r = np.random.default_rng(1)
    n = 6
    p = O.OracleParams(nx=n, ny=n, bc="cavity", lam_override=(0,) * 9, lam_phi_override=(0,) * 9,
                       phi_wall=0.0, phi_lid=0.0)
    f = 0.1 + r.random((9, n, n)); g = 0.1 + r.random((9, n, n))
    L = O.OracleLattice(p).set_state(f, g)
    for _ in range(3):
        L.step(1)
    L.set_state(L.f[OPP].copy(), L.g[OPP].copy())
    for _ in range(3):
        L.step(1)
    np.testing.assert_allclose(L.f[OPP], f, rtol=1e-13)
    # anti-bounce-back with phi_w = 0 flips the sign at each wall hit: |g| returns
    np.testing.assert_allclose(np.abs(L.g[OPP]), g, rtol=1e-13)
    assert abs(L.f.sum() - f.sum()) < 1e-12


# -------------------------------------------------------------- conservation
def test_periodic_conservation():
    """Periodic Taylor-Green with a curved scalar: sum rho and sum phi constant
    over 1000 steps to round-off (measured 5e-13 on a sum of 4096)."""
    F = inputs.taylor_green(64, 0.01, phi_amp=0.1)
    L = O.OracleLattice(tg_params(64)).init(F.rho, F.ux, F.uy, F.phi, F.grads)
    s0 = L.sums(); L.step(1000); s1 = L.sums()
    assert abs(s1["mass"] - s0["mass"]) < 1e-10
    assert abs(s1["scalar"] - s0["scalar"]) < 1e-10


def test_cavity_mass_exact_with_moving_lid():
    """The lid's momentum term cancels pairwise at every top node, so total
    mass stays constant to round-off (measured 2e-13)."""
    n = 24
    p = tg_params(n, 0.05, bc="cavity", u_lid=0.1, phi_lid=1.0, phi_wall=0.0)
    F = inputs.rest(n, n)
    L = O.OracleLattice(p).init(F.rho, F.ux, F.uy, F.phi)
    m0 = L.sums()["mass"]; L.step(500)
    assert abs(L.sums()["mass"] - m0) < 1e-11
    assert np.abs(L.fields()["ux"]).max() > 1e-3  # the lid did drive the flow


def test_cavity_mirror_symmetry():
    """Reversing the lid velocity mirrors the flow: u_x(x) -> -u_x(L-x),
    u_y(x) -> u_y(L-x), phi(x) -> phi(L-x) (measured 4e-16)."""
    n = 20
    out = []
    for U in (0.1, -0.1):
        p = tg_params(n, 0.05, bc="cavity", u_lid=U, phi_lid=1.0, phi_wall=0.0)
        F = inputs.rest(n, n)
        out.append(O.OracleLattice(p).init(F.rho, F.ux, F.uy, F.phi).step(300).fields())
    a, b = out
    assert np.abs(a["ux"] + b["ux"][:, ::-1]).max() < 1e-14
    assert np.abs(a["uy"] - b["uy"][:, ::-1]).max() < 1e-14
    assert np.abs(a["phi"] - b["phi"][:, ::-1]).max() < 1e-14
    assert np.abs(a["ux"]).max() > 1e-3


# ------------------------------------------------------------ analytic flows
def test_taylor_green_velocity_and_vorticity():
    """64^2, U0 = 0.01, nu = 0.01, 1000 steps, uniform scalar: u and the local
    vorticity against the decaying Taylor-Green closed form.
    Measured: E_u = 3.2e-5, E_omega = 3.3e-3, E_S = 7.7e-4."""
    L = run_tg(64, 0.01, 1000)
    f = L.fields(); a = A.taylor_green(64, 0.01, 0.01, 1000)
    eu = math.sqrt(A.rel_l2(f["ux"], a["ux"]) ** 2 / 2 + A.rel_l2(f["uy"], a["uy"]) ** 2 / 2)
    assert eu < 6e-5
    assert A.rel_l2(f["omega"], a["omega"]) < 6e-3
    assert A.rel_l2(f["sxx"], a["sxx"]) < 1.5e-3
    assert A.rel_l2(f["syy"], a["syy"]) < 1.5e-3


@pytest.mark.slow
def test_taylor_green_second_order_convergence():
    """Diffusive scaling (U0 ~ 1/N, steps ~ N^2, nu fixed) over N = 32, 64, 128:
    velocity and local vorticity errors fall with order 2 (Sec. 5.2.1 reports a
    slope of -2.0 for E_g,omega).  Measured orders: u 1.9/2.0, omega 2.0/2.0."""
    eu, eo = [], []
    for n, u0, steps in ((32, 0.02, 250), (64, 0.01, 1000), (128, 0.005, 4000)):
        f = run_tg(n, u0, steps).fields(); a = A.taylor_green(n, u0, 0.01, steps)
        eu.append(A.rel_l2(f["ux"], a["ux"]))
        eo.append(A.rel_l2(f["omega"], a["omega"]))
    for e in (eu, eo):
        orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
        assert all(1.8 <= o <= 2.2 for o in orders), (e, orders)


def test_pure_diffusion_of_scalar():
    """U0 = 0: the scalar sine decays as exp(-2 D k^2 t) (pins D_phi of Sec. 3),
    with second-order convergence under diffusive scaling.
    Measured relative errors of the decaying part: 5.2e-3 (32^2), 1.3e-3 (64^2)."""
    errs = []
    for n, t in ((32, 200), (64, 800)):
        L = run_tg(n, 0.0, t, D=0.02, phi_amp=0.1)
        errs.append(A.rel_l2(L.fields()["phi"] - 1.0, A.diffusion_sine(n, 0.1, 0.02, t) - 1.0))
    assert errs[1] < 2e-3
    assert 1.8 < math.log2(errs[0] / errs[1]) < 2.2


def test_strain_rate_and_vorticity_match_central_differences():
    """Cell by cell, the local S_ij and omega agree with central differences of
    the oracle's own velocity (difference O(dx^2) + O(Ma^2)).  Measured 1.1e-3
    (S) and 4.7e-3 (omega) relative L2 at 64^2 after 300 steps."""
    L = run_tg(64, 0.01, 300)
    f = L.fields()
    cd = lambda a, ax: (np.roll(a, -1, ax) - np.roll(a, 1, ax)) / 2
    ux, uy = f["ux"], f["uy"]
    dxux, dyux, dxuy, dyuy = cd(ux, 1), cd(ux, 0), cd(uy, 1), cd(uy, 0)
    assert A.rel_l2(f["sxx"], dxux) < 3e-3
    assert A.rel_l2(f["syy"], dyuy) < 3e-3
    assert A.rel_l2(f["omega"], dxuy - dyux) < 1e-2
    # S_xy of this flow is zero to leading order; compare with the gradient scale
    assert np.sqrt(np.mean((f["sxy"] - 0.5 * (dxuy + dyux)) ** 2)) < 1e-3 * np.abs(dxuy).max()


def test_vorticity_independent_of_beta():
    """The recovered vorticity does not depend on the choice of beta2 beyond
    the truncation error (Sec. 4).  Measured spread 2.0e-3 relative."""
    om = [run_tg(48, 0.01, 400, beta2=b2).fields()["omega"] for b2 in (0.8, 0.9, 0.95)]
    assert A.rel_l2(om[0], om[1]) < 6e-3 and A.rel_l2(om[2], om[1]) < 6e-3


def test_equal_betas_reduce_scalar_to_flow_relation():
    """beta1 = beta2 = 1: the scalar scheme is the standard one and N^phi
    carries the same strain information as N (measured 1e-3 relative)."""
    f = run_tg(48, 0.01, 300, beta2=1.0).fields(extra=True)
    # for this flow N is small (dxuy + dyux ~ 0): compare against the shear scale
    scale = np.abs(f["dxux"]).max()
    assert np.sqrt(np.mean((f["nxy_phi"] - f["nxy"]) ** 2)) < 5e-3 * scale


@pytest.mark.parametrize("php", [1.0, 1.2])
def test_couette_channel(php):
    """Periodic channel, static bottom wall, top wall moving at U: steady linear
    velocity and scalar (exact for half-way walls), exact shear rate, and the
    local vorticity equal to -U/H away from the first wall row (the
    scalar-gradient correction term of N^phi is exercised because phi varies
    linearly).  Measured: interior vorticity exact to 1e-6 relative."""
    n, U = 24, 0.02
    p = tg_params(n, 0.1, bc="channel", u_lid=U, phi_lid=2.0, phi_wall=1.0, omega_phi_hi=php)
    p.nx = 4
    F = inputs.rest(4, n, phi=1.5)
    L = O.OracleLattice(p).init(F.rho, F.ux, F.uy, F.phi)
    L.step(int(10 * n * n / 0.1))
    f = L.fields(extra=True)
    y = np.arange(n) + 0.5
    assert np.abs(f["ux"][:, 0] - U * y / n).max() < 1e-7
    assert np.abs(f["phi"][:, 0] - (1.0 + y / n)).max() < 1e-10
    assert np.abs(f["sxy"] - U / n / 2).max() < 1e-7
    assert np.abs(f["dyphi"] - 1.0 / n).max() < 1e-9
    inner = slice(8, n - 8) if php != 1.0 else slice(1, n - 1)
    np.testing.assert_allclose(f["omega"][inner], -U / n, rtol=1e-4)
    # the wall-adjacent row is not covered by the bulk relations
    assert abs(f["omega"][0, 0] / (-U / n) - 1) > 0.5


def test_fixed_scalar_laplace_solution():
    """Cavity at rest, phi = 1 on the top wall and 0 elsewhere: the steady
    scalar solves Laplace's equation (Fourier series).  Measured relative L2
    error 3.7e-3 at 32^2 (corner singularities dominate)."""
    n = 32
    p = tg_params(n, 0.1, D=0.1, bc="cavity", u_lid=0.0, phi_lid=1.0, phi_wall=0.0)
    F = inputs.rest(n, n)
    L = O.OracleLattice(p).init(F.rho, F.ux, F.uy, F.phi)
    L.step(6000)
    err = A.rel_l2(L.fields()["phi"], A.laplace_lid(n))
    assert err < 1e-2, err
