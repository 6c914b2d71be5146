"""Pins of the oracle's lattice algebra against what the paper prints and what
the mathematics fixes (no GPU)."""
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    return np.loadtxt(os.path.join(GOLD, name), comments="#")


# change of basis q (bare raw moments, App. B order) -> m (Sec. 2 order):
# m3 = kxx + kyy, m4 = kxx - kyy, all others identical.
C = np.eye(9)
C[3, 3], C[3, 4], C[4, 3], C[4, 4] = 1, 1, 1, -1


def test_inverse_matches_appendix_b():
    """T^-1 built by Gaussian elimination equals App. B's printed P^-1 once the
    (kxx+kyy, kxx-kyy) rows are mapped back to (kxx, kyy)."""
    g = _load("app_b_inverse.txt")
    Pinv = g[:, :1] * g[:, 1:]
    T, Ti, _, _, _ = O.lattice()
    np.testing.assert_allclose(Ti @ C, Pinv, atol=1e-14)
    np.testing.assert_allclose(T @ Ti, np.eye(9), atol=1e-14)


def test_forward_matches_appendix_d():
    """T from the basis polynomials equals C . P with P from App. D (a)."""
    P = _load("app_d_forward.txt")
    T, _, _, _, _ = O.lattice()
    np.testing.assert_array_equal(T, C @ P)


def test_velocities_and_rest_weights():
    """D2Q9 velocities of Sec. 2; rest equilibrium = textbook weights 4/9, 1/9, 1/36."""
    _, _, ex, ey, w = O.lattice()
    assert sorted(zip(ex.tolist(), ey.tolist())) == sorted(
        [(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)])
    assert (ex[0], ey[0]) == (0, 0)
    assert all(abs(ex[a]) + abs(ey[a]) == 1 for a in range(1, 5))
    np.testing.assert_allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, rtol=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equilibrium_hydrodynamic_moments(seed):
    """The flow equilibrium reproduces the Maxwellian moments the NSE need:
    sum f = rho, sum f e = rho u, sum f e e = c_s^2 rho I + rho u u (direct sums
    over the velocities, not through T)."""
    r = np.random.default_rng(seed)
    rho, ux, uy, phi = 1 + 0.1 * r.random(), 0.1 * r.standard_normal(), 0.1 * r.standard_normal(), 0.5 + r.random()
    p = O.OracleParams(nx=1, ny=1)
    meq, neq = O.equilibria(p, rho, ux, uy, phi)
    _, Ti, ex, ey, _ = O.lattice()
    feq, geq = Ti @ meq, Ti @ neq
    cs2 = 1 / 3
    for h, d in ((feq, rho), (geq, phi)):
        assert np.isclose(h.sum(), d, rtol=1e-14)
        assert np.isclose((h * ex).sum(), d * ux, atol=1e-15)
        assert np.isclose((h * ey).sum(), d * uy, atol=1e-15)
        assert np.isclose((h * ex * ex).sum(), cs2 * d + d * ux * ux, rtol=1e-13)
        assert np.isclose((h * ey * ey).sum(), cs2 * d + d * uy * uy, rtol=1e-13)
        assert np.isclose((h * ex * ey).sum(), d * ux * uy, atol=1e-15)


def test_scalar_anisotropy_only_in_third_order():
    """beta1, beta2 change only the two third-order off-diagonal equilibria of
    the scalar (Eq. eqmrawmoment_CDE), by (beta - 1) c_sphi^2 phi u."""
    ux, uy, phi = 0.03, -0.05, 1.7
    a = O.equilibria(O.OracleParams(nx=1, ny=1, beta1=1.0, beta2=1.0), 1.0, ux, uy, phi)[1]
    b = O.equilibria(O.OracleParams(nx=1, ny=1, beta1=1.3, beta2=0.8), 1.0, ux, uy, phi)[1]
    d = b - a
    assert np.all(np.abs(d[[0, 1, 2, 3, 4, 5, 8]]) < 1e-16)
    assert np.isclose(d[6], 0.3 / 3 * phi * uy) and np.isclose(d[7], -0.2 / 3 * phi * ux)
    # with beta1 = beta2 = 1 the scalar equilibria equal the flow ones with rho -> phi
    m = O.equilibria(O.OracleParams(nx=1, ny=1), phi, ux, uy, 1.0)[0]
    np.testing.assert_allclose(a, m, rtol=1e-15)


@pytest.mark.parametrize("seed", range(4))
def test_collision_invariants(seed):
    """Collision conserves rho and rho u (flow, F = 0) and phi (scalar)."""
    r = np.random.default_rng(seed)
    _, _, ex, ey, w = O.lattice()
    f = w * (1 + 0.05 * r.standard_normal(9))
    g = w * (1 + 0.05 * r.standard_normal(9))
    p = O.OracleParams(nx=1, ny=1, omega_nu=1.7, omega_bulk=1.1, omega_hi=1.3, omega_phi=1.5,
                       omega_phi_hi=0.9)
    fs, gs = O.collide_node(p, f, g)
    assert abs(fs.sum() - f.sum()) < 1e-15
    assert abs((fs * ex).sum() - (f * ex).sum()) < 1e-15
    assert abs((fs * ey).sum() - (f * ey).sum()) < 1e-15
    assert abs(gs.sum() - g.sum()) < 1e-15
    # first-order scalar moments relax (they are not invariants)
    assert abs((gs * ex).sum() - (g * ex).sum()) > 1e-6


def test_full_relaxation_reaches_equilibrium():
    """With every rate 1 (except the conserved moments) the post-collision
    moments are the equilibria of the pre-collision rho, u, phi."""
    r = np.random.default_rng(7)
    T, _, ex, ey, w = O.lattice()
    f = w * (1 + 0.05 * r.standard_normal(9))
    g = w * (1 + 0.05 * r.standard_normal(9))
    p = O.OracleParams(nx=1, ny=1, omega_nu=1, omega_bulk=1, omega_hi=1, omega_phi=1, omega_phi_hi=1,
                       beta1=1.2, beta2=0.7)
    fs, gs = O.collide_node(p, f, g)
    rho = f.sum(); ux = (f * ex).sum() / rho; uy = (f * ey).sum() / rho
    meq, neq = O.equilibria(p, rho, ux, uy, g.sum())
    np.testing.assert_allclose(T @ fs, meq, atol=1e-15)
    np.testing.assert_allclose(T @ gs, neq, atol=1e-15)


def test_storage_rounding_matches_ieee():
    """The rounding emulation matches numpy's IEEE binary32/binary16 casts and a
    bit-level round-to-nearest-even of binary32 to bfloat16."""
    r = np.random.default_rng(3)
    v = np.concatenate([r.standard_normal(4000) * 10.0 ** r.integers(-9, 4, 4000),
                        [65519.0, 65520.0, 6.0e-8, 2.9e-8, 1e-10, 0.0, -1.5e-5]])
    for storage in ("fp32", "fp16", "bf16"):
        got = O.round_storage(storage, v)
        if storage == "fp32":
            ref = v.astype(np.float32).astype(np.float64)
        elif storage == "fp16":
            with np.errstate(over="ignore"):
                ref = v.astype(np.float16).astype(np.float64)
        else:
            # bf16 from the binary64 value: round the binary64 significand to 8 bits
            # via exact integer arithmetic on the mantissa (RNE).
            m, e = np.frexp(v)
            q = np.ldexp(m, 8)
            fl = np.floor(q); frac = q - fl
            up = (frac > 0.5) | ((frac == 0.5) & (fl % 2 == 1))
            ref = np.ldexp(fl + up, e - 8)
        np.testing.assert_array_equal(got, ref, err_msg=storage)
