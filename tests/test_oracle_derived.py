"""Pins of the oracle's derived fields (the velocity-gradient invariants Q, R
and the Lamb vector named in Sec. 1, and the individual cross derivatives of
Eqs. offdiagvelderivativeresult1/2) against identities and library routines
that do not share their formulas."""
import numpy as np

import oracle as O
from tests import analytic as A
from tests.test_oracle_dynamics import run_tg


def tg_derived(n=48, steps=200):
    L = run_tg(n, 0.01, steps)
    f = L.fields(extra=True)
    return f, O.derived(f)


def gradient_tensor(d):
    A_ = np.zeros(d["dxux"].shape + (3, 3))   # A[i, j] = d_j u_i
    A_[..., 0, 0] = d["dxux"]; A_[..., 0, 1] = d["dyux"]
    A_[..., 1, 0] = d["dxuy"]; A_[..., 1, 1] = d["dyuy"]
    return A_


def test_q_is_minus_half_trace_of_a_squared():
    """Q = -tr(A^2)/2 (S:S - Omega:Omega split, valid for any A)."""
    f, d = tg_derived()
    A_ = gradient_tensor(d)
    q2 = -0.5 * np.trace(A_ @ A_, axis1=-2, axis2=-1)
    assert np.max(np.abs(d["q"] - q2)) < 1e-12 * np.max(np.abs(q2))


def test_r_from_trace_of_a_cubed():
    """tr(A^3) = S_ij S_jk S_ki + 3/4 omega_i omega_j S_ij - 3/4 omega^2 tr(S), so
    R = (tr(A^3) + 3/4 omega^2 tr S) / 3 (a matrix power, not the S/omega split);
    and for a planar flow R is of the order of tr(S) (zero if incompressible)."""
    f, d = tg_derived()
    A_ = gradient_tensor(d)
    trS = d["dxux"] + d["dyuy"]
    r2 = (np.trace(A_ @ A_ @ A_, axis1=-2, axis2=-1) + 0.75 * d["omega_z"] ** 2 * trS) / 3.0
    scale = np.max(np.abs(d["omega_z"])) ** 3
    assert np.max(np.abs(d["r"] - r2)) < 1e-12 * scale
    assert np.max(np.abs(d["r"])) < 1e-2 * scale


def test_lamb_vector_is_cross_product():
    f, d = tg_derived()
    om = np.stack([np.zeros_like(f["omega"]), np.zeros_like(f["omega"]), f["omega"]], -1)
    u = np.stack([f["ux"], f["uy"], np.zeros_like(f["ux"])], -1)
    L = np.cross(om, u)
    np.testing.assert_allclose(d["lamb_x"], L[..., 0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(d["lamb_y"], L[..., 1], rtol=0, atol=1e-15)
    assert np.all(d["lamb_z"] == 0)
    # omega from the Levi-Civita contraction is the Sec. 4 omega
    np.testing.assert_allclose(d["omega_z"], f["omega"], rtol=1e-12, atol=1e-18)


def test_taylor_green_q_and_cross_derivatives_match_analytic():
    """Decaying Taylor-Green vortex: Q = -tr(A^2)/2 of the analytic gradient, and
    the individual cross derivatives d_y u_x, d_x u_y, within the method's
    truncation (measured 5.7e-3, 4.6e-3, 4.1e-3 relative L2 at 48^2)."""
    n, u0, steps = 48, 0.01, 200
    f, d = tg_derived(n, steps)
    a = A.taylor_green(n, u0, 0.01, steps)      # run_tg's viscosity
    Aa = gradient_tensor(a)
    qa = -0.5 * np.trace(Aa @ Aa, axis1=-2, axis2=-1)
    e = (A.rel_l2(d["q"], qa), A.rel_l2(d["dyux"], a["dyux"]), A.rel_l2(d["dxuy"], a["dxuy"]))
    print("E_Q, E_dyux, E_dxuy", e)
    assert max(e) < 1e-2
