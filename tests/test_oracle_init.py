"""Pins of the oracle's initial state for the MRT and SRT scalar models: the
equilibria plus the Chapman-Enskog non-equilibrium moments of
Eqs. (strainratexxpyy)-(strainratexy) (flow: m3, m4, m5) and
Eqs. (1stnoneqmmomentx_CDE), (1stnoneqmmomenty_CDE),
(offdiagonal2ndnoneqmmoment_CDE) (scalar: n1, n2, n5).

Two independent checks, neither of which retypes the init formulas:

* round trip: the Sec. 4 relations of ``fields`` (pinned on their own by the
  Taylor-Green closed form and by central differences of the oracle's own
  velocity) return every input gradient at t = 0, for arbitrary gradient
  fields, with and without a body force;
* no initial transient: the non-equilibrium part the init writes is the one the
  collision-and-stream dynamics maintains, so the recovered gradients barely
  change over the first step.  A slip in a Chapman-Enskog term (sign, factor,
  rate) leaves a non-equilibrium part the collision has to relax, and the
  fields jump by O(1) in one step; the planted cases (one input gradient plane
  negated, or all halved) show it.
"""
import numpy as np
import pytest

import oracle as O
from paper_1908_06742_gb300 import inputs
from tests.test_oracle_dynamics import tg_params

GRADS = ("dxux", "dyux", "dxuy", "dyuy", "dxphi", "dyphi")


def params(n, model, **kw):
    p = tg_params(n, 0.01, D=0.02, omega_phi_hi=1.3, **kw)
    p.scalar_model = model
    return p


@pytest.mark.parametrize("model", ["mrt", "srt"])
@pytest.mark.parametrize("case", ["taylor_green", "random", "distinct_rates"])
def test_init_fields_round_trip(model, case):
    """Taylor-Green with a non-uniform scalar, or seeded random fields with
    random (inconsistent) gradients, the last with every relaxation rate
    different (so a rate taken from the wrong moment shows): rho, u, phi and
    all six gradients come back from the t = 0 state to rounding."""
    if case == "taylor_green":
        n = 32
        F = inputs.taylor_green(n, 0.02, phi_amp=0.1)
    else:
        n = 24
        F = inputs.random_state(n, n, seed=11)
    p = params(n, model)
    if case == "distinct_rates":
        p.lam_override = (0, 0, 0, 1.15, 1.6, 1.7, 1.1, 1.3, 1.0)
        p.lam_phi_override = (0, 1.5, 1.75, 1.3, 1.25, 1.35, 1.2, 1.05, 1.4)
    L = O.OracleLattice(p).init(F.rho, F.ux, F.uy, F.phi, F.grads)
    f = L.fields(extra=True)
    for k in ("rho", "ux", "uy", "phi"):
        np.testing.assert_allclose(f[k], getattr(F, k), rtol=0, atol=1e-15)
    g = np.asarray(F.grads)
    for i, k in enumerate(GRADS):
        np.testing.assert_allclose(f[k], g[i], rtol=0, atol=1e-11 * np.abs(g[i]).max())


def test_init_fields_round_trip_with_force():
    """With a body force the init holds f-bar = f - S/2 (Sec. 2); the fields
    add S/2 back, so the round trip still returns u and every gradient."""
    n = 24
    F = inputs.random_state(n, n, seed=12)
    p = params(n, "mrt", fx=2e-5, fy=-1e-5)
    r = np.random.default_rng(3)
    L = O.OracleLattice(p).set_force(1e-5 * r.standard_normal((2, n, n)))
    L.init(F.rho, F.ux, F.uy, F.phi, F.grads)
    f = L.fields(extra=True)
    np.testing.assert_allclose(f["ux"], F.ux, rtol=0, atol=1e-15)
    np.testing.assert_allclose(f["uy"], F.uy, rtol=0, atol=1e-15)
    g = np.asarray(F.grads)
    for i, k in enumerate(GRADS):
        np.testing.assert_allclose(f[k], g[i], rtol=0, atol=1e-11 * np.abs(g[i]).max())


def first_step_jump(model, F, grads, names):
    """RMS change of each recovered field over the first step, relative to its
    RMS after the step (64^2, nu = 0.01, D = 0.02, other rates 1.2 / 1.3)."""
    n = F.rho.shape[0]
    L = O.OracleLattice(params(n, model)).init(F.rho, F.ux, F.uy, F.phi, grads)
    f0 = L.fields(extra=True)
    L.step(1)
    f1 = L.fields(extra=True)
    return {k: float(np.sqrt(np.mean((f1[k] - f0[k]) ** 2) / np.mean(f1[k] ** 2))) for k in names}


@pytest.mark.parametrize("model", ["mrt", "srt"])
def test_init_has_no_velocity_gradient_transient(model):
    """Sine waves 64^2 with every velocity-gradient component nonzero (shear and
    divergence, so m3, m4 and m5 all carry a Chapman-Enskog part) and a uniform
    scalar: S, the cross derivatives and omega change by at most 6 % over the
    first step (measured 0.3 % for S, 0.6-4 % for the cross derivatives and
    omega).  Planted slips of the flow terms (one gradient plane negated, the
    shear pair doubled, all halved) make at least one of them jump by more than
    30 % (measured 46-233 %)."""
    F = inputs.sine_waves(64)
    names = GRADS[:4] + ("sxx", "sxy", "syy", "omega")
    j = first_step_jump(model, F, F.grads, names)
    print(model, "correct", j)
    assert max(j.values()) < 0.06, j
    planted = [(-1.0, (i,)) for i in range(4)] + [(2.0, (1, 2)), (0.5, (0, 1, 2, 3))]
    for factor, planes in planted:
        g = F.grads.copy()
        for i in planes:
            g[i] *= factor
        jp = first_step_jump(model, F, g, names)
        print(model, "planted", factor, planes, jp)
        assert max(jp.values()) > 0.3, (factor, planes, jp)


@pytest.mark.parametrize("model", ["mrt", "srt"])
def test_init_has_no_scalar_gradient_transient(model):
    """Taylor-Green 64^2 with phi = 1 + 0.1 sin sin: the scalar gradient changes
    by at most 5 % over the first step (measured 1.5-2 %); with either scalar
    gradient plane negated, or both halved, it jumps by more than 50 %
    (measured 64-139 %)."""
    F = inputs.taylor_green(64, 0.01, phi_amp=0.1)
    names = ("dxphi", "dyphi")
    j = first_step_jump(model, F, F.grads, names)
    print(model, "correct", j)
    assert max(j.values()) < 0.05, j
    for factor, i in ((-1, 4), (-1, 5), (0.5, None)):
        g = F.grads.copy()
        if i is None:
            g[4:] *= factor
        else:
            g[i] *= factor
        jp = first_step_jump(model, F, g, names)
        print(model, "planted", factor, i, jp)
        assert max(jp.values()) > 0.5, (factor, i, jp)
