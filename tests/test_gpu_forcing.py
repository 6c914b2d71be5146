"""Parity of the forced CUDA path (Sec. 2 body force: source moments, f-bar =
f - S/2, u = (sum f-bar e + F/2)/rho) with the FP64 oracle, on the paper's
forced validation flows (Secs. 5.1-5.3) and on random states element by
element.  Bounds as in the unforced parity tests: 1e-5 relative L2 on u, phi
and S for FP32 storage, or 1.2 times the emulated FP32-storage floor (the
oracle run with every stored population rounded to FP32) where that floor
itself lies above 1e-5; omega within three times the emulated floor."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1908_06742_gb300 import build as B
from paper_1908_06742_gb300 import ddflb as D
from paper_1908_06742_gb300 import inputs
from tests import analytic as A
from tests.gpu_helpers import as_f32, gpu_config, np64, oracle_params, rate, rel_l2, run_both, spec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    D.load()


def fields64(g):
    return {k: np64(v) for k, v in g.fields().items()}


def errors(fg, fo, rows=slice(None)):
    """Relative-L2 errors: u (both components together), phi, S (worst
    component over the RMS of the largest) and omega, over the given rows."""
    e = {}
    e["u"] = rel_l2(np.stack([fg["ux"][rows], fg["uy"][rows]]),
                    np.stack([fo["ux"][rows], fo["uy"][rows]]))
    e["phi"] = rel_l2(fg["phi"][rows], fo["phi"][rows])
    ref = math.sqrt(max(np.mean(fo[k][rows] ** 2) for k in ("sxx", "sxy", "syy")))
    e["S"] = max(math.sqrt(np.mean((fg[k][rows] - fo[k][rows]) ** 2)) for k in ("sxx", "sxy", "syy")) / ref
    e["omega"] = rel_l2(fg["omega"][rows], fo["omega"][rows])
    return e


def emulated_fields(s, F, steps, use_grads=False, force=None):
    o = O.OracleLattice(oracle_params(s, "fp32"))
    if force is not None:
        o.set_force(np.asarray(force, np.float32).astype(np.float64))
    F = as_f32(F)
    o.init(F.rho, F.ux, F.uy, F.phi, F.grads if use_grads else None).step(steps)
    return o.fields()


def check(e, floor, target=1e-5):
    """u, phi, S within the target, or within 1.2 times the emulated storage
    floor where the floor is above the target: the long forced channel run
    (30000 steps of a steady force) rounds the stored momentum the same way
    every step, and FP32 storage alone leaves u at 1.35e-5 there; the kernel's
    compensated arithmetic lands on that floor (1.31e-5).  omega within three
    times the floor."""
    for k, v in e.items():
        if k == "omega":
            assert v <= max(target, 3 * floor[k]), (k, v, floor[k])
        else:
            assert v <= max(target, 1.2 * floor[k]), (k, v, target, floor[k])


# --------------------------------------------------------------- element by element
@pytest.mark.parametrize("bc", ["periodic", "cavity", "channel"])
@pytest.mark.parametrize("shape", [(200, 77), (2, 3)])
def test_forced_init_and_step_elementwise(bc, shape):
    """Constant force plus a random force field, modulated in time: the initial
    f-bar and five forced steps match the oracle population by population."""
    nx, ny = shape
    s = spec(nx, ny, bc=bc, nu=0.05, D_phi=0.02, u_lid=0.05, phi_lid=1.3, phi_wall=0.7,
             fx=2e-4, fy=-1e-4, f_omega=0.3)
    F = inputs.random_state(nx, ny, seed=5 * nx + ny)
    field = 1e-3 * np.random.default_rng(nx + ny).standard_normal((2, ny, nx))
    g, o = run_both(s, F, 0, force=field)
    f0, g0 = g.populations()
    np.testing.assert_allclose(np64(f0), o.f, rtol=0, atol=1e-7)
    np.testing.assert_allclose(np64(g0), o.g, rtol=0, atol=1e-7)
    g.step(5)
    o.step(5)
    f, gg = g.populations()
    np.testing.assert_allclose(np64(f), o.f, rtol=0, atol=5e-7)
    np.testing.assert_allclose(np64(gg), o.g, rtol=0, atol=5e-7)
    fg, fo = fields64(g), o.fields()
    for k in ("rho", "ux", "uy", "phi"):
        np.testing.assert_allclose(fg[k], fo[k], rtol=0, atol=2e-6)


def test_uniform_force_momentum_balance_gpu():
    """Periodic box, uniform force: total momentum grows by N F per step and the
    mass stays constant (FP64 sums of the FP32 fields)."""
    n, Fx, Fy = 64, 3e-5, -1e-5
    s = spec(n, n, nu=0.05, fx=Fx, fy=Fy)
    F = inputs.taylor_green(n, 0.01, phi_amp=0.1)
    g = D.Lattice(gpu_config(s)).init(F.rho, F.ux, F.uy, F.phi)
    a = fields64(g); m0 = g.stats()["mass"]
    g.step(40)
    b = fields64(g)
    for k, Fk in (("ux", Fx), ("uy", Fy)):
        dj = np.sum(b["rho"] * b[k]) - np.sum(a["rho"] * a[k])
        assert abs(dj - 40 * n * n * Fk) < 1e-4 * abs(40 * n * n * Fk), (k, dj)
    assert abs(g.stats()["mass"] - m0) < 1e-7 * n * n


def test_force_field_removed_restores_unforced_path():
    n = 48
    s0 = spec(n, n, nu=0.02)
    F = inputs.taylor_green(n, 0.02, phi_amp=0.1)
    a = D.Lattice(gpu_config(s0)).init(F.rho, F.ux, F.uy, F.phi).step(20)
    b = D.Lattice(gpu_config(s0))
    b.set_force_field(np.full((2, n, n), 1e-4)).set_force_field(None)
    b.init(F.rho, F.ux, F.uy, F.phi).step(20)
    fa, _ = a.populations(); fb, _ = b.populations()
    assert torch.equal(fa, fb)


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_forced_16bit_paired_request_matches_one_node_kernel(storage):
    """A forced context runs the one-node kernel even when the paired kernel is
    requested: both requests give bit-identical states."""
    n = 64
    s = spec(n, n, nu=0.02, fx=1e-5, storage=storage, scale=256.0)
    F = inputs.taylor_green(n, 0.02, phi_amp=0.1)
    out = []
    for path in (1, 2):
        g = D.Lattice(gpu_config(s)).set_path(path)
        g.init(F.rho, F.ux, F.uy, F.phi).step(30)
        out.append(g.populations())
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


# --------------------------------------------------------------- Sec. 5 flows
def test_poiseuille_gpu():
    """Sec. 5.1 channel, H = 32, F = 1e-6, nu = 0.1, tau^phi = 0.57, walls at
    phi = 1 / 2, 30000 steps: the GPU matches the oracle (u, phi, S at 1e-5,
    omega at three times the FP32-storage floor) and the analytic profile."""
    H, nu, F = 32, 0.1, 1e-6
    s = spec(3, H, bc="channel", nu=nu, hi=1.0, phi_hi=1.0,
             omega_g=(0, 1 / 0.57, 1 / 0.57, 1, 1, 1, 1, 1, 1),
             omega_f=(0, 0, 0, 1.0, rate(nu), rate(nu), 1.0, 1.0, 1.0),
             phi_wall=1.0, phi_lid=2.0, fx=F)
    st = inputs.rest(3, H, phi=1.5)
    g, o = run_both(s, st, 30000, use_grads=False)
    fg, fo = fields64(g), o.fields()
    e = errors(fg, fo)
    floor = errors(emulated_fields(s, st, 30000), fo)
    print("poiseuille", e, "floor", floor)
    check(e, floor)
    ua, oa = A.poiseuille(H, F, nu)
    assert A.rel_l2(fg["ux"][:, 0], ua) < 1e-3
    assert A.rel_l2(fg["omega"][1:-1, 0], oa[1:-1]) < 0.03


def test_four_rolls_mill_gpu():
    """Sec. 5.2 four-rolls mill, N = 48, force field F = 2 nu k^2 u0 (sin sin,
    cos cos), phi = 2, tau^phi = 0.57, to steady state: GPU vs oracle, and both
    vs the analytic velocity and vorticity."""
    n, u0, nu = 48, 0.01, 0.1
    a = A.four_rolls(n, u0, nu)
    s = spec(n, n, nu=nu, hi=1.2, omega_g=(0,) + (1 / 0.57,) * 2 + (1.2,) * 6)
    st = inputs.rest(n, n, phi=2.0)
    st = type(st)(st.rho, a["ux"], a["uy"], st.phi, None)
    k = 2 * math.pi / n
    steps = int(12 / (2 * nu * k * k))
    g, o = run_both(s, st, steps, use_grads=False, force=a["force"])
    fg, fo = fields64(g), o.fields()
    e = errors(fg, fo)
    floor = errors(emulated_fields(s, st, steps, force=a["force"]), fo)
    print("four rolls", e, "floor", floor)
    check(e, floor)
    assert A.rel_l2(fg["ux"], a["ux"]) < 5e-3
    assert math.sqrt(np.sum((fg["omega"] - a["omega"]) ** 2) / np.sum(a["omega"] ** 2)) < 1e-2


def test_womersley_gpu():
    """Sec. 5.3 pulsatile channel, 3 x 101, F = 1e-5 cos(2 pi t / 10000),
    tau = 0.781: started from the analytic profile, the GPU follows the oracle
    through one period and at 4 phases of the next (the modulation is applied
    at the step's own time on both sides)."""
    T, Fm, H, tau = 10000, 1e-5, 101, 0.781
    Om = 2 * math.pi / T
    nu = (tau - 0.5) / 3
    s = spec(3, H, bc="channel", omega_f=(0, 0, 0, 1.0, 1 / tau, 1 / tau, 1.0, 1.0, 1.0),
             omega_g=(0, 1 / 0.57, 1 / 0.57, 1, 1, 1, 1, 1, 1), phi_wall=1.0, phi_lid=2.0,
             fx=Fm, f_omega=Om)
    y = np.arange(H) + 0.5
    u0, om0 = A.womersley(H, Fm, Om, nu, 0.0)
    grads = np.zeros((6, H, 3))
    grads[1] = np.repeat(-om0[:, None], 3, axis=1)
    grads[5] = 1.0 / H
    st = inputs.Fields(np.ones((H, 3)), np.repeat(u0[:, None], 3, axis=1), np.zeros((H, 3)),
                      np.repeat((1.0 + y / H)[:, None], 3, axis=1), grads)
    g, o = run_both(s, st, T)
    em = O.OracleLattice(oracle_params(s, "fp32"))
    F = as_f32(st)
    em.init(F.rho, F.ux, F.uy, F.phi, F.grads).step(T)
    for _ in range(4):
        fg, fo = fields64(g), o.fields()
        e = errors(fg, fo)
        floor = errors(em.fields(), fo)
        print("womersley t", o.t, e, "floor", floor)
        check(e, floor)
        ua, _ = A.womersley(H, Fm, Om, nu, o.t)
        assert np.linalg.norm(fg["ux"][:, 0] - ua) / np.linalg.norm(ua) < 1e-3
        for L in (g, o, em):
            L.step(T // 4)
