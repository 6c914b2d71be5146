"""Shared set-up of the GPU parity tests: one parameter spec drives both the
CUDA library (through the C ABI binding) and the FP64 oracle, with identical
relaxation rates given explicitly to each side."""
import math

import numpy as np

import oracle as O
from paper_1908_06742_gb300 import ddflb as D


def rate(nu):
    # nu = c_s^2 (1/omega - 1/2) with c_s^2 = 1/3, evaluated in the test
    return 1.0 / (3.0 * nu + 0.5)


def spec(nx, ny, bc="periodic", nu=0.01, D_phi=None, hi=1.2, phi_hi=1.2, beta2=0.9, u_lid=0.0,
         phi_lid=1.0, phi_wall=0.0, storage="fp32", scale=0.0, check_every=0, host_io=False,
         omega_f=None, omega_g=None, fx=0.0, fy=0.0, f_omega=0.0):
    D_phi = nu if D_phi is None else D_phi
    wf = omega_f or (0, 0, 0, hi, rate(nu), rate(nu), hi, hi, hi)
    wg = omega_g or (0, rate(D_phi), rate(D_phi), phi_hi, phi_hi, phi_hi, phi_hi, phi_hi, phi_hi)
    return dict(nx=nx, ny=ny, bc=bc, wf=tuple(wf), wg=tuple(wg), beta2=beta2, u_lid=u_lid,
                phi_lid=phi_lid, phi_wall=phi_wall, storage=storage, scale=scale,
                check_every=check_every, host_io=host_io, fx=fx, fy=fy, f_omega=f_omega)


def gpu_config(s):
    return D.Config(nx=s["nx"], ny=s["ny"], bc=s["bc"], storage=s["storage"], omega_f=s["wf"],
                    omega_g=s["wg"], beta2=s["beta2"], u_lid=s["u_lid"], phi_lid=s["phi_lid"],
                    phi_wall=s["phi_wall"], scale_f=s["scale"], scale_g=s["scale"],
                    check_every=s["check_every"], host_io=s["host_io"], fx=s.get("fx", 0.0),
                    fy=s.get("fy", 0.0), force_omega=s.get("f_omega", 0.0))


def oracle_params(s, storage="fp64"):
    st = {"fp32": "fp32", "fp16": "fp16", "bf16": "bf16", "fp64": "fp64"}[storage]
    sc = s["scale"] if s["scale"] > 0 and storage in ("fp16", "bf16") else 1.0
    return O.OracleParams(nx=s["nx"], ny=s["ny"], bc=s["bc"], lam_override=s["wf"],
                          lam_phi_override=s["wg"], beta2=s["beta2"], u_lid=s["u_lid"],
                          phi_lid=s["phi_lid"], phi_wall=s["phi_wall"], storage=st,
                          scale_f=sc, scale_g=sc, fx=s.get("fx", 0.0), fy=s.get("fy", 0.0),
                          f_omega=s.get("f_omega", 0.0))


def as_f32(F):
    """The inputs both sides receive: the FP32 values the library is given,
    widened back to FP64 for the oracle, so the two start from identical data."""
    r = lambda a: None if a is None else np.asarray(a, np.float32).astype(np.float64)
    return type(F)(r(F.rho), r(F.ux), r(F.uy), r(F.phi), r(F.grads))


def run_both(s, F, steps, use_grads=True, oracle_storage="fp64", force=None):
    """Initialise both sides from the same fields (and the same optional body
    force field [2, ny, nx], rounded to FP32 for both), advance ``steps``;
    return (gpu Lattice, oracle Lattice)."""
    F = as_f32(F)
    g = D.Lattice(gpu_config(s))
    o = O.OracleLattice(oracle_params(s, oracle_storage))
    if force is not None:
        force = np.asarray(force, np.float32).astype(np.float64)
        g.set_force_field(force)
        o.set_force(force)
    g.init(F.rho, F.ux, F.uy, F.phi, F.grads if use_grads else None)
    g.step(steps)
    o.init(F.rho, F.ux, F.uy, F.phi, F.grads if use_grads else None)
    o.step(steps)
    return g, o


def np64(t):
    return t.detach().double().cpu().numpy()


def rel_l2(a, b):
    return float(math.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))
