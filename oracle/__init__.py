"""FP64 CPU oracle of the DDF-MRT lattice Boltzmann step with local vorticity.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path never
does.  It shares no code with the CUDA library: the arithmetic lives in
``ddflb_oracle.c`` (plain loops, 9x9 matrix products built from the paper's
definitions, double precision), this module only marshals numpy arrays.

Paper: Hajabdollahi & Premnath, "Local vorticity computation in double
distribution functions based lattice Boltzmann methods for flow and scalar
transport", arXiv 1908.06742.
  * lattice, basis T, raw moments ........ Sec. 2, Eqs. (particlevelocities)-(rawmomentdefinitions)
  * flow MRT collision, equilibria ....... Sec. 2, Eqs. (MRT-LBEfluidmotion_transformed), (eqmrawmoment)
  * scalar MRT with beta anisotropy ...... Sec. 3, Eqs. (MRT-LBECDE), (eqmrawmoment_CDE)
  * local strain rate and vorticity ...... Sec. 4, Eqs. (crossderivativeRHS1)-(vorticityexpression)
  * walls, lid, fixed scalar, periodic ... Sec. 5
  * body force (f-bar transformation) ..... Sec. 2, Eq. (MRT-LBEfluidmotion_transformed)
  * SRT / cascaded / central-moment scalar  Apps. B, C, D

Parity status of each function is recorded in the tests that pin it
(tests/test_oracle_*.py).  ``fields`` for the lid-driven cavity has no external
reference solution (parity unpinned beyond conservation, mirror symmetry and the
scalar Laplace solution at rest).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional

import numpy as np

from . import build as _build

Q = 9
BC = {"periodic": 0, "cavity": 1, "channel": 2}
STORAGE = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}
# scalar collision: Sec. 3 MRT, App. B SRT, App. C cascaded, App. D central moments
SCALAR_MODEL = {"mrt": 0, "srt": 1, "cascaded": 2, "central": 3}

_D = ctypes.POINTER(ctypes.c_double)


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("bc", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("lam", ctypes.c_double * Q), ("lam_phi", ctypes.c_double * Q),
        ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
        ("cs2", ctypes.c_double), ("cs2_phi", ctypes.c_double),
        ("rho0", ctypes.c_double), ("phi0", ctypes.c_double),
        ("u_lid", ctypes.c_double), ("phi_lid", ctypes.c_double), ("phi_wall", ctypes.c_double),
        ("phi_min", ctypes.c_double),
        ("scale_f", ctypes.c_double), ("scale_g", ctypes.c_double),
        ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("f_omega", ctypes.c_double),
        ("scalar_model", ctypes.c_int32), ("pad_", ctypes.c_int32),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_lattice.argtypes = [ctypes.c_double, _D, _D, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_int32), _D]
        L.orc_equilibria.argtypes = [ctypes.POINTER(_Params), ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, _D, _D]
        L.orc_collide_node.argtypes = [ctypes.POINTER(_Params), _D, _D, _D, _D]
        L.orc_init.argtypes = [ctypes.POINTER(_Params), _D, _D, _D, _D, _D, _D, _D, _D]
        L.orc_step.argtypes = [ctypes.POINTER(_Params), _D, _D, _D, _D, ctypes.c_int64, _D,
                               ctypes.c_int64]
        L.orc_fields.argtypes = [ctypes.POINTER(_Params), _D, _D, _D, _D, _D, ctypes.c_int64]
        L.orc_sums.argtypes = [ctypes.POINTER(_Params), _D, _D, _D, _D, ctypes.c_int64]
        L.orc_round.argtypes = [ctypes.c_int32, _D, ctypes.c_int64]
        L.orc_threads.argtypes = [ctypes.c_int]
        L.orc_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def omega_from_diffusivity(nu: float, cs2: float = 1.0 / 3.0) -> float:
    """Relaxation rate for a kinematic viscosity or diffusivity:
    nu = c_s^2 (1/omega - 1/2) (Sec. 2, after Eq. hydrodynamic_fields; Sec. 3 for D_phi)."""
    return 1.0 / (nu / cs2 + 0.5)


@dataclasses.dataclass
class OracleParams:
    nx: int
    ny: int
    bc: str = "periodic"
    omega_nu: float = 1.0          # omega_4 = omega_5 (shear viscosity)
    omega_bulk: float = 1.0        # omega_3
    omega_hi: float = 1.0          # omega_6, omega_7, omega_8
    omega_phi: float = 1.0         # omega_1^phi = omega_2^phi (diffusivity)
    omega_phi_hi: float = 1.0      # omega_3^phi .. omega_8^phi
    beta1: float = 1.0
    beta2: float = 0.9
    cs2: float = 1.0 / 3.0
    cs2_phi: float = 1.0 / 3.0
    rho0: float = 1.0
    phi0: float = 1.0
    u_lid: float = 0.0
    phi_lid: float = 1.0
    phi_wall: float = 0.0
    phi_min: float = 1e-3
    storage: str = "fp64"
    scale_f: float = 1.0
    scale_g: float = 1.0
    fx: float = 0.0                # constant body force (Sec. 2)
    fy: float = 0.0
    f_omega: float = 0.0           # force modulation cos(f_omega t), 0 = steady
    scalar_model: str = "mrt"      # "mrt" (Sec. 3), "srt" (App. B), "cascaded" (App. C), "central" (App. D)
    lam_override: Optional[tuple] = None      # full 9-entry flow diagonal (tests)
    lam_phi_override: Optional[tuple] = None  # full 9-entry scalar diagonal (tests)

    def lam(self):
        if self.lam_override is not None:
            return list(self.lam_override)
        # diag(0,0,0,w3,w4,w5,w6,w7,w8), Eq. (relaxationtimematrix_fluidmotion)
        return [0.0, 0.0, 0.0, self.omega_bulk, self.omega_nu, self.omega_nu,
                self.omega_hi, self.omega_hi, self.omega_hi]

    def lam_phi(self):
        if self.lam_phi_override is not None:
            return list(self.lam_phi_override)
        # diag(0,w1..w8), Eq. (relaxationtimematrix_CDE)
        h = self.omega_phi_hi
        return [0.0, self.omega_phi, self.omega_phi, h, h, h, h, h, h]

    def c(self) -> _Params:
        p = _Params()
        p.nx, p.ny, p.bc, p.storage = self.nx, self.ny, BC[self.bc], STORAGE[self.storage]
        for k, v in enumerate(self.lam()):
            p.lam[k] = v
        for k, v in enumerate(self.lam_phi()):
            p.lam_phi[k] = v
        p.beta1, p.beta2 = self.beta1, self.beta2
        p.cs2, p.cs2_phi = self.cs2, self.cs2_phi
        p.rho0, p.phi0 = self.rho0, self.phi0
        p.u_lid, p.phi_lid, p.phi_wall = self.u_lid, self.phi_lid, self.phi_wall
        p.phi_min = self.phi_min
        p.scale_f, p.scale_g = self.scale_f, self.scale_g
        p.fx, p.fy, p.f_omega = self.fx, self.fy, self.f_omega
        p.scalar_model = SCALAR_MODEL[self.scalar_model]
        return p


def lattice(cs2: float = 1.0 / 3.0):
    """(T, T^-1, e_x, e_y, rest weights) as the oracle builds them."""
    T = np.zeros((Q, Q)); Ti = np.zeros((Q, Q))
    ex = np.zeros(Q, np.int32); ey = np.zeros(Q, np.int32); w = np.zeros(Q)
    lib().orc_lattice(cs2, _ptr(T), _ptr(Ti), ex.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                      ey.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _ptr(w))
    return T, Ti, ex, ey, w


def equilibria(p: OracleParams, rho, ux, uy, phi):
    meq = np.zeros(Q); neq = np.zeros(Q)
    cp = p.c()
    lib().orc_equilibria(ctypes.byref(cp), rho, ux, uy, phi, _ptr(meq), _ptr(neq))
    return meq, neq


def collide_node(p: OracleParams, f, g):
    f = np.ascontiguousarray(f, np.float64); g = np.ascontiguousarray(g, np.float64)
    fs = np.zeros(Q); gs = np.zeros(Q)
    cp = p.c()
    lib().orc_collide_node(ctypes.byref(cp), _ptr(f), _ptr(g), _ptr(fs), _ptr(gs))
    return fs, gs


def round_storage(storage: str, v):
    """Round-to-nearest-even of each value to the storage format (emulation)."""
    a = np.array(v, dtype=np.float64, copy=True).ravel()
    lib().orc_round(STORAGE[storage], _ptr(a), a.size)
    return a


def threads(n: int = 0) -> int:
    """Set (n > 0) and return the OpenMP thread count the oracle uses."""
    return lib().orc_threads(int(n))


FIELD_NAMES = ("rho", "ux", "uy", "phi", "sxx", "sxy", "syy", "omega")
EXTRA_NAMES = ("dxux", "dyux", "dxuy", "dyuy", "nxy", "nxy_phi", "dxphi", "dyphi")


def derived(fields: dict) -> dict:
    """Velocity-gradient invariants and the Lamb vector named in Sec. 1, from
    the oracle's ``fields(extra=True)``: the gradient tensor A_ij = d_j u_i is
    embedded in 3-D (no z dependence, u_z = 0) and the definitions are
    evaluated as written with the Levi-Civita tensor:
      S = (A + A^T)/2,  omega_i = eps_ijk d_j u_k,
      Q = -S_ij S_ij / 2 + omega_k omega_k / 4,
      R = (S_ij S_jk S_ki + 3/4 omega_i omega_j S_ij) / 3,
      L_i = eps_ijk omega_j u_k.
    Also returns the gradients (dxux, dyux, dxuy, dyuy, dxphi, dyphi)."""
    ny, nx = fields["ux"].shape
    G = np.zeros((ny, nx, 3, 3))     # G[..., j, k] = d_j u_k
    G[..., 0, 0] = fields["dxux"]; G[..., 1, 0] = fields["dyux"]
    G[..., 0, 1] = fields["dxuy"]; G[..., 1, 1] = fields["dyuy"]
    A = np.swapaxes(G, -1, -2)       # A[..., i, j] = d_j u_i
    S = 0.5 * (A + np.swapaxes(A, -1, -2))
    eps = np.zeros((3, 3, 3))
    for i, j, k in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        eps[i, j, k] = 1.0
        eps[i, k, j] = -1.0
    om = np.einsum("ijk,...jk->...i", eps, G)
    u = np.stack([fields["ux"], fields["uy"], np.zeros_like(fields["ux"])], axis=-1)
    Q = -0.5 * np.einsum("...ij,...ij->...", S, S) + 0.25 * np.einsum("...k,...k->...", om, om)
    R = (np.einsum("...ij,...jk,...ki->...", S, S, S) +
         0.75 * np.einsum("...i,...j,...ij->...", om, om, S)) / 3.0
    Lv = np.einsum("ijk,...j,...k->...i", eps, om, u)
    return {"dxux": fields["dxux"], "dyux": fields["dyux"], "dxuy": fields["dxuy"],
            "dyuy": fields["dyuy"], "dxphi": fields["dxphi"], "dyphi": fields["dyphi"],
            "q": Q, "r": R, "lamb_x": Lv[..., 0], "lamb_y": Lv[..., 1], "omega_z": om[..., 2],
            "lamb_z": Lv[..., 2]}


class OracleLattice:
    """Two D2Q9 lattices (flow f, scalar g) advanced in FP64 on the CPU."""

    def __init__(self, params: OracleParams):
        self.p = params
        self._cp = params.c()
        shape = (Q, params.ny, params.nx)
        self.f = np.zeros(shape); self.g = np.zeros(shape)
        self._fs = np.zeros(shape); self._gs = np.zeros(shape)
        self.force = None   # optional body-force field [2, ny, nx] added to (fx, fy)
        self.t = 0

    def set_force(self, field):
        """Spatially varying body force (Fx, Fy) per node, [2, ny, nx]."""
        self.force = None if field is None else np.ascontiguousarray(field, np.float64).reshape(
            2, self.p.ny, self.p.nx)
        return self

    def init(self, rho, ux, uy, phi, grads=None):
        c = lambda a: np.ascontiguousarray(np.broadcast_to(a, (self.p.ny, self.p.nx)), np.float64)
        rho, ux, uy, phi = c(rho), c(ux), c(uy), c(phi)
        gr = None if grads is None else np.ascontiguousarray(grads, np.float64).reshape(6, self.p.ny, self.p.nx)
        lib().orc_init(ctypes.byref(self._cp), _ptr(rho), _ptr(ux), _ptr(uy), _ptr(phi), _ptr(gr),
                       _ptr(self.f), _ptr(self.g), _ptr(self.force))
        self.t = 0
        return self

    def set_state(self, f, g):
        self.f[...] = f; self.g[...] = g
        return self

    def step(self, n: int = 1):
        lib().orc_step(ctypes.byref(self._cp), _ptr(self.f), _ptr(self.g), _ptr(self._fs),
                       _ptr(self._gs), int(n), _ptr(self.force), int(self.t))
        self.t += n
        return self

    def fields(self, extra: bool = False) -> dict:
        ny, nx = self.p.ny, self.p.nx
        out = np.zeros((8, ny, nx))
        ex = np.zeros((8, ny, nx)) if extra else None
        lib().orc_fields(ctypes.byref(self._cp), _ptr(self.f), _ptr(self.g), _ptr(out), _ptr(ex),
                         _ptr(self.force), int(self.t))
        d = {k: out[i] for i, k in enumerate(FIELD_NAMES)}
        if extra:
            d.update({k: ex[i] for i, k in enumerate(EXTRA_NAMES)})
        return d

    def sums(self):
        out = np.zeros(3)
        lib().orc_sums(ctypes.byref(self._cp), _ptr(self.f), _ptr(self.g), _ptr(out),
                       _ptr(self.force), int(self.t))
        return {"mass": out[0], "scalar": out[1], "u2": out[2]}
