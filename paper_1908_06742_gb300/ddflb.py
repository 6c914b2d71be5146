"""Python binding of the C ABI in include/ddflb.h (argument marshalling only).

Every step of the method runs in the CUDA library libddflb.so; this module
loads it with ctypes, allocates the caller-owned device memory with PyTorch and
passes raw pointers and the current CUDA stream.  There is no CPU fallback:
without the built library every entry point raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libddflb.so")

OK, EINVAL, ENOMEM, ECUDA, EDIVERGED, ENOTCONVERGED, ETIMEOUT = range(7)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EDIVERGED", "ENOTCONVERGED", "ETIMEOUT"]
BC = {"periodic": 0, "cavity": 1, "channel": 2}
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}
SCALAR_MODEL = {"mrt": 0, "srt": 1, "cascaded": 2, "central": 3}
FLAG_HOST_IO = 1
FIELD_NAMES = ("rho", "ux", "uy", "phi", "sxx", "sxy", "syy", "omega")
DERIVED_NAMES = ("dxux", "dyux", "dxuy", "dyuy", "dxphi", "dyphi", "q", "r", "lamb_x", "lamb_y")


class DdflbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    """Mirror of ddflb_params."""
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("bc", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("omega_f", ctypes.c_double * 9), ("omega_g", ctypes.c_double * 9),
        ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
        ("cs2", ctypes.c_double), ("cs2_phi", ctypes.c_double),
        ("rho0", ctypes.c_double), ("phi0", ctypes.c_double),
        ("u_lid", ctypes.c_double), ("phi_lid", ctypes.c_double), ("phi_wall", ctypes.c_double),
        ("phi_min", ctypes.c_double),
        ("scale_f", ctypes.c_double), ("scale_g", ctypes.c_double),
        ("check_every", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("force_omega", ctypes.c_double),
        ("scalar_model", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


_VP = ctypes.c_void_p
_FP = ctypes.c_void_p  # device pointers travel as integers
_lib = None

# name -> (restype, argtypes); every symbol declared in include/ddflb.h
SIGNATURES = {
    "ddflb_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(Params)]),
    "ddflb_create": (ctypes.c_int, [ctypes.POINTER(Params), _VP, ctypes.c_size_t, _VP,
                                    ctypes.POINTER(_VP)]),
    "ddflb_init": (ctypes.c_int, [_VP, _FP, _FP, _FP, _FP, _FP]),
    "ddflb_init_host": (ctypes.c_int, [_VP, _FP, _FP, _FP, _FP, _FP]),
    "ddflb_step": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "ddflb_fields": (ctypes.c_int, [_VP] + [_FP] * 8),
    "ddflb_fields_host": (ctypes.c_int, [_VP] + [_FP] * 8),
    "ddflb_derived": (ctypes.c_int, [_VP] + [_FP] * 10),
    "ddflb_fields_host_async": (ctypes.c_int, [_VP] + [_FP] * 8),
    "ddflb_set_io_streams": (ctypes.c_int, [_VP, _VP, _VP]),
    "ddflb_io_wait": (ctypes.c_int, [_VP]),
    "ddflb_populations": (ctypes.c_int, [_VP, _FP, _FP]),
    "ddflb_run_to_tolerance": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int64, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_int64)]),
    "ddflb_stats": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_int64)]),
    "ddflb_state_bytes": (ctypes.c_size_t, [_VP]),
    "ddflb_get_state": (ctypes.c_int, [_VP, _FP, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int64)]),
    "ddflb_set_state": (ctypes.c_int, [_VP, _FP, ctypes.c_size_t, ctypes.c_int64]),
    "ddflb_destroy": (ctypes.c_int, [_VP]),
    "ddflb_reduce_noalloc": (ctypes.c_int, [ctypes.POINTER(Params), _FP, ctypes.c_size_t,
                                            ctypes.c_int32, _FP, _VP]),
    "ddflb_batch_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.POINTER(Params)]),
    "ddflb_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(Params), _VP,
                                          ctypes.c_size_t, _VP, ctypes.POINTER(_VP)]),
    "ddflb_batch_set_run": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int32, ctypes.c_double,
                                           ctypes.c_int32]),
    "ddflb_batch_set_tiles": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "ddflb_batch_set_instance_run": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_double,
                                                    ctypes.c_int64]),
    "ddflb_batch_set_schedule": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "ddflb_batch_get_schedule": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32)]),
    "ddflb_batch_get_tiles": (ctypes.c_int, [_VP] + [ctypes.POINTER(ctypes.c_int32)] * 3),
    "ddflb_batch_init": (ctypes.c_int, [_VP, ctypes.c_int32, _FP, _FP, _FP, _FP, _FP]),
    "ddflb_batch_step": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "ddflb_batch_fields": (ctypes.c_int, [_VP, ctypes.c_int32] + [_FP] * 8),
    "ddflb_batch_stats": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "ddflb_batch_debug_skip_barrier": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "ddflb_batch_autotune": (ctypes.c_int, [_VP, ctypes.c_int32] +
                             [ctypes.POINTER(ctypes.c_int32)] * 3 + [ctypes.POINTER(ctypes.c_double)]),
    "ddflb_set_path": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "ddflb_autotune": (ctypes.c_int, [_VP, ctypes.c_int32] + [ctypes.POINTER(ctypes.c_int32)] * 3 +
                       [ctypes.POINTER(ctypes.c_double)]),
    "ddflb_set_block": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32]),
    "ddflb_set_force_field": (ctypes.c_int, [_VP, _FP]),
    # y-slab decomposition of one lattice
    "ddflb_slab_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(Params), ctypes.c_int32,
                                                     ctypes.c_int32]),
    "ddflb_slab_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int32, ctypes.c_int32,
                                         _VP, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)]),
    "ddflb_halo_elems": (ctypes.c_size_t, [_VP]),
    "ddflb_halo_pack": (ctypes.c_int, [_VP, _FP, _FP]),
    "ddflb_halo_unpack": (ctypes.c_int, [_VP, _FP, _FP]),
    "ddflb_halo_exchange_local": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int32]),
    "ddflb_sums": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    # warm-start surrogate network kernels
    "ddflb_nn_gemm": (ctypes.c_int, [_FP, _FP] + [ctypes.c_int32] * 5 +
                      [_FP, ctypes.c_int32, _FP, ctypes.c_int32, _FP] + [ctypes.c_int32] * 3 +
                      [_FP, _VP]),
    "ddflb_nn_set_gemm_path": (ctypes.c_int, [ctypes.c_int32]),
    "ddflb_nn_take_error": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), _VP]),
    "ddflb_nn_conv3x3": (ctypes.c_int, [_FP] + [ctypes.c_int32] * 5 +
                         [_FP, ctypes.c_int32, _FP, ctypes.c_int32, _FP, ctypes.c_int32, _FP,
                          ctypes.c_int32, ctypes.c_int32, _VP]),
    "ddflb_nn_set_conv_path": (ctypes.c_int, [ctypes.c_int32]),
    "ddflb_nn_conv3x3_flip": (ctypes.c_int, [_FP, ctypes.c_int32, ctypes.c_int32, _FP, _VP]),
    "ddflb_nn_im2col": (ctypes.c_int, [_FP] + [ctypes.c_int32] * 5 + [_FP, ctypes.c_int32, _VP]),
    "ddflb_nn_col2im": (ctypes.c_int, [_FP] + [ctypes.c_int32] * 4 + [_FP, ctypes.c_int32, _VP]),
    "ddflb_nn_transpose": (ctypes.c_int, [_FP] + [ctypes.c_int32] * 3 + [_FP, _VP]),
    "ddflb_nn_pool": (ctypes.c_int, [_FP] + [ctypes.c_int32] * 5 + [_FP, ctypes.c_int32, _VP]),
    "ddflb_nn_pool_bwd": (ctypes.c_int, [_FP] + [ctypes.c_int32] * 5 +
                          [_FP, ctypes.c_int32, ctypes.c_int32, _VP]),
    "ddflb_nn_upsample": (ctypes.c_int, [_FP] + [ctypes.c_int32] * 5 + [_FP, ctypes.c_int32, _VP]),
    "ddflb_nn_upsample_bwd": (ctypes.c_int, [_FP] + [ctypes.c_int32] * 5 +
                              [_FP, ctypes.c_int32, _VP]),
    "ddflb_nn_act_bwd": (ctypes.c_int, [_FP, _FP, ctypes.c_int64] + [ctypes.c_int32] * 4 +
                         [_FP, ctypes.c_int32, _VP]),
    "ddflb_nn_bias_grad": (ctypes.c_int, [_FP, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                          _FP, _VP]),
    "ddflb_nn_mse": (ctypes.c_int, [_FP, _FP, ctypes.c_int64, _FP, _FP, _FP, _VP]),
    "ddflb_nn_adam": (ctypes.c_int, [_FP, _FP, _FP, _FP, _FP, ctypes.c_int64] +
                      [ctypes.c_float] * 4 + [ctypes.c_int64, ctypes.c_float, _VP]),
    "ddflb_nn_cast_bf16": (ctypes.c_int, [_FP, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                          _FP, ctypes.c_int32, _VP]),
    "ddflb_warm_fields": (ctypes.c_int, [_FP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, _FP, _FP, _FP, _FP, _FP, _VP]),
    "ddflb_batch_destroy": (ctypes.c_int, [_VP]),
    "ddflb_last_error": (ctypes.c_char_p, []),
    "ddflb_version": (ctypes.c_char_p, []),
}

INST_CONVERGED, INST_DIVERGED, INST_CAPPED = 1, 2, 4


def load(path: str = LIB_PATH):
    """Load libddflb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} not built: run __graft_entry__.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int):
    if status != OK:
        raise DdflbError(status, load().ddflb_last_error().decode())


def relaxation_rate(diffusivity: float, cs2: float = 1.0 / 3.0) -> float:
    """omega for a viscosity or diffusivity: nu = cs2 (1/omega - 1/2) (Secs. 2, 3)."""
    return 1.0 / (diffusivity / cs2 + 0.5)


@dataclasses.dataclass
class Config:
    """User-facing parameters; ``to_c`` fills the ABI struct."""
    nx: int
    ny: int
    bc: str = "periodic"
    storage: str = "fp32"
    nu: float = 0.01            # kinematic viscosity -> omega_4 = omega_5
    diffusivity: float = 0.01   # D_phi -> omega_1^phi = omega_2^phi
    omega_bulk: float = 1.2     # omega_3
    omega_hi: float = 1.2       # omega_6..8
    omega_phi_hi: float = 1.2   # omega_3^phi..omega_8^phi
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
    scale_f: float = 0.0
    scale_g: float = 0.0
    check_every: int = 0
    host_io: bool = False
    omega_f: Optional[tuple] = None   # explicit 9-entry diagonals override the above
    omega_g: Optional[tuple] = None
    scalar_model: str = "mrt"   # "mrt" (Sec. 3), "srt" (App. B), "cascaded" (App. C), "central" (App. D)
    fx: float = 0.0             # body force (Sec. 2), times cos(force_omega t)
    fy: float = 0.0
    force_omega: float = 0.0

    def rates(self):
        wf = self.omega_f or (0.0, 0.0, 0.0, self.omega_bulk, relaxation_rate(self.nu, self.cs2),
                              relaxation_rate(self.nu, self.cs2), self.omega_hi, self.omega_hi,
                              self.omega_hi)
        wphi = relaxation_rate(self.diffusivity, self.cs2_phi)
        h = self.omega_phi_hi
        wg = self.omega_g or (0.0, wphi, wphi, h, h, h, h, h, h)
        return tuple(wf), tuple(wg)

    def to_c(self) -> Params:
        p = Params()
        p.nx, p.ny = self.nx, self.ny
        p.bc, p.storage = BC[self.bc], STORAGE[self.storage]
        wf, wg = self.rates()
        for k in range(9):
            p.omega_f[k] = wf[k]
            p.omega_g[k] = wg[k]
        p.beta1, p.beta2 = self.beta1, self.beta2
        p.cs2, p.cs2_phi = self.cs2, self.cs2_phi
        p.rho0, p.phi0 = self.rho0, self.phi0
        p.u_lid, p.phi_lid, p.phi_wall = self.u_lid, self.phi_lid, self.phi_wall
        p.phi_min = self.phi_min
        p.scale_f, p.scale_g = self.scale_f, self.scale_g
        p.check_every = self.check_every
        p.flags = FLAG_HOST_IO if self.host_io else 0
        p.fx, p.fy, p.force_omega = self.fx, self.fy, self.force_omega
        p.scalar_model = SCALAR_MODEL[self.scalar_model]
        return p


def workspace_bytes(cfg: Config) -> int:
    p = cfg.to_c()
    n = load().ddflb_workspace_bytes(ctypes.byref(p))
    if n == 0:
        _check(EINVAL)
    return n


NOALLOC_MAX_NODES = 1 << 20


def reduce_noalloc(cfg: Config, state, mode: int, out, stream=None):
    """ddflb_reduce_noalloc on a raw state tensor (as from Lattice.get_state):
    writes (mass, scalar, sum |u|^2, residual) into the 4-double device tensor
    ``out`` without allocating device memory."""
    import torch
    p = cfg.to_c()
    st = stream or torch.cuda.current_stream()
    _check(load().ddflb_reduce_noalloc(ctypes.byref(p), state.data_ptr(), state.numel(),
                                       int(mode), out.data_ptr(), st.cuda_stream))
    return out


def warm_fields(pred, u_lid: float, omega_scale: float, phi_lo: float = 0.0, phi_hi: float = 1.0,
                stream=None):
    """ddflb_warm_fields on a device FP32 prediction [ny, nx, C] (C >= 5):
    returns device (rho, ux, uy, phi, grads[6]) for Lattice.init / Batch.init."""
    import torch
    ny, nx, C = pred.shape
    assert pred.dtype == torch.float32 and pred.is_contiguous() and pred.is_cuda
    planes = torch.empty((10, ny, nx), dtype=torch.float32, device=pred.device)
    st = stream or torch.cuda.current_stream(pred.device)
    _check(load().ddflb_warm_fields(pred.data_ptr(), nx, ny, C, float(u_lid), float(omega_scale),
                                    float(phi_lo), float(phi_hi), planes[0].data_ptr(),
                                    planes[1].data_ptr(), planes[2].data_ptr(),
                                    planes[3].data_ptr(), planes[4].data_ptr(), st.cuda_stream))
    return planes[0], planes[1], planes[2], planes[3], planes[4:]


def _dptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


class Lattice:
    """One pair of D2Q9 lattices (flow f, scalar g) resident on the GPU; with
    ``rows = (y0, count)``, the y-slab of those rows of the lattice ``cfg``
    (ddflb_slab_create: fields, force field and sums cover its own rows)."""

    def __init__(self, cfg: Config, device=None, stream=None, rows=None):
        import torch
        self.torch = torch
        self.cfg = cfg
        self.device = torch.device(device or "cuda")
        self.lib = load()
        self._p = cfg.to_c()
        if rows is None:
            nbytes = workspace_bytes(cfg)
        else:
            nbytes = self.lib.ddflb_slab_workspace_bytes(ctypes.byref(self._p), int(rows[0]),
                                                         int(rows[1]))
            if nbytes == 0:
                _check(EINVAL)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        h = _VP()
        if rows is None:
            _check(self.lib.ddflb_create(ctypes.byref(self._p), self.workspace.data_ptr(), nbytes,
                                         self.stream.cuda_stream, ctypes.byref(h)))
        else:
            _check(self.lib.ddflb_slab_create(ctypes.byref(self._p), int(rows[0]), int(rows[1]),
                                              self.workspace.data_ptr(), nbytes,
                                              self.stream.cuda_stream, ctypes.byref(h)))
        self._h = h
        self.rows = rows
        self.shape = (cfg.ny if rows is None else int(rows[1]), cfg.nx)

    # -- helpers
    def _dev(self, a):
        t = self.torch
        if a is None:
            return None
        if isinstance(a, np.ndarray):
            a = t.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
        return a.to(device=self.device, dtype=t.float32).contiguous()

    def _empty(self, *lead):
        return self.torch.empty(*lead, *self.shape, dtype=self.torch.float32, device=self.device)

    # -- ABI
    def init(self, rho, ux, uy, phi, grads=None):
        self._keep = [self._dev(a) for a in (rho, ux, uy, phi, grads)]
        r, u, v, p, g = self._keep
        _check(self.lib.ddflb_init(self._h, _dptr(r), _dptr(u), _dptr(v), _dptr(p), _dptr(g)))
        return self

    def init_host(self, rho, ux, uy, phi, grads=None):
        """Host (CPU, ideally pinned) float32 tensors; copies run inside the call."""
        args = [None if a is None else a.data_ptr() for a in (rho, ux, uy, phi, grads)]
        _check(self.lib.ddflb_init_host(self._h, *args))
        return self

    def step(self, n: int = 1):
        _check(self.lib.ddflb_step(self._h, int(n)))
        return self

    def fields(self, names=FIELD_NAMES) -> dict:
        out = {k: (self._empty() if k in names else None) for k in FIELD_NAMES}
        _check(self.lib.ddflb_fields(self._h, *[_dptr(out[k]) for k in FIELD_NAMES]))
        return {k: v for k, v in out.items() if v is not None}

    def derived(self, names=DERIVED_NAMES) -> dict:
        """Velocity and scalar gradients, Q, R and the Lamb vector (one pass)."""
        out = {k: (self._empty() if k in names else None) for k in DERIVED_NAMES}
        _check(self.lib.ddflb_derived(self._h, *[_dptr(out[k]) for k in DERIVED_NAMES]))
        return {k: v for k, v in out.items() if v is not None}

    def fields_host(self, out: dict) -> dict:
        """Write fields into host float32 tensors given by name (synchronises)."""
        _check(self.lib.ddflb_fields_host(
            self._h, *[(out[k].data_ptr() if k in out else None) for k in FIELD_NAMES]))
        return out

    def fields_host_async(self, out: dict) -> dict:
        """Queue the fields into host float32 tensors (pinned); valid after io_wait()."""
        _check(self.lib.ddflb_fields_host_async(
            self._h, *[(out[k].data_ptr() if k in out else None) for k in FIELD_NAMES]))
        return out

    def set_io_streams(self, upload=None, download=None):
        """Run host uploads / downloads on two torch.cuda.Streams (None, None: the
        context stream), overlapping them with the time steps."""
        self._io = (upload, download)
        _check(self.lib.ddflb_set_io_streams(
            self._h, None if upload is None else upload.cuda_stream,
            None if download is None else download.cuda_stream))
        return self

    def io_wait(self):
        _check(self.lib.ddflb_io_wait(self._h))
        return self

    def populations(self):
        f, g = self._empty(9), self._empty(9)
        _check(self.lib.ddflb_populations(self._h, f.data_ptr(), g.data_ptr()))
        return f, g

    def run_to_tolerance(self, tol: float = 1e-8, max_steps: int = 10_000_000,
                         stall_checks: int = 0) -> dict:
        """Step until the residual (checked every check_every steps) is below
        tol.  Returns {"status": "OK" | "ENOTCONVERGED" | "EDIVERGED", "steps": n,
        "message": ...}; other errors raise."""
        k = ctypes.c_int64()
        st = self.lib.ddflb_run_to_tolerance(self._h, float(tol), int(max_steps),
                                             int(stall_checks), ctypes.byref(k))
        if st not in (OK, ENOTCONVERGED, EDIVERGED):
            _check(st)
        return {"status": STATUS_NAMES[st], "steps": k.value,
                "message": "" if st == OK else self.lib.ddflb_last_error().decode()}

    def stats(self) -> dict:
        m, s, r = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        k = ctypes.c_int64()
        st = self.lib.ddflb_stats(self._h, ctypes.byref(m), ctypes.byref(s), ctypes.byref(r),
                                  ctypes.byref(k))
        if st not in (OK, EDIVERGED):
            _check(st)
        return {"mass": m.value, "scalar": s.value, "residual": r.value, "step": k.value,
                "diverged": st == EDIVERGED}

    def autotune(self, trial_steps=10, cache=True):
        """Pick the step kernel's block shape (cached by workload signature);
        must run before init (it overwrites the state)."""
        from . import tuning
        key = tuning.key("lattice", [self.cfg])
        hit = tuning.lookup(key) if cache else None
        if hit:
            _check(self.lib.ddflb_set_block(self._h, *hit["choice"][:2]))
            _check(self.lib.ddflb_set_path(self._h, hit["choice"][2]))
            return hit
        bx, by, pth, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        _check(self.lib.ddflb_autotune(self._h, int(trial_steps), ctypes.byref(bx),
                                       ctypes.byref(by), ctypes.byref(pth), ctypes.byref(ms)))
        rec = {"choice": [bx.value, by.value, pth.value], "ms_per_step": ms.value}
        if cache:
            tuning.store(key, rec)
        return rec

    def set_force_field(self, field):
        """Spatially varying body force [2, ny, nx] (F_x, F_y) added to (fx, fy);
        kept alive by this object.  None removes it."""
        self._force = None if field is None else self._dev(field).reshape(2, *self.shape).contiguous()
        _check(self.lib.ddflb_set_force_field(self._h, _dptr(self._force)))
        return self

    def set_path(self, path: int):
        """Step kernel variant: 0 automatic (16-bit storage: groups of 4 nodes
        where nx is a multiple of 4, else pairs on periodic lattices), 1 one node
        per thread, 2 paired nodes, 3 groups of 4 nodes.  All give the same
        state."""
        _check(self.lib.ddflb_set_path(self._h, int(path)))
        return self

    def state_bytes(self) -> int:
        return self.lib.ddflb_state_bytes(self._h)

    def get_state(self):
        buf = self.torch.empty(self.state_bytes(), dtype=self.torch.uint8, device=self.device)
        k = ctypes.c_int64()
        _check(self.lib.ddflb_get_state(self._h, buf.data_ptr(), buf.numel(), ctypes.byref(k)))
        return buf, k.value

    def set_state(self, buf, step: int):
        _check(self.lib.ddflb_set_state(self._h, buf.data_ptr(), buf.numel(), int(step)))
        return self

    def sums(self, mode: int = 0):
        """FP64 sums over this context's nodes (ddflb_sums): mass and scalar
        deviations, sum |u|^2, and sum |u - u_snap|^2 (mode bit 1); mode bit 2
        stores the snapshot.  Synchronises."""
        out = (ctypes.c_double * 4)()
        _check(self.lib.ddflb_sums(self._h, int(mode), out))
        return {"mass_dev": out[0], "scalar_dev": out[1], "u2": out[2], "du2": out[3]}

    def halo_elems(self) -> int:
        return self.lib.ddflb_halo_elems(self._h)

    def halo_pack(self, down, up):
        """Outgoing face rows into device tensors of halo_elems() storage
        elements (None for a wall face)."""
        _check(self.lib.ddflb_halo_pack(self._h, _dptr(down), _dptr(up)))

    def halo_unpack(self, from_below, from_above):
        _check(self.lib.ddflb_halo_unpack(self._h, _dptr(from_below), _dptr(from_above)))

    def close(self):
        if getattr(self, "_h", None):
            self.lib.ddflb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SlabLattice:
    """One lattice divided into ``parts`` y-slabs held on one device (the
    decomposition a multi-GPU run uses, with the halo exchange done by one
    kernel): every step advances each slab, then refreshes all ghost rows.
    Bit-identical to the undivided Lattice."""

    def __init__(self, cfg: Config, parts: int, device=None, stream=None):
        from .distributed import slab_rows
        import torch
        self.torch = torch
        self.cfg = cfg
        self.lib = load()
        self.stream = stream or torch.cuda.current_stream(torch.device(device or "cuda"))
        self.rows = [slab_rows(cfg.ny, parts, k) for k in range(parts)]
        self.slabs = [Lattice(cfg, device=device, stream=self.stream, rows=r) for r in self.rows]
        self._hs = (_VP * parts)(*[s._h for s in self.slabs])
        self.t = 0

    def _split(self, a):
        return [None if a is None else a[..., y0:y0 + h, :] for y0, h in self.rows]

    def init(self, rho, ux, uy, phi, grads=None):
        parts = [self._split(None if a is None else self.slabs[0]._dev(a))
                 for a in (rho, ux, uy, phi, grads)]
        for k, s in enumerate(self.slabs):
            s.init(*[None if p is None else p[k] for p in parts])
        self.t = 0
        return self

    def step(self, n: int = 1):
        for _ in range(int(n)):
            for s in self.slabs:
                _check(self.lib.ddflb_step(s._h, 1))
            _check(self.lib.ddflb_halo_exchange_local(self._hs, len(self.slabs)))
            self.t += 1
        return self

    def fields(self, names=FIELD_NAMES) -> dict:
        parts = [s.fields(names) for s in self.slabs]
        return {k: self.torch.cat([p[k] for p in parts], dim=0) for k in parts[0]}

    def populations(self):
        parts = [s.populations() for s in self.slabs]
        return (self.torch.cat([p[0] for p in parts], dim=1),
                self.torch.cat([p[1] for p in parts], dim=1))

    def sums(self, mode: int = 0) -> dict:
        """Sums over the whole lattice (FP64, slab by slab)."""
        tot = {"mass_dev": 0.0, "scalar_dev": 0.0, "u2": 0.0, "du2": 0.0}
        for s in self.slabs:
            for k, v in s.sums(mode).items():
                tot[k] += v
        return tot


class Batch:
    """Independent lattice pairs of uneven sizes advanced together on the GPU
    (one persistent cooperative launch per chunk of steps)."""

    def __init__(self, cfgs, device=None, stream=None):
        import torch
        self.torch = torch
        self.cfgs = list(cfgs)
        self.n = len(self.cfgs)
        self.device = torch.device(device or "cuda")
        self.lib = load()
        self._p = (Params * self.n)(*[c.to_c() for c in self.cfgs])
        nbytes = self.lib.ddflb_batch_workspace_bytes(self.n, self._p)
        if nbytes == 0:
            _check(EINVAL)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        h = _VP()
        _check(self.lib.ddflb_batch_create(self.n, self._p, self.workspace.data_ptr(), nbytes,
                                           self.stream.cuda_stream, ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def set_run(self, tol=0.0, steps_per_launch=500, barrier_timeout_s=2.0, scalar_residual=False):
        _check(self.lib.ddflb_batch_set_run(self._h, float(tol), int(steps_per_launch),
                                            float(barrier_timeout_s), int(bool(scalar_residual))))
        return self

    def set_tiles(self, tile_x, tile_y, blocks_per_sm=0):
        _check(self.lib.ddflb_batch_set_tiles(self._h, tile_x, tile_y, blocks_per_sm))
        return self

    def set_schedule(self, schedule: int):
        """0: one persistent cooperative launch per chunk of steps (device-wide
        barrier between steps); 1: one launch per step and tile-per-CTA, the
        chunk captured as a graph.  Same results."""
        _check(self.lib.ddflb_batch_set_schedule(self._h, int(schedule)))
        return self

    def schedule(self) -> int:
        v = ctypes.c_int32()
        _check(self.lib.ddflb_batch_get_schedule(self._h, ctypes.byref(v)))
        return v.value

    def set_instance_run(self, i, tol=-1.0, max_steps=0):
        """Instance i's own tolerance (negative: the batch's) and step limit
        (0: none); a limited instance that has not converged is frozen with
        INST_CAPPED."""
        _check(self.lib.ddflb_batch_set_instance_run(self._h, int(i), float(tol), int(max_steps)))
        return self

    def tiles(self):
        v = [ctypes.c_int32() for _ in range(3)]
        _check(self.lib.ddflb_batch_get_tiles(self._h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def init(self, i, rho, ux, uy, phi, grads=None):
        t = self.torch
        dev = lambda a: None if a is None else (
            t.from_numpy(np.ascontiguousarray(a, np.float32)) if isinstance(a, np.ndarray) else a
        ).to(device=self.device, dtype=t.float32).contiguous()
        keep = [dev(a) for a in (rho, ux, uy, phi, grads)]
        self._keep[i] = keep
        _check(self.lib.ddflb_batch_init(self._h, int(i), *[_dptr(a) for a in keep]))
        return self

    def step(self, n=1):
        _check(self.lib.ddflb_batch_step(self._h, int(n)))
        return self

    def fields(self, i, names=FIELD_NAMES):
        c = self.cfgs[i]
        out = {k: (self.torch.empty((c.ny, c.nx), dtype=self.torch.float32, device=self.device)
                   if k in names else None) for k in FIELD_NAMES}
        _check(self.lib.ddflb_batch_fields(self._h, int(i), *[_dptr(out[k]) for k in FIELD_NAMES]))
        return {k: v for k, v in out.items() if v is not None}

    def stats(self):
        r = np.zeros(self.n, np.float64)
        f = np.zeros(self.n, np.int32)
        s = np.zeros(self.n, np.int64)
        t = np.zeros(self.n, np.int64)
        i0 = np.zeros(self.n, np.int64)
        st = self.lib.ddflb_batch_stats(self._h, r.ctypes.data, f.ctypes.data, s.ctypes.data,
                                        t.ctypes.data, i0.ctypes.data)
        return {"residual": r, "flags": f, "steps_to_tol": s, "state_time": t, "init_time": i0,
                "status": st}

    def debug_skip_barrier(self, block):
        _check(self.lib.ddflb_batch_debug_skip_barrier(self._h, int(block)))
        return self

    def autotune(self, trial_steps=20, cache=True):
        """Pick tile shape and residency (cached by workload signature); must
        run before any init (it overwrites every instance's state)."""
        from . import tuning
        key = tuning.key("batch", self.cfgs)
        hit = tuning.lookup(key) if cache else None
        if hit and len(hit["choice"]) == 4:
            self.set_schedule(hit["choice"][3])
            return self.set_tiles(*hit["choice"][:3]), hit
        v = [ctypes.c_int32() for _ in range(3)]
        ms = ctypes.c_double()
        _check(self.lib.ddflb_batch_autotune(self._h, int(trial_steps),
                                             *[ctypes.byref(x) for x in v], ctypes.byref(ms)))
        rec = {"choice": [x.value for x in v] + [self.schedule()], "ms_per_step": ms.value}
        if cache:
            tuning.store(key, rec)
        return self, rec

    def close(self):
        if getattr(self, "_h", None):
            self.lib.ddflb_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
