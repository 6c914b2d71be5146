"""ddflb_reduce_noalloc: the reductions for callers that cannot allocate device
memory at the point of the call (code where cudaMalloc is not allowed, plug-ins
that are handed only existing buffers).  Its scratch is a fixed device array
inside the library, so the only memory the caller passes is the state to reduce
and four output doubles.

Checked against the existing entry point (ddflb_stats after ddflb_step's own
residual check) on two calls in a row: the first stores the velocity snapshot,
the second reduces the next state and measures the residual against it.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1908_06742_gb300 import build as B
from paper_1908_06742_gb300 import ddflb as D
from paper_1908_06742_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_reduce_noalloc_matches_stats():
    assert torch.cuda.is_available(), "GPU test"
    B.build()
    D.load()
    n, k = 96, 50
    rate = 1.0 / (3 * 0.064 + 0.5)
    cfg = D.Config(nx=n, ny=n, bc="cavity", u_lid=0.1, phi_lid=1.0, phi_wall=0.0,
                   omega_f=(0, 0, 0, 1.2, rate, rate, 1.2, 1.2, 1.2),
                   omega_g=(0, rate, rate, 1.2, 1.2, 1.2, 1.2, 1.2, 1.2), check_every=k)
    F = inputs.rest(n, n, phi=0.5)
    lat = D.Lattice(cfg).init(F.rho, F.ux, F.uy, F.phi).step(k)
    ref_prev = lat.stats()                      # t = k
    s_prev, _ = lat.get_state()
    s_prev = s_prev.clone()
    lat.step(k)                                 # t = 2k: the library's own residual check
    ref = lat.stats()                           # residual = |u(2k) - u(k)| / (k |u(2k)|)
    s_now, _ = lat.get_state()
    s_now = s_now.clone()

    out1 = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    out2 = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    D.reduce_noalloc(cfg, s_prev, 2, out1)      # first call: sums + store the snapshot
    D.reduce_noalloc(cfg, s_now, 1, out2)       # second call: sums + residual vs snapshot
    torch.cuda.synchronize()
    a, b = out1.cpu().numpy(), out2.cpu().numpy()

    # Both sides run the same reduction kernels, with the same fixed summation
    # order, on the same states: the sums agree to the last bits.
    assert abs(a[0] - ref_prev["mass"]) <= 1e-12 * abs(ref_prev["mass"])
    assert abs(a[1] - ref_prev["scalar"]) <= 1e-12 * abs(ref_prev["scalar"])
    assert math.isnan(a[3])
    assert abs(b[0] - ref["mass"]) <= 1e-12 * abs(ref["mass"])
    assert abs(b[1] - ref["scalar"]) <= 1e-12 * abs(ref["scalar"])
    assert ref["residual"] > 0
    # the no-allocation call reports the raw ratio |u(2k) - u(k)| / |u(2k)|
    # against its snapshot; the library divides it by the check interval k
    assert abs(b[3] / k - ref["residual"]) <= 1e-12 * ref["residual"], (b[3], ref["residual"])
    # sum |u|^2 against the velocity the library's fields report (the same FP32
    # values, summed in FP64 in another order)
    f = lat.fields()
    u2 = float(np.sum(f["ux"].double().cpu().numpy() ** 2 + f["uy"].double().cpu().numpy() ** 2))
    assert u2 > 0 and abs(b[2] - u2) <= 1e-12 * u2, (b[2], u2)

    # sizes beyond the scratch are rejected with a clear message, nothing launched
    big = D.Config(nx=2048, ny=1024, bc="periodic")
    with pytest.raises(D.DdflbError, match="at most"):
        D.reduce_noalloc(big, s_now, 0, out1)

    # a snapshot is tied to its grid: one stored on 96 x 96 does not serve a
    # 48 x 192 state of the same node count
    tall = D.Config(nx=48, ny=192, bc="cavity", u_lid=0.1, phi_lid=1.0, phi_wall=0.0,
                    omega_f=cfg.omega_f, omega_g=cfg.omega_g)
    Ft = inputs.rest(48, 192, phi=0.5)
    s_tall, _ = D.Lattice(tall).init(Ft.rho, Ft.ux, Ft.uy, Ft.phi).step(3).get_state()
    D.reduce_noalloc(cfg, s_now, 2, out1)
    with pytest.raises(D.DdflbError, match="48 x 192"):
        D.reduce_noalloc(tall, s_tall, 1, out2)
    D.reduce_noalloc(tall, s_tall, 2, out2)     # storing its own snapshot works
    D.reduce_noalloc(tall, s_tall, 1, out2)
    torch.cuda.synchronize()
    assert out2[3].item() == 0.0
