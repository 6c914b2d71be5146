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

    # same tolerances as the stats parity test
    assert abs(a[0] - ref_prev["mass"]) < 1e-6 and abs(a[1] - ref_prev["scalar"]) < 1e-6
    assert math.isnan(a[3])
    assert abs(b[0] - ref["mass"]) < 1e-6 and abs(b[1] - ref["scalar"]) < 1e-6
    assert ref["residual"] > 0
    # the no-allocation call reports the raw ratio against its snapshot; the
    # library divides it by the check interval
    assert abs(b[3] / k - ref["residual"]) <= 0.02 * ref["residual"], (b[3], ref["residual"])
    assert b[2] > 0

    # sizes beyond the scratch are rejected with a clear message, nothing launched
    big = D.Config(nx=2048, ny=1024, bc="periodic")
    with pytest.raises(D.DdflbError, match="at most"):
        D.reduce_noalloc(big, s_now, 0, out1)
