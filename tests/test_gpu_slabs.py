"""y-slab decomposition of one lattice (the locality of the collide-and-stream
update, Secs. 2-3): a lattice cut into slabs of rows that exchange 3
populations x 2 lattices x nx values per face after every step reproduces the
undivided lattice bit for bit.  Both exchange routes are covered: the one
kernel that copies between slabs held on one device, and pack -> (any
transport) -> unpack, the route of one slab per process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1908_06742_gb300 import build as B
from paper_1908_06742_gb300 import ddflb as D
from paper_1908_06742_gb300 import inputs
from paper_1908_06742_gb300.distributed import slab_rows
from tests.gpu_helpers import as_f32, gpu_config, spec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    D.load()


def make_spec(bc, nx, ny, storage="fp32", scale=0.0):
    return spec(nx, ny, bc=bc, nu=0.05, D_phi=0.02, u_lid=0.05, phi_lid=1.3, phi_wall=0.7,
                storage=storage, scale=scale)


def whole_run(s, F, steps, force=None):
    g = D.Lattice(gpu_config(s))
    if force is not None:
        g.set_force_field(force)
    return g.init(F.rho, F.ux, F.uy, F.phi, F.grads).step(steps)


@pytest.mark.parametrize("bc", ["periodic", "cavity", "channel"])
@pytest.mark.parametrize("parts", [2, 4])
@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_slabs_bit_identical_local_exchange(bc, parts, storage):
    """Random state with gradients on a ragged 70 x 45 lattice (uneven slab
    heights), 25 steps: every population, every field and the sums of the
    divided run equal the undivided run's."""
    nx, ny, steps = 70, 45, 25
    s = make_spec(bc, nx, ny, storage, 2.0 ** 10 if storage == "fp16" else 0.0)
    F = as_f32(inputs.random_state(nx, ny, seed=7 * parts + ny))
    whole = whole_run(s, F, steps)
    sl = D.SlabLattice(gpu_config(s), parts).init(F.rho, F.ux, F.uy, F.phi, F.grads).step(steps)
    fw, gw = whole.populations()
    fs, gs = sl.populations()
    assert torch.equal(fw, fs) and torch.equal(gw, gs)
    a, b = whole.fields(), sl.fields()
    for k in a:
        assert torch.equal(torch.nan_to_num(a[k], nan=7.0), torch.nan_to_num(b[k], nan=7.0)), k
    # FP64 sums over the slabs against the whole lattice's (other summation order)
    sw, ss = whole.sums(), sl.sums()
    for k in ("mass_dev", "scalar_dev", "u2"):
        assert abs(sw[k] - ss[k]) <= 1e-12 * max(abs(sw[k]), 1e-300) + 1e-16, (k, sw[k], ss[k])


@pytest.mark.parametrize("bc", ["periodic", "cavity", "channel"])
def test_slabs_pack_unpack_route(bc):
    """Three slabs stepped one by one with the halos packed into tensors,
    passed on, and unpacked (what the multi-process run does through NCCL):
    bit-identical to the undivided lattice after 12 steps; with a steady body
    force field split by rows and a single-row slab in the middle."""
    nx, ny, steps = 64, 21, 12
    s = make_spec(bc, nx, ny)
    s["fx"], s["fy"] = 1e-6, -2e-6
    F = as_f32(inputs.random_state(nx, ny, seed=31))
    force = np.random.default_rng(2).standard_normal((2, ny, nx)).astype(np.float32) * 1e-6
    whole = whole_run(s, F, steps, force=force)
    rows = [(0, 10), (10, 1), (11, 10)]
    cfg = gpu_config(s)
    slabs = []
    for y0, h in rows:
        L = D.Lattice(cfg, rows=(y0, h))
        L.set_force_field(force[:, y0:y0 + h])
        sl = (slice(y0, y0 + h),)
        L.init(F.rho[sl], F.ux[sl], F.uy[sl], F.phi[sl], F.grads[:, y0:y0 + h])
        slabs.append(L)
    n = slabs[0].halo_elems()
    assert n == 6 * nx
    periodic = bc == "periodic"
    P = len(slabs)
    for _ in range(steps):
        for L in slabs:
            L.step(1)
        down = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in slabs]
        up = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in slabs]
        for k, L in enumerate(slabs):
            has_below = periodic or k > 0
            has_above = periodic or k < P - 1
            L.halo_pack(down[k] if has_below else None, up[k] if has_above else None)
        for k, L in enumerate(slabs):
            below = (k - 1) % P if (periodic or k > 0) else None
            above = (k + 1) % P if (periodic or k < P - 1) else None
            L.halo_unpack(None if below is None else up[below],
                          None if above is None else down[above])
    fw, gw = whole.populations()
    fs = torch.cat([L.populations()[0] for L in slabs], dim=1)
    gs = torch.cat([L.populations()[1] for L in slabs], dim=1)
    assert torch.equal(fw, fs) and torch.equal(gw, gs)


def test_slab_residual_from_sums_matches_whole():
    """The residual a divided cavity computes from the slabs' FP64 sums (mode
    bit 2 stores the snapshot, K steps later bit 1 compares) equals the
    undivided lattice's own residual check."""
    n, K = 48, 40
    s = make_spec("cavity", n, n)
    s["check_every"] = K
    F = as_f32(inputs.rest(n, n, phi=0.5))
    whole = D.Lattice(gpu_config(s)).init(F.rho, F.ux, F.uy, F.phi).step(2 * K)
    r_whole = whole.stats()["residual"]
    s2 = dict(s)
    s2["check_every"] = 0
    sl = D.SlabLattice(gpu_config(s2), 3).init(F.rho, F.ux, F.uy, F.phi)
    sl.step(K)
    sl.sums(mode=2)
    sl.step(K)
    t = sl.sums(mode=1)
    r_slab = np.sqrt(t["du2"] / t["u2"]) / K
    assert r_whole > 0 and abs(r_slab - r_whole) <= 1e-12 * r_whole, (r_slab, r_whole)


def test_slab_argument_errors():
    """Rows outside the lattice, internal checks on a slab with ghost rows,
    several steps per call, mismatched slab sets: EINVAL, nothing launched."""
    cfg = gpu_config(make_spec("periodic", 32, 16))
    with pytest.raises(D.DdflbError, match="outside"):
        D.Lattice(cfg, rows=(10, 8))
    s = make_spec("periodic", 32, 16)
    s["check_every"] = 10
    with pytest.raises(D.DdflbError, match="check_every"):
        D.Lattice(gpu_config(s), rows=(0, 8))
    a = D.Lattice(cfg, rows=(0, 8))
    with pytest.raises(D.DdflbError, match="one step"):
        a.step(2)
    b = D.Lattice(cfg, rows=(8, 8))
    lib = D.load()
    hs = (D._VP * 2)(b._h, a._h)                      # wrong order
    with pytest.raises(D.DdflbError, match="starts at row"):
        D._check(lib.ddflb_halo_exchange_local(hs, 2))
    whole = D.Lattice(cfg, rows=(0, 16))              # the whole lattice: no ghost rows
    with pytest.raises(D.DdflbError, match="neighbouring slab"):
        whole.halo_pack(torch.empty(6 * 32, dtype=torch.int32, device="cuda"), None)
    assert slab_rows(16, 3, 0) == (0, 6) and slab_rows(16, 3, 2) == (11, 5)
