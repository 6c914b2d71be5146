"""Warm-start preparation on the device (ddflb_warm_fields): the network's
prediction becomes the init fields and gradients without a host round trip.
Checked bit for bit against a float32 numpy restatement (the same operations
in the same order: np.gradient's central / one-sided differences, the S_xy /
omega split), then fed to the init through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1908_06742_gb300 import build as B
from paper_1908_06742_gb300 import ddflb as D
from tests.gpu_helpers import np64

pytestmark = pytest.mark.gpu

OMEGA_SCALE = 20.0


@pytest.fixture(scope="module", autouse=True)
def built():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    D.load()


def numpy_warm(pred, U, n):
    """float32 restatement: u = U p0, U p1; phi = clip(p2, 0, 1);
    omega = p3 * scale * U / n; rho = 1 + p4 U U; gradients by np.gradient
    (central inside, one-sided at the edges); d_x u_y, d_y u_x = S_xy +- omega / 2."""
    U = np.float32(U)
    ux = pred[..., 0] * U
    uy = pred[..., 1] * U
    phi = np.clip(pred[..., 2], np.float32(0), np.float32(1))
    om = pred[..., 3] * np.float32(OMEGA_SCALE) * U / np.float32(n)
    rho = np.float32(1) + pred[..., 4] * U * U
    dyux, dxux = np.gradient(ux)
    dyuy, dxuy = np.gradient(uy)
    sxy = np.float32(0.5) * (dxuy + dyux)
    dxuy, dyux = sxy + np.float32(0.5) * om, sxy - np.float32(0.5) * om
    dyphi, dxphi = np.gradient(phi)
    return rho, ux, uy, phi, np.stack([dxux, dyux, dxuy, dyuy, dxphi, dyphi])


@pytest.mark.parametrize("n", [2, 37, 256, 300])
def test_warm_fields_match_numpy(n):
    rng = np.random.default_rng(n)
    pred = rng.standard_normal((n, n, 8)).astype(np.float32)
    pred[..., 2] = rng.uniform(-0.2, 1.2, (n, n)).astype(np.float32)   # clipping exercised
    U = 0.0734
    got = D.warm_fields(torch.from_numpy(pred).cuda(), U, OMEGA_SCALE)
    want = numpy_warm(pred, U, n)
    for g, w in zip(got, want):
        w = np.asarray(w, np.float32)
        assert g.dtype == torch.float32
        assert np.array_equal(g.cpu().numpy(), w), float(np.abs(g.cpu().numpy() - w).max())


def test_warm_fields_feed_init_without_host_copy():
    """The device planes go straight into ddflb_init; the populations equal
    those of an init from the same fields uploaded from the host."""
    n = 64
    rng = np.random.default_rng(3)
    pred = (0.3 * rng.standard_normal((n, n, 8))).astype(np.float32)
    pred[..., 2] = rng.uniform(0, 1, (n, n)).astype(np.float32)
    U = 0.08
    cfg = D.Config(nx=n, ny=n, bc="cavity", u_lid=U, phi_lid=1.0, phi_wall=0.0, nu=0.05,
                   diffusivity=0.05)
    dev = D.warm_fields(torch.from_numpy(pred).cuda(), U, OMEGA_SCALE)
    a = D.Lattice(cfg).init(*dev)
    b = D.Lattice(cfg).init(*[np.ascontiguousarray(x) for x in numpy_warm(pred, U, n)])
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert torch.equal(fa, fb) and torch.equal(ga, gb)


def test_warm_fields_argument_errors():
    p = torch.zeros((8, 8, 4), device="cuda")
    out = torch.empty((10, 8, 8), device="cuda")
    lib = D.load()
    ptrs = [out[i].data_ptr() for i in range(5)]
    with pytest.raises(D.DdflbError, match="channel stride"):
        D._check(lib.ddflb_warm_fields(p.data_ptr(), 8, 8, 4, 0.1, 20.0, 0.0, 1.0, *ptrs, None))
    with pytest.raises(D.DdflbError, match="u_lid"):
        D._check(lib.ddflb_warm_fields(p.data_ptr(), 8, 8, 5, 0.0, 20.0, 0.0, 1.0, *ptrs, None))
    with pytest.raises(D.DdflbError, match="NULL"):
        D._check(lib.ddflb_warm_fields(None, 8, 8, 5, 0.1, 20.0, 0.0, 1.0, *ptrs, None))
