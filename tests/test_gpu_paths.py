"""The two step-kernel variants for 16-bit storage (one node per thread, and
two adjacent nodes per thread with aligned pair accesses) give bit-identical
states on every boundary kind and on ragged sizes that end mid-warp; odd nx
falls back to the one-node kernel; the default path for 16-bit storage is the
paired kernel."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1908_06742_gb300 import build as B
from paper_1908_06742_gb300 import ddflb as D
from paper_1908_06742_gb300 import inputs
from tests.gpu_helpers import gpu_config, spec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    D.load()


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
@pytest.mark.parametrize("bc", ["periodic", "cavity", "channel"])
@pytest.mark.parametrize("shape", [(200, 77), (130, 66), (2, 5), (66, 3), (131, 40)])
def test_pair_kernel_bit_identical(storage, bc, shape):
    nx, ny = shape
    s = spec(nx, ny, bc=bc, nu=0.05, D_phi=0.02, u_lid=0.05, phi_lid=1.3, phi_wall=0.7,
             storage=storage, scale=2.0 ** 10 if storage == "fp16" else 0.0)
    F = inputs.random_state(nx, ny, seed=nx * 3 + ny)
    out = []
    for path, block in ((1, (128, 1)), (2, (32, 4))):
        lat = D.Lattice(gpu_config(s)).set_path(path)
        D._check(lat.lib.ddflb_set_block(lat._h, *block))
        lat.init(F.rho, F.ux, F.uy, F.phi, F.grads).step(7)
        out.append(lat.populations())   # every node (the raw buffer's row padding is never written)
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
@pytest.mark.parametrize("shape,bc", [((200, 77), "periodic"), ((132, 66), "periodic"),
                                      ((4, 5), "periodic"), ((1024, 33), "periodic"),
                                      ((130, 40), "periodic"), ((200, 50), "cavity"),
                                      ((256, 37), "cavity"), ((4, 3), "cavity"), ((8, 2), "cavity"),
                                      ((132, 66), "channel"), ((8, 2), "channel"),
                                      ((130, 9), "channel")])
def test_quad_kernel_bit_identical(storage, shape, bc):
    """Path 3 (four nodes per thread, nx a multiple of 4, node by node next to
    walls; otherwise the paired or one-node kernel) against path 1, 7 steps."""
    nx, ny = shape
    s = spec(nx, ny, bc=bc, nu=0.05, D_phi=0.02, u_lid=0.05, phi_lid=1.3, phi_wall=0.7,
             storage=storage, scale=2.0 ** 10 if storage == "fp16" else 0.0)
    F = inputs.random_state(nx, ny, seed=nx * 7 + ny)
    out = []
    for path in (1, 3):
        lat = D.Lattice(gpu_config(s)).set_path(path)
        lat.init(F.rho, F.ux, F.uy, F.phi, F.grads).step(7)
        out.append(lat.populations())
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


@pytest.mark.parametrize("bc,storage,check_every,f_omega", [
    ("cavity", "fp32", 100, 0.0), ("periodic", "fp16", 0, 0.0), ("channel", "bf16", 50, 0.0),
    ("periodic", "fp32", 0, 0.01)])
def test_step_graph_replay_matches_single_steps(bc, storage, check_every, f_omega):
    """ddflb_step(n) replays captured 64-step graphs between checks (no
    time-modulated force); n calls of ddflb_step(1) never do.  Same state,
    residual and step count, also across a change of step kernel mid-run."""
    nx, ny = 96, 40
    s = spec(nx, ny, bc=bc, nu=0.05, D_phi=0.02, u_lid=0.05, phi_lid=1.3, phi_wall=0.7,
             storage=storage, scale=2.0 ** 10 if storage == "fp16" else 0.0,
             check_every=check_every, fx=1e-5 if f_omega else 0.0, f_omega=f_omega)
    F = inputs.random_state(nx, ny, seed=31)
    a = D.Lattice(gpu_config(s)).init(F.rho, F.ux, F.uy, F.phi, F.grads)
    b = D.Lattice(gpu_config(s)).init(F.rho, F.ux, F.uy, F.phi, F.grads)
    a.step(1000)
    for _ in range(1000):
        b.step(1)
    a.set_path(1).step(300)
    b.set_path(1)
    for _ in range(300):
        b.step(1)
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert torch.equal(fa, fb) and torch.equal(ga, gb)
    sa, sb = a.stats(), b.stats()
    assert sa["step"] == sb["step"] == 1300
    if check_every:
        assert sa["residual"] == sb["residual"]


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_default_path_for_16bit_storage_is_the_pair_kernel(storage):
    """Path 0 (default) steps 16-bit lattices with the paired kernel: same
    state as path 2 and as path 1, on a lattice with an odd-width wrap."""
    nx, ny = 130, 41
    s = spec(nx, ny, nu=0.05, D_phi=0.02, storage=storage,
             scale=2.0 ** 10 if storage == "fp16" else 0.0)
    F = inputs.random_state(nx, ny, seed=17)
    out = []
    for path in (0, 1, 2):
        lat = D.Lattice(gpu_config(s)).set_path(path)
        lat.init(F.rho, F.ux, F.uy, F.phi, F.grads).step(9)
        out.append(lat.populations())
    for k in (1, 2):
        assert torch.equal(out[0][0], out[k][0]) and torch.equal(out[0][1], out[k][1])


def test_pair_kernel_matches_oracle_emulation_scale():
    """The paired kernel at the benchmark's FP16 settings (scale 2^10) stays on
    the FP16 storage floor for a Taylor-Green lattice (u within 2e-3)."""
    n = 64
    s = spec(n, n, storage="fp16", scale=2.0 ** 10)
    F = inputs.taylor_green(n, 0.01, phi_amp=0.1)
    a = D.Lattice(gpu_config(s)).set_path(2).init(F.rho, F.ux, F.uy, F.phi, F.grads).step(200)
    b = D.Lattice(gpu_config(s)).set_path(1).init(F.rho, F.ux, F.uy, F.phi, F.grads).step(200)
    fa, fb = a.fields(), b.fields()
    for k in D.FIELD_NAMES:
        assert torch.equal(torch.nan_to_num(fa[k], 9.0), torch.nan_to_num(fb[k], 9.0)), k


# --------------------------------------------------------------- host I/O pipeline
def test_pipelined_host_io_matches_synchronous():
    """Three rounds of init_host -> steps -> fields_host_async with the copies on
    an I/O stream (each round with different inputs, results read only after
    the last round's io_wait for the final round) give the same fields as the
    synchronous path round by round."""
    import torch
    n, steps = 96, 40
    cfg = D.Config(nx=n, ny=n, nu=0.02, host_io=True)
    ins = []
    for r in range(3):
        F = inputs.taylor_green(n, 0.01 * (r + 1), phi_amp=0.1)
        ins.append([torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()
                    for a in (F.rho, F.ux, F.uy, F.phi, F.grads)])
    ref = []
    a = D.Lattice(cfg)
    for h in ins:
        out = {k: torch.empty((n, n)).pin_memory() for k in D.FIELD_NAMES}
        a.init_host(*h).step(steps).fields_host(out)
        ref.append({k: v.clone() for k, v in out.items()})
    b = D.Lattice(cfg).set_io_streams(torch.cuda.Stream(), torch.cuda.Stream())
    outs = [{k: torch.empty((n, n)).pin_memory() for k in D.FIELD_NAMES} for _ in ins]
    for h, out in zip(ins, outs):
        b.init_host(*h).step(steps).fields_host_async(out)
    b.io_wait()
    for r, (o, w) in enumerate(zip(outs, ref)):
        for k in D.FIELD_NAMES:
            assert torch.equal(o[k], w[k]), (r, k)
