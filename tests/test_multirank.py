"""The N > 1 launch path on CPU with gloo, world size 2 (no GPU): the
benchmark's rank helpers (barrier, max over ranks, per-rank instance draws for
weak scaling) and a torchrun launch of the reference arm, where rank 0 alone
prints the JSON line and the other rank exits 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_setup(None)
    assert (w, r) == (world, rank)
    bench.barrier(w)
    m = bench.max_over_ranks(w, float(rank + 1) * 1.5)
    from paper_1908_06742_gb300 import inputs
    draws = inputs.cavity_batch(8, seed=rank)   # what rank r advances in the batched workload
    out[rank] = (m, [d["n"] for d in draws], [round(d["re"], 6) for d in draws])
    dist.destroy_process_group()


def test_rank_helpers_gloo():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 3.0           # max over ranks
    assert out[0][2] != out[1][2]                  # each rank draws its own instances


def test_torchrun_reference_arm_two_ranks():
    env = dict(os.environ)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


# ------------------------------------------------------------------ partition
def test_shard_indices_partition():
    """Every instance belongs to exactly one rank, for any world size."""
    from paper_1908_06742_gb300.distributed import shard_indices
    for world in (1, 2, 3, 5, 8):
        parts = [shard_indices(512, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(512))
        assert max(map(len, parts)) - min(map(len, parts)) <= 1


def _cavity_params(n, re):
    import oracle as O
    U = 0.1
    return O.OracleParams(nx=n, ny=n, bc="cavity", u_lid=U, phi_lid=1.0, phi_wall=0.0,
                          omega_nu=O.omega_from_diffusivity(U * n / re), omega_bulk=1.2,
                          omega_hi=1.2, omega_phi=O.omega_from_diffusivity(U * n / re),
                          omega_phi_hi=1.2)


def _instance_sums(d, steps):
    """One batched cavity draw advanced by the oracle: its mass, scalar and
    sum |u|^2 (what the batch reports per instance)."""
    import oracle as O
    from paper_1908_06742_gb300 import inputs
    n = d["n"]
    F = inputs.rest(n, n, phi=0.0)
    L = O.OracleLattice(_cavity_params(n, d["re"])).init(F.rho, F.ux, F.uy, F.phi)
    s = L.step(steps).sums()
    return (s["mass"], s["scalar"], s["u2"])


def _batch_worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo")
    from paper_1908_06742_gb300 import inputs
    from paper_1908_06742_gb300.distributed import gather_indexed, shard_indices
    draws = inputs.cavity_batch(10, seed=0, sizes=(6, 8, 10))   # the same set on every rank
    mine = shard_indices(len(draws), rank, world)
    local = {i: _instance_sums(draws[i], 30) for i in mine}
    merged = gather_indexed(local, world)
    if rank == 0:
        out["merged"] = merged
        out["owned"] = {r: shard_indices(len(draws), r, world) for r in range(world)}
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_batch_partition_and_gather_gloo(world):
    """Rank r advances instances r, r + N, ... of the seed-0 draw; rank 0
    gathers the per-instance results in global order, equal to one rank
    advancing all of them."""
    from paper_1908_06742_gb300 import inputs
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_batch_worker, args=(world, free_port(), out), nprocs=world, join=True)
    draws = inputs.cavity_batch(10, seed=0, sizes=(6, 8, 10))
    single = [_instance_sums(d, 30) for d in draws]
    assert out["merged"] == single          # bit-identical, in global order
    owned = sorted(i for v in out["owned"].values() for i in v)
    assert owned == list(range(len(draws)))


# ------------------------------------------------------------------ data-parallel gradients
def _grad_worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo")
    import numpy as np
    from oracle import unet as U
    from paper_1908_06742_gb300.distributed import average_gradients, shard_indices
    r = np.random.default_rng(0)
    P = U.init_params(4, 3, 2, seed=1)
    X = r.standard_normal((4 * world, 8, 8, 3))         # the global batch
    T = r.standard_normal((4 * world, 8, 8, 2))
    mine = shard_indices(X.shape[0], rank, world)
    o, a = U.forward(P, X[mine])
    G = U.backward(P, a, o, T[mine])
    names = sorted(G)
    ts = [torch.from_numpy(np.ascontiguousarray(G[k][j])) for k in names for j in (0, 1)]
    average_gradients(ts, world)
    if rank == 0:
        out["avg"] = [t.numpy().copy() for t in ts]
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_gradient_allreduce_equals_global_batch_gloo(world):
    """Each rank takes its part of a global batch through the FP64 network
    oracle; after the gradient average every rank holds the gradient of the
    loss over the whole batch (one process computing it directly)."""
    import numpy as np
    from oracle import unet as U
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_grad_worker, args=(world, free_port(), out), nprocs=world, join=True)
    r = np.random.default_rng(0)
    P = U.init_params(4, 3, 2, seed=1)
    X = r.standard_normal((4 * world, 8, 8, 3))
    T = r.standard_normal((4 * world, 8, 8, 2))
    o, a = U.forward(P, X)
    G = U.backward(P, a, o, T)
    ref = [G[k][j] for k in sorted(G) for j in (0, 1)]
    for got, want in zip(out["avg"], ref):
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15 * np.abs(want).max())


# ------------------------------------------------------------------ y-slab halo exchange
def _slab_worker(rank, world, port, bc, nx, ny, steps, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo")
    import numpy as np
    import oracle as O
    from paper_1908_06742_gb300 import inputs
    from paper_1908_06742_gb300.distributed import (allreduce_sums, gather_indexed, halo_exchange,
                                                    slab_rows)
    p = _slab_params(bc, nx, ny)
    F = inputs.random_state(nx, ny, seed=5)
    full = O.OracleLattice(p).init(F.rho, F.ux, F.uy, F.phi, F.grads)   # t = 0 of the whole lattice
    y0, h = slab_rows(ny, world, rank)
    periodic = bc == "periodic"
    lo = 1 if (periodic or rank > 0) else 0          # ghost rows of this rank's slab
    hi = 1 if (periodic or rank < world - 1) else 0
    # the rank's slab plus ghost rows, as a lattice of the same boundary kind:
    # the owned rows pull only from the ghost rows, never from the fake walls or
    # wrap beyond them
    q = _slab_params(bc, nx, h + lo + hi)
    ext = O.OracleLattice(q)
    f = np.zeros((9, h + lo + hi, nx)); g = np.zeros_like(f)
    f[:, lo:lo + h] = full.f[:, y0:y0 + h]; g[:, lo:lo + h] = full.g[:, y0:y0 + h]
    for _ in range(steps):
        # pre-collision state (both lattices, all 9 populations) of the owned
        # boundary rows goes to the neighbours, whose ghost rows collide it
        down = torch.from_numpy(np.stack([f[:, lo], g[:, lo]]).copy())
        up = torch.from_numpy(np.stack([f[:, lo + h - 1], g[:, lo + h - 1]]).copy())
        from_below, from_above = halo_exchange(down, up, world, rank, periodic)
        if lo:
            f[:, 0], g[:, 0] = from_below[0].numpy(), from_below[1].numpy()
        if hi:
            f[:, -1], g[:, -1] = from_above[0].numpy(), from_above[1].numpy()
        ext.set_state(f, g).step(1)
        f, g = ext.f.copy(), ext.g.copy()
    own = O.OracleLattice(_slab_params("periodic", nx, h)).set_state(
        f[:, lo:lo + h].copy(), g[:, lo:lo + h].copy())
    s = own.sums()
    tot = allreduce_sums([s["mass"], s["scalar"], s["u2"]], world)
    merged = gather_indexed({rank: (f[:, lo:lo + h].copy(), g[:, lo:lo + h].copy())}, world)
    if rank == 0:
        out["f"] = np.concatenate([m[0] for m in merged], axis=1)
        out["g"] = np.concatenate([m[1] for m in merged], axis=1)
        out["sums"] = tot
    dist.destroy_process_group()


def _slab_params(bc, nx, ny):
    import oracle as O
    return O.OracleParams(nx=nx, ny=ny, bc=bc, omega_nu=O.omega_from_diffusivity(0.05),
                          omega_bulk=1.2, omega_hi=1.2, omega_phi=O.omega_from_diffusivity(0.02),
                          omega_phi_hi=1.2, u_lid=0.05, phi_lid=1.3, phi_wall=0.7)


@pytest.mark.parametrize("bc,world", [("periodic", 2), ("periodic", 3), ("channel", 3),
                                      ("cavity", 2)])
def test_slab_halo_exchange_oracle_gloo(bc, world):
    """A lattice cut into y-slabs over CPU ranks (gloo), each advanced by the
    FP64 oracle with its ghost rows refreshed through the host halo exchange
    before every step: the gathered state equals the undivided oracle run bit
    for bit, and the FP64 all-reduced sums equal its sums.  World size 2 on a
    periodic lattice has one peer as both neighbours (message order decides)."""
    import numpy as np
    import oracle as O
    from paper_1908_06742_gb300 import inputs
    nx, ny, steps = 12, 11, 8
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_slab_worker, args=(world, free_port(), bc, nx, ny, steps, out), nprocs=world,
             join=True)
    F = inputs.random_state(nx, ny, seed=5)
    ref = O.OracleLattice(_slab_params(bc, nx, ny)).init(F.rho, F.ux, F.uy, F.phi, F.grads)
    ref.step(steps)
    assert np.array_equal(out["f"], ref.f) and np.array_equal(out["g"], ref.g)
    s = ref.sums()
    for got, want in zip(out["sums"], (s["mass"], s["scalar"], s["u2"])):
        assert abs(got - want) <= 1e-12 * abs(want)
