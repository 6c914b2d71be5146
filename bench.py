"""Throughput benchmark of the fused DDF lattice Boltzmann step on GB300.

One benchmark step = one run of the throughput workload: ``--lb-steps`` fused
time steps of a Taylor-Green lattice pair (flow + scalar, D2Q9 each) followed by
the local strain-rate / vorticity fields of the final state.  Prints one JSON
line (rank 0).  ``--impl reference`` times the FP64 CPU checker on a bounded
sample of the same workload instead.

Launch: ``python bench.py [--gpus N --steps K --warmup W]``; for N > 1 under
torch.distributed.run, every rank advances its own lattice (replicas, weak
scaling) and the slowest rank's time counts.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DDF-LB MLUPS with local ω/S, % of HBM peak; surrogate steps-to-steady saved"
BYTES_PER_CELL = {"fp32": 144, "fp16": 72, "bf16": 72}  # 18 populations read + written


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=16384, help="grid side of the Taylor-Green lattice")
    ap.add_argument("--lb-steps", type=int, default=200, help="fused time steps per benchmark step")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--step-path", type=int, default=0, choices=[0, 1, 2, 3],
                    help="step kernel (ddflb_set_path): 0 default (groups of 4 nodes for "
                         "16-bit storage), 1 one node per thread, 2 node pairs, 3 groups of 4")
    ap.add_argument("--scalar-model", default="mrt", choices=["mrt", "srt", "cascaded", "central"],
                    help="scalar collision (Sec. 3 MRT, App. B SRT, App. C cascaded, App. D central)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="tg",
                    choices=["tg", "sweep", "batch", "cavity", "surrogate", "gemm", "slabs",
                             "conv"],
                    help="tg: Taylor-Green throughput point; sweep: Taylor-Green at N = 1024, "
                         "4096, 8192, 16384 for each storage; batch: 512 uneven cavities; "
                         "cavity: 256^2 cavities run to steady state; slabs: one lattice "
                         "divided into y-slabs, one per rank, halos exchanged every step")
    ap.add_argument("--instances", type=int, default=512)
    ap.add_argument("--schedule", default="auto", choices=["auto", "0", "1"],
                    help="batch: launch schedule (0 persistent, 1 one launch per step; auto: "
                         "the autotuner's choice over both)")
    ap.add_argument("--tiles", default="64x4", help="batch tile shape when --schedule is not auto")
    ap.add_argument("--boot", type=int, default=0,
                    help="surrogate: training draws run from rest before a first network "
                         "warm-starts the remaining ones (0: all from rest)")
    ap.add_argument("--conv-path", type=int, default=0, choices=[0, 1],
                    help="conv workload: 0 halo bands where W is a multiple of 128 and C >= 128, "
                         "1 one box per tap everywhere")
    ap.add_argument("--gemm-shape", default=None,
                    help="gemm workload: one M,N,K,splits shape instead of the U-Net set")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = str(device_index)
        try:  # nvidia-smi numbering can differ from CUDA's: select by PCI bus id
            import torch
            pr = torch.cuda.get_device_properties(device_index)
            self.idx = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
        except Exception:
            pass
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v: float) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, v: float) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_to_rank0(world, obj):
    """Python objects of every rank, in rank order, on rank 0 (None elsewhere)."""
    if world == 1:
        return [obj]
    import torch.distributed as dist
    out = [None] * world
    dist.all_gather_object(out, obj)
    return out


def rates(nu):
    w = 1.0 / (3.0 * nu + 0.5)  # nu = c_s^2 (1/omega - 1/2), c_s^2 = 1/3
    return (0, 0, 0, 1.2, w, w, 1.2, 1.2, 1.2), (0, w, w, 1.2, 1.2, 1.2, 1.2, 1.2, 1.2)


def workload_name(args):
    model = "" if args.scalar_model == "mrt" else f" ({args.scalar_model} scalar collision)"
    return (f"taylor-green {args.n}x{args.n}, D2Q9 flow + scalar{model}, {args.storage} storage, "
            f"{args.lb_steps} fused steps + local S/omega fields per benchmark step")


# ------------------------------------------------------------------ CPU checker
def cpu_sample(seconds: float = 12.0, n: int = 1024, lb_per_call: int = 2):
    """Time the FP64 checker on Taylor-Green n^2 (the sweep's error-reference
    size) for about ``seconds``: returns (MLUPS, cores, description)."""
    import oracle as O
    from paper_1908_06742_gb300 import inputs
    cores = O.threads(os.cpu_count() or 1)
    wf, wg = rates(0.01)
    F = inputs.taylor_green(n, 0.01, phi_amp=0.1)
    L = O.OracleLattice(O.OracleParams(nx=n, ny=n, lam_override=wf, lam_phi_override=wg))
    L.init(F.rho, F.ux, F.uy, F.phi, F.grads)
    L.step(1)
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        L.step(lb_per_call)
        done += lb_per_call
    L.fields()
    dt = time.perf_counter() - t0
    return n * n * done / dt / 1e6, cores, f"FP64 checker, taylor-green {n}x{n}, {done} steps + fields, {dt:.1f} s"


def run_reference(args, world, rank):
    """The reference arm: the FP64 CPU checker on a bounded sample per step."""
    if rank != 0:
        return
    import oracle as O
    from paper_1908_06742_gb300 import inputs
    cores = O.threads(os.cpu_count() or 1)
    n, lb = 1024, 4
    wf, wg = rates(0.01)
    F = inputs.taylor_green(n, 0.01, phi_amp=0.1)
    L = O.OracleLattice(O.OracleParams(nx=n, ny=n, lam_override=wf, lam_phi_override=wg))
    L.init(F.rho, F.ux, F.uy, F.phi, F.grads)
    for _ in range(args.warmup):
        L.step(lb); L.fields()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        L.step(lb); L.fields()
    dt = time.perf_counter() - t0
    v = n * n * lb * args.steps / dt / 1e6
    sample = f"FP64 checker, taylor-green {n}x{n}, {lb} steps + fields per benchmark step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args), "sample": sample},
        "cpu_baseline": {"value": round(v, 3), "unit": "MLUPS", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(v, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------ GPU arm
def step_kernel_name(args):
    """The step kernel the Taylor-Green context runs for --step-path (the
    paired kernel takes 16-bit storage, even n and the MRT / SRT scalar)."""
    if (args.step_path in (0, 3) and args.storage != "fp32" and args.n % 4 == 0
            and args.scalar_model in ("mrt", "srt")):
        return "k_step_quad"
    # the Taylor-Green lattice is periodic: there the default takes pairs when
    # n is not a multiple of 4
    pair = args.step_path in (2, 3) or (args.step_path == 0 and args.storage != "fp32")
    if pair and args.storage != "fp32" and args.n % 2 == 0 and args.scalar_model in ("mrt", "srt"):
        return "k_step_pair"
    return "k_step"


def traffic_per_launch(args, n_cells):
    """DRAM bytes per step-kernel launch from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    return traffic_record(f"{step_kernel_name(args)}_{args.storage}" + (
        "" if args.scalar_model == "mrt" else f"_{args.scalar_model}"), n_cells)


def traffic_record(key, n_units):
    """DRAM bytes per node (node-step for the batch) recorded by ncu in
    profiles/traffic.json under `key`, times n_units; None if there is no record
    or the kernel sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        import hashlib
        e = d.get(key)
        if not e:
            return None
        h = hashlib.sha256()
        for s in e["source_files"]:
            with open(os.path.join(ROOT, s), "rb") as fh:
                h.update(fh.read())
        if e.get("source_sha256") != h.hexdigest():
            return None
        return e["dram_bytes_per_cell"] * n_units
    except Exception:
        return None


def traffic_source(key, units):
    """Where the traffic figure comes from: the ncu capture recorded under key,
    per cell, scaled to this launch."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            e = json.load(f).get(key)
    except Exception:
        e = None
    if not e:
        return None
    return (f"ncu dram__bytes_read.sum + dram__bytes_write.sum per cell on {e['measured_on']}; "
            f"x {units} (traffic grows in proportion to the cells a launch updates)")


def run_ours(args, world, rank, local):
    import torch
    from paper_1908_06742_gb300 import build as B
    from paper_1908_06742_gb300 import ddflb as D
    from paper_1908_06742_gb300 import inputs

    B.build()
    D.load()
    dev = torch.device("cuda", local)
    n, lb = args.n, args.lb_steps
    wf, wg = rates(0.01)
    cfg = D.Config(nx=n, ny=n, storage=args.storage, omega_f=wf, omega_g=wg,
                   scale_f=2.0 ** 10 if args.storage == "fp16" else 0.0,
                   scale_g=2.0 ** 10 if args.storage == "fp16" else 0.0,
                   host_io=not args.no_e2e, scalar_model=args.scalar_model)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        lat = D.Lattice(cfg, device=dev, stream=stream)
        if args.step_path:
            lat.set_path(args.step_path)
        T = inputs.taylor_green(n, 0.01, phi_amp=0.1, xp=torch, device=dev)
        f32 = [a.float() for a in (T.rho, T.ux, T.uy, T.phi, T.grads)]
        del T
        lat.init(*f32)
        outs = {k: torch.empty((n, n), dtype=torch.float32, device=dev) for k in D.FIELD_NAMES}
        fptrs = [outs[k].data_ptr() for k in D.FIELD_NAMES]
        lib = lat.lib

        def bench_step():
            D._check(lib.ddflb_step(lat._h, lb))
            D._check(lib.ddflb_fields(lat._h, *fptrs))

        for _ in range(args.warmup):
            bench_step()
        stream.synchronize()

        # timed region: K benchmark steps, events on the launching stream
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        clocks = ClockSampler(local)
        barrier(world)
        torch.cuda.synchronize(dev)
        clocks.start()
        t_host = time.perf_counter()
        for a, b, c in ev:
            a.record(stream)
            D._check(lib.ddflb_step(lat._h, lb))
            b.record(stream)
            D._check(lib.ddflb_fields(lat._h, *fptrs))
            c.record(stream)
        torch.cuda.synchronize(dev)
        t_host = time.perf_counter() - t_host
        barrier(world)
        clk = clocks.stop()
        total_ms = sum(a.elapsed_time(c) for a, _, c in ev)
        step_ms = sum(a.elapsed_time(b) for a, b, _ in ev)
        total_ms = max_over_ranks(world, total_ms)
        launches = args.steps * (lb + 1)

        cells = n * n
        value = world * cells * lb * args.steps / (total_ms / 1e3) / 1e6
        kernel_s = step_ms / 1e3 / (lb * args.steps)     # average k_step launch duration
        algo_bytes = BYTES_PER_CELL[args.storage] * cells
        peak, kind = peaks()
        achieved = algo_bytes / kernel_s / 1e9
        stats = lat.stats()

        # end to end through the C ABI with host buffers: copy in, init, steps, fields out
        e2e = None
        if not args.no_e2e:
            pin = lambda t: t.cpu().pin_memory()
            h_in = [pin(a) for a in f32]
            h_out = {k: torch.empty((n, n), dtype=torch.float32).pin_memory()
                     for k in D.FIELD_NAMES}
            del f32
            e2e_steps = max(1, args.steps)
            # host copies on their own stream: the upload of step k+1 and the
            # download of step k overlap with the time steps (ordered by events)
            lat.set_io_streams(torch.cuda.Stream(dev), torch.cuda.Stream(dev))
            lat.init_host(*h_in).step(lb)
            lat.fields_host(h_out)
            barrier(world)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                lat.init_host(*h_in)
                lat.step(lb)
                lat.fields_host_async(h_out)
            lat.io_wait()
            torch.cuda.synchronize(dev)
            dt = max_over_ranks(world, time.perf_counter() - t0)
            e2e = {"value": round(world * cells * lb * e2e_steps / dt / 1e6, 1), "unit": "MLUPS",
                   "h2d_bytes_per_step": int(sum(a.numel() * 4 for a in h_in)),
                   "d2h_bytes_per_step": int(8 * cells * 4), "steps": e2e_steps}

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu:
        v, cores, sample = cpu_sample()
        cpu = {"value": round(v, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": sample}
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(args), "grid": n, "lb_steps_per_step": lb,
                   "storage": args.storage, "parallelism": "replicas" if world > 1 else "single",
                   "l2": f"inputs larger than L2 ({algo_bytes / 2 / 1e9:.1f} GB of populations per buffer)",
                   "hbm_pct": round(100 * achieved / peak, 1)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_kind": kind,
                     "kernel": step_kernel_name(args),
                     "algorithmic_bytes_per_launch": algo_bytes,
                     "traffic": traffic_per_launch(args, cells),
                     "traffic_source": traffic_source(step_kernel_name(args) + "_" + args.storage
                                                      + ("" if args.scalar_model == "mrt"
                                                         else "_" + args.scalar_model),
                                                      "cells of this launch")},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "host_wall_s": round(t_host, 3),
        "checks": {"mass": stats["mass"], "diverged": stats["diverged"]},
    }
    print(json.dumps(line))


def batch_configs(args, rank, world):
    """512 lid-driven cavities (seed 0): size uniform over {64..512}, Re
    log-uniform in [100, 3200], Pe = Re, lid 0.1, FP32.  The instances are
    partitioned over ranks (rank r advances r, r + N, ...): strong scaling.
    Returns (global indices, configs) of this rank's instances."""
    from paper_1908_06742_gb300 import ddflb as D
    from paper_1908_06742_gb300 import inputs
    from paper_1908_06742_gb300.distributed import shard_indices
    draws = inputs.cavity_batch(args.instances, seed=0)
    mine = shard_indices(len(draws), rank, world)
    cfgs = []
    for d in (draws[i] for i in mine):
        n, U = d["n"], 0.1
        w = 1.0 / (3.0 * U * n / d["re"] + 0.5)          # nu = U L / Re, L = n
        wg = 1.0 / (3.0 * U * n / d["pe"] + 0.5)
        cfgs.append(D.Config(nx=n, ny=n, bc="cavity", u_lid=U, phi_lid=1.0, phi_wall=0.0,
                             omega_f=(0, 0, 0, 1.2, w, w, 1.2, 1.2, 1.2),
                             omega_g=(0, wg, wg, 1.2, 1.2, 1.2, 1.2, 1.2, 1.2),
                             check_every=100))
    return mine, cfgs


def run_batch(args, world, rank, local):
    import numpy as np
    import torch
    from paper_1908_06742_gb300 import build as B
    from paper_1908_06742_gb300 import ddflb as D
    from paper_1908_06742_gb300 import inputs

    B.build()
    D.load()
    dev = torch.device("cuda", local)
    from paper_1908_06742_gb300.distributed import gather_indexed
    lb = args.lb_steps if args.lb_steps != 200 else 1000
    mine, cfgs = batch_configs(args, rank, world)
    cells = sum(c.nx * c.ny for c in cfgs)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        b = D.Batch(cfgs, device=dev, stream=stream)
        b.set_run(tol=0.0, steps_per_launch=lb)
        if args.schedule == "auto":
            _, tune = b.autotune(trial_steps=20, cache=False)
        else:
            tx, ty = (int(v) for v in args.tiles.split("x"))
            b.set_schedule(int(args.schedule)).set_tiles(tx, ty)
            tune = {"choice": list(b.tiles()) + [b.schedule()], "forced": True}
        starts = [inputs.rest(c.nx, c.ny, phi=0.0) for c in cfgs]
        for i, F in enumerate(starts):
            b.init(i, F.rho, F.ux, F.uy, F.phi)
        for _ in range(args.warmup):
            b.step(lb)
        stream.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        clocks = ClockSampler(local)
        barrier(world)
        torch.cuda.synchronize(dev)
        clocks.start()
        for a, c in ev:
            a.record(stream)
            b.step(lb)
            c.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        clk = clocks.stop()
        local_ms = sum(a.elapsed_time(c) for a, c in ev)
        total_ms = max_over_ranks(world, local_ms)
        st = b.stats()
        job_cells = sum_over_ranks(world, float(cells))      # all 512 instances
        value = job_cells * lb * args.steps / (total_ms / 1e3) / 1e6
        peak, kind = peaks()
        # this rank's kernel against this GPU's copy peak
        achieved = 144 * cells * lb * args.steps / (local_ms / 1e3) / 1e9
        # per-instance flags of the whole job, in global order, on rank 0
        flags = gather_indexed({i: int(f) for i, f in zip(mine, st["flags"])}, world)
        e2e = None
        if not args.no_e2e:
            h_in = [{k: torch.from_numpy(np.ascontiguousarray(getattr(F, k), np.float32)).pin_memory()
                     for k in ("rho", "ux", "uy", "phi")} for F in starts]
            h_out = [torch.empty((c.ny, c.nx), dtype=torch.float32).pin_memory() for c in cfgs]
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for i in range(len(cfgs)):
                h = h_in[i]
                b.init(i, h["rho"], h["ux"], h["uy"], h["phi"])
            b.step(lb)
            for i in range(len(cfgs)):
                h_out[i].copy_(b.fields(i, names=("omega",))["omega"], non_blocking=True)
            torch.cuda.synchronize(dev)
            dt = max_over_ranks(world, time.perf_counter() - t0)
            e2e = {"value": round(job_cells * lb / dt / 1e6, 1), "unit": "MLUPS",
                   "h2d_bytes_per_step": int(16 * cells), "d2h_bytes_per_step": int(4 * cells),
                   "steps": 1}
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.instances} lid-driven cavities, sizes 64..512, Re "
                               f"log-uniform [100, 3200], Pe = Re, fp32, {lb} steps per "
                               f"benchmark step, residual check every 100 steps",
                   "parallelism": (f"instances partitioned over {world} ranks" if world > 1
                                   else "single"),
                   "cells": int(job_cells), "cells_rank0": cells, "tiles": tune,
                   "l2": f"{288 * cells / 1e9:.1f} GB of populations on rank 0"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_kind": kind,
                     "kernel": "k_batch" if tune["choice"][3] == 0 else "k_batch_tile",
                     # bytes per node-step from a 64-cavity capture, times this launch's
                     # node-steps (traffic grows in proportion: every node-step moves the
                     # same 18 planes)
                     "algorithmic_bytes_per_launch": 144 * cells * lb,
                     "traffic": traffic_record("k_batch_fp32", cells * lb),
                     "traffic_source": traffic_source("k_batch_fp32", "node-steps of this launch")},
        "cpu_baseline": None, "e2e": e2e,
        # schedule 0: one cooperative launch per chunk of lb steps; schedule 1: per
        # step the node kernel, the sums kernel and the check kernel, then the
        # state-time update
        "gpu_launches": args.steps * (1 if tune["choice"][3] == 0 else 3 * lb + 1),
        "clocks": clk,
        "checks": {"flags_nonzero": int(sum(f != 0 for f in flags)), "instances": len(flags),
                   "status": int(st["status"])},
    }
    print(json.dumps(line))


def run_cavity(args, world, rank, local):
    """Lid-driven cavities 256^2 at Re 100, 400, 1000 (lid 0.1, Pe = Re, phi = 1
    on the lid, 0 on the other walls), run until the velocity residual is below
    1e-8, with S and omega written every 1000 steps.  The three cavities are
    independent lattices, each on its own stream (their step graphs run
    concurrently); every 1000 steps each writes its fields and its residual is
    read.  One benchmark step = the whole run to steady state (or the step
    cap), timed on the host around the device work."""
    import torch
    from paper_1908_06742_gb300 import build as B
    from paper_1908_06742_gb300 import ddflb as D
    from paper_1908_06742_gb300 import inputs
    from paper_1908_06742_gb300.distributed import shard_indices

    B.build()
    D.load()
    dev = torch.device("cuda", local)
    n, U, res_all = 256, 0.1, (100.0, 400.0, 1000.0)
    cap, chunk = 4_000_000, 1000
    # the three cavities are independent: rank r advances cavities r, r + N, ...
    # (strong scaling: the job's work is fixed; ranks beyond the third idle)
    mine = shard_indices(len(res_all), rank, world)
    res = tuple(res_all[i] for i in mine)
    cfgs = []
    for re in res:
        w = 1.0 / (3.0 * U * n / re + 0.5)
        cfgs.append(D.Config(nx=n, ny=n, bc="cavity", u_lid=U, phi_lid=1.0, phi_wall=0.0,
                             omega_f=(0, 0, 0, 1.2, w, w, 1.2, 1.2, 1.2),
                             omega_g=(0, w, w, 1.2, 1.2, 1.2, 1.2, 1.2, 1.2),
                             check_every=chunk))
    streams = [torch.cuda.Stream(dev) for _ in cfgs]
    lats = []
    for c, st in zip(cfgs, streams):
        with torch.cuda.stream(st):
            lats.append(D.Lattice(c, device=dev, stream=st))
    out = [{k: torch.empty((n, n), device=dev) for k in ("sxx", "sxy", "syy", "omega")}
           for _ in cfgs]
    runs = []
    for rep in range(args.warmup + args.steps):
        if not cfgs:               # a rank without a cavity joins the collectives only
            barrier(world)         # (the same sequence as the ranks below)
            barrier(world)
            dt = max_over_ranks(world, 0.0)
            upd = sum_over_ranks(world, 0.0)
            if rep >= args.warmup:
                runs.append((dt, upd, [], []))
            continue
        F = inputs.rest(n, n, phi=0.0)
        for lat, st in zip(lats, streams):
            with torch.cuda.stream(st):
                lat.init(F.rho, F.ux, F.uy, F.phi)
        torch.cuda.synchronize(dev)
        steps, res_now = [0] * len(cfgs), [float("nan")] * len(cfgs)
        active = [True] * len(cfgs)
        barrier(world)
        t0 = time.perf_counter()
        while any(active):
            for i, (lat, st) in enumerate(zip(lats, streams)):
                if not active[i]:
                    continue
                with torch.cuda.stream(st):
                    lat.step(chunk)
                    o = out[i]   # S and omega every 1000 steps
                    D._check(lat.lib.ddflb_fields(lat._h, None, None, None, None,
                                                  o["sxx"].data_ptr(), o["sxy"].data_ptr(),
                                                  o["syy"].data_ptr(), o["omega"].data_ptr()))
                steps[i] += chunk
            for i, lat in enumerate(lats):
                if active[i]:
                    res_now[i] = lat.stats()["residual"]
                    if res_now[i] < 1e-8 or steps[i] >= cap:
                        active[i] = False
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        barrier(world)
        dt = max_over_ranks(world, dt)
        upd = sum_over_ranks(world, float(sum(steps) * n * n))   # whole-job node updates
        if rep >= args.warmup:
            runs.append((dt, upd, list(steps), list(res_now)))
    # per-cavity step counts and residuals of the last run, from every rank
    last = gather_to_rank0(world, list(zip(res, runs[-1][2], runs[-1][3])))
    if rank != 0:
        return
    dt = sum(r[0] for r in runs)
    upd = sum(r[1] for r in runs)
    per = sorted(x for part in last for x in part)
    res = tuple(x[0] for x in per)
    steps, res_now = [x[1] for x in per], [x[2] for x in per]
    line = {
        "metric": METRIC, "value": round(upd / dt / 1e6, 1), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / len(runs) * 1e3, 1),
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "lid-driven cavity 256x256, lid 0.1, Re 100/400/1000, Pe = Re, "
                               "fp32, run to residual < 1e-8, S and omega every 1000 steps; three "
                               "lattices on three streams",
                   "parallelism": "cavities partitioned over ranks" if world > 1 else "single",
                   "l2": "9.4 MB of populations per cavity: L2-resident",
                   "timing": "host clock around the whole run to steady state"},
        "steps_to_steady": {str(int(r)): int(s) for r, s in zip(res, steps)},
        "final_residual": {str(int(r)): float(x) for r, x in zip(res, res_now)},
        "converged": [bool(x < 1e-8) for x in res_now],
    }
    print(json.dumps(line))


def run_slabs(args, world, rank, local):
    """One periodic Taylor-Green lattice of n x (n N) nodes divided into N
    y-slabs of n x n, one per rank (weak scaling).  Every time step each rank
    advances its slab, packs the 3 populations x 2 lattices x n values that
    cross each face, swaps them with its two neighbours (NCCL send/receive)
    and unpacks them into its ghost rows.  With N = 1 the slab is the whole
    lattice and nothing is exchanged."""
    import torch
    from paper_1908_06742_gb300 import build as B
    from paper_1908_06742_gb300 import ddflb as D
    from paper_1908_06742_gb300 import inputs
    from paper_1908_06742_gb300.distributed import allreduce_sums, halo_exchange

    B.build()
    D.load()
    dev = torch.device("cuda", local)
    n, lb = args.n, args.lb_steps
    ny = n * world
    wf, wg = rates(0.01)
    cfg = D.Config(nx=n, ny=ny, storage=args.storage, omega_f=wf, omega_g=wg,
                   scale_f=2.0 ** 10 if args.storage == "fp16" else 0.0,
                   scale_g=2.0 ** 10 if args.storage == "fp16" else 0.0)
    y0 = rank * n
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        lat = D.Lattice(cfg, device=dev, stream=stream, rows=(y0, n))
        T = inputs.taylor_green(n, 0.01, phi_amp=0.1, ny=ny, window=(0, y0, n, n), xp=torch,
                                device=dev)
        lat.init(*[a.float() for a in (T.rho, T.ux, T.uy, T.phi, T.grads)])
        del T
        elem = torch.int32 if args.storage == "fp32" else torch.int16
        m = lat.halo_elems()
        down = torch.empty(m, dtype=elem, device=dev)
        up = torch.empty(m, dtype=elem, device=dev)

        def one_step():
            lat.step(1)
            if world > 1:
                lat.halo_pack(down, up)
                # NCCL's stream waits for the current stream (the pack) and the
                # current stream waits for the exchange (req.wait), no host sync
                fb, fa = halo_exchange(down, up, world, rank, periodic=True)
                lat.halo_unpack(fb, fa)

        for _ in range(args.warmup * lb):
            one_step()
        torch.cuda.synchronize(dev)
        clocks = ClockSampler(local)
        barrier(world)
        torch.cuda.synchronize(dev)
        clocks.start()
        t0 = time.perf_counter()
        for _ in range(args.steps * lb):
            one_step()
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        barrier(world)
        clk = clocks.stop()
        dt = max_over_ranks(world, dt)
        s = lat.sums()
        mass_dev, _, _ = allreduce_sums([s["mass_dev"], s["scalar_dev"], s["u2"]], world,
                                        device=dev)
    if rank != 0:
        return
    value = n * ny * lb * args.steps / dt / 1e6
    print(json.dumps({
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"taylor-green {n}x{ny} divided into {world} y-slabs of {n}x{n}, "
                               f"{args.storage} storage, {lb} fused steps per benchmark step, "
                               f"halo exchange every step",
                   "parallelism": f"y-slabs over {world} ranks" if world > 1 else "single",
                   "timing": "host clock around the steps and exchanges"},
        "clocks": clk, "gpu_launches": args.steps * lb * (3 if world > 1 else 1),
        "checks": {"mass_dev": mass_dev}}))


def run_surrogate(args, world, rank, local):
    """Learned warm start: steady cavity data from the method, U-Net training on
    the GPU (data parallel over ranks: each rank generates and trains on its
    share of the draws, gradients averaged), then held-out cavities run to
    residual 1e-8 from rest and from the prediction, next to a long-run
    reference.  Reports the steps-to-steady ratio (cold / warm), aggregate and
    median, and the final omega error of both runs against the reference."""
    import torch
    from paper_1908_06742_gb300 import build as B
    from paper_1908_06742_gb300 import surrogate as S
    B.build()
    torch.cuda.set_device(local)
    t0 = time.perf_counter()
    r = S.experiment(n=args.n if args.n != 16384 else 128, n_train=args.instances,
                     n_test=64, epochs=args.lb_steps if args.lb_steps != 200 else 60,
                     boot=args.boot, log=lambda s: print(s, file=sys.stderr), world=world,
                     rank=rank)
    dt = time.perf_counter() - t0
    if rank != 0:
        return
    rows = r.pop("rows")
    print(json.dumps({
        "metric": METRIC, "value": round(r["steps_saved_ratio"], 3),
        "unit": "steps-to-steady ratio (cold / warm)", "n_gpus": world, "steps": 1, "warmup": 0,
        "ms_per_step": round(dt * 1e3, 1), "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"learned warm start: {r['n_train']} steady {r['grid']}^2 cavities "
                               f"(Re 100-3200, Pe 50-3200, lid 0.05-0.1) for training "
                               f"({r['n_boot']} from rest, the rest warm-started by a network "
                               f"trained on those), {r['n_test']} held-out draws run to residual "
                               f"1e-8, capped runs counted at the cap",
                   "parallelism": f"data parallel over {world} ranks" if world > 1 else "single"},
        "surrogate": r,
        "per_case": rows[:64],
    }))


# U-Net convolution GEMMs (C = A . B^T): forward (pixels x Cout x 9 Cin) at the
# 128^2 / batch-16 training size, and weight gradients (Cout x 9 Cin x pixels,
# split-K)
GEMM_SHAPES = [(262144, 32, 144, 1), (65536, 64, 288, 1), (16384, 128, 576, 1),
               (4096, 128, 1152, 1), (65536, 128, 1152, 1), (16384, 256, 2304, 1),
               (128, 1152, 65536, 16)]


def run_sweep(args, world, rank, local):
    """Throughput sweep: decaying Taylor-Green (U0 = 0.01, nu = D = 0.01) on N x N
    lattices, N = 1024, 4096, 8192, 16384, FP32 / FP16 / BF16 storage (default
    step kernel of each), --lb-steps fused steps timed with CUDA events after
    as many untimed ones.  A row whose two population buffers fit in the 129 MB
    L2 is marked l2_resident (its GB/s are not HBM figures)."""
    import torch
    from paper_1908_06742_gb300 import build as B
    from paper_1908_06742_gb300 import ddflb as D
    from paper_1908_06742_gb300 import inputs

    B.build()
    D.load()
    dev = torch.device("cuda", local)
    peak, kind = peaks()
    wf, wg = rates(0.01)
    rows = []
    stream = torch.cuda.Stream(dev)
    for st in ("fp32", "fp16", "bf16"):
        for n in (1024, 4096, 8192, 16384):
            a = argparse.Namespace(**vars(args))
            a.n, a.storage, a.step_path = n, st, 0
            cfg = D.Config(nx=n, ny=n, storage=st, omega_f=wf, omega_g=wg,
                           scale_f=2.0 ** 10 if st == "fp16" else 0.0,
                           scale_g=2.0 ** 10 if st == "fp16" else 0.0)
            with torch.cuda.stream(stream):
                lat = D.Lattice(cfg, device=dev, stream=stream)
                T = inputs.taylor_green(n, 0.01, phi_amp=0.1, xp=torch, device=dev)
                lat.init(*[t.float() for t in (T.rho, T.ux, T.uy, T.phi, T.grads)])
                del T
                lb = args.lb_steps
                lat.step(lb)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                barrier(world)
                torch.cuda.synchronize(dev)
                e0.record(stream)
                lat.step(lb)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ms = max_over_ranks(world, e0.elapsed_time(e1))
                diverged = lat.stats()["diverged"]
                del lat
            torch.cuda.empty_cache()
            bpc = BYTES_PER_CELL[st]
            gbs = bpc * n * n * lb / (ms / 1e3) / 1e9
            rows.append({"n": n, "storage": st, "kernel": step_kernel_name(a),
                         "mlups": round(world * n * n * lb / (ms / 1e3) / 1e6, 1),
                         "gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
                         "l2_resident": bpc * n * n < 129e6, "diverged": bool(diverged)})
    if rank != 0:
        return
    top = [r for r in rows if r["n"] == 16384 and r["storage"] == "fp32"][0]
    print(json.dumps({
        "metric": METRIC, "value": top["mlups"], "unit": "MLUPS", "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"taylor-green throughput sweep, N = 1024..16384, fp32/fp16/bf16, "
                               f"{args.lb_steps} timed fused steps each; value = fp32 at 16384^2"},
        "roofline": {"bound": "hbm", "achieved": top["gbs"], "peak": peak, "unit": "GB/s",
                     "frac": top["frac"], "peak_kind": kind, "kernel": top["kernel"]},
        "rows": rows}))


def run_gemm(args, world, rank, local):
    """BF16 GEMM throughput of the surrogate's contraction shapes on the
    tensor-core paths (0: tcgen05 + TMA, persistent; 1: mma.sync; 2: tcgen05,
    one tile per CTA), CUDA events per shape."""
    import torch
    from paper_1908_06742_gb300 import build as B
    from paper_1908_06742_gb300 import ddflb as D
    B.build()
    torch.cuda.set_device(local)
    lib = D.load()
    shapes = GEMM_SHAPES
    if args.gemm_shape:
        shapes = [tuple(int(v) for v in args.gemm_shape.split(","))]
    rows, tot = [], {0: [0.0, 0.0], 1: [0.0, 0.0], 2: [0.0, 0.0]}
    st = torch.cuda.current_stream()
    for M, N, K, sp in shapes:
        g = torch.Generator(device="cuda").manual_seed(M + N + K)
        A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
        Bm = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
        C = torch.empty(M, N, device="cuda")
        part = torch.empty(sp * M * N, device="cuda") if sp > 1 else None
        row = {"M": M, "N": N, "K": K, "splits": sp}
        for path in (0, 1, 2):
            D._check(lib.ddflb_nn_set_gemm_path(path))

            def call():
                D._check(lib.ddflb_nn_gemm(A.data_ptr(), Bm.data_ptr(), M, N, K, K, K,
                                           C.data_ptr(), N, None, 0, None, 0, 0, sp,
                                           None if part is None else part.data_ptr(),
                                           st.cuda_stream))
            for _ in range(args.warmup):
                call()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(args.steps):
                call()
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            fl = 2.0 * M * N * K
            row[f"ms_path{path}"] = round(ms, 4)
            row[f"tflops_path{path}"] = round(fl / ms / 1e9, 1)
            tot[path][0] += fl
            tot[path][1] += ms
        rows.append(row)
    D._check(lib.ddflb_nn_set_gemm_path(0))
    err = ctypes.c_int32(-1)
    D._check(lib.ddflb_nn_take_error(ctypes.byref(err), None))
    if rank != 0:
        return
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak, kind = float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        peak, kind = 1900.0, "fallback"
    agg = {p: tot[p][0] / tot[p][1] / 1e9 for p in tot}
    print(json.dumps({
        "metric": "BF16 GEMM TFLOP/s, surrogate convolution shapes (aggregate)",
        "value": round(agg[0], 1), "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(tot[0][1], 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "U-Net convolution GEMMs (forward and weight-gradient shapes)",
                   "kernel": "tcgen05 + TMA persistent (path 0); mma.sync (path 1); "
                             "tcgen05 one tile per CTA (path 2)"},
        "roofline": {"bound": "tensor", "achieved": round(agg[0], 1), "peak": peak,
                     "unit": "TFLOP/s", "frac": round(agg[0] / peak, 4), "peak_kind": kind},
        "mma_sync_tflops": round(agg[1], 1), "tcgen05_tile_per_cta_tflops": round(agg[2], 1),
        "device_error_word": err.value, "shapes": rows}))


# U-Net 3x3 convolutions that take the implicit path (input channels a
# multiple of 64), forward, at 256^2 / batch 16 (width 32): (H, W, Cin, Cout)
CONV_SHAPES = [(256, 256, 64, 32), (128, 128, 64, 64), (128, 128, 128, 64), (128, 128, 64, 32),
               (64, 64, 64, 128), (64, 64, 128, 128), (64, 64, 256, 128), (64, 64, 128, 64),
               (32, 32, 128, 128)]


def run_conv(args, world, rank, local):
    """The surrogate's 3x3 convolutions: implicit GEMM on tcgen05 (4-D TMA
    boxes per tap, no patch matrix) against im2col + the tcgen05 GEMM, CUDA
    events per shape; reports the aggregate BF16 TFLOP/s of the implicit form
    and the DRAM-free bound of each (2 P N 9 C flops)."""
    import torch
    from paper_1908_06742_gb300 import build as B
    from paper_1908_06742_gb300 import ddflb as D
    B.build()
    torch.cuda.set_device(local)
    lib = D.load()
    D._check(lib.ddflb_nn_set_conv_path(args.conv_path))
    st = torch.cuda.current_stream()
    Bt = 16
    rows, tot = [], {"implicit": [0.0, 0.0], "im2col": [0.0, 0.0]}
    for H, W, C, N in CONV_SHAPES:
        g = torch.Generator(device="cuda").manual_seed(H + C + N)
        X = torch.randn(Bt, H, W, C, device="cuda", generator=g).to(torch.bfloat16)
        Wt = (0.05 * torch.randn(N, 9 * C, device="cuda", generator=g)).to(torch.bfloat16)
        Y = torch.empty(Bt * H * W, N, dtype=torch.bfloat16, device="cuda")
        col = torch.empty(Bt * H * W, 9 * C, dtype=torch.bfloat16, device="cuda")
        P = Bt * H * W

        def implicit():
            D._check(lib.ddflb_nn_conv3x3(X.data_ptr(), Bt, H, W, C, C, Wt.data_ptr(), N, None,
                                          0, Y.data_ptr(), N, None, 1, 0, st.cuda_stream))

        def explicit():
            D._check(lib.ddflb_nn_im2col(X.data_ptr(), Bt, H, W, C, C, col.data_ptr(), 0,
                                         st.cuda_stream))
            D._check(lib.ddflb_nn_gemm(col.data_ptr(), Wt.data_ptr(), P, N, 9 * C, 9 * C, 9 * C,
                                       None, 0, Y.data_ptr(), N, None, 1, 0, 1, None,
                                       st.cuda_stream))
        row = {"H": H, "W": W, "C": C, "N": N, "pixels": P}
        fl = 2.0 * P * N * 9 * C
        for tag, fn in (("implicit", implicit), ("im2col", explicit)):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(args.steps):
                fn()
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            row[f"ms_{tag}"] = round(ms, 4)
            row[f"tflops_{tag}"] = round(fl / ms / 1e9, 1)
            tot[tag][0] += fl
            tot[tag][1] += ms
        # bytes the implicit form must move at least: activation in, output out, weights
        row["min_bytes"] = P * C * 2 + P * N * 2 + N * 9 * C * 2
        row["gbs_implicit"] = round(row["min_bytes"] / (row["ms_implicit"] / 1e3) / 1e9, 1)
        rows.append(row)
        del X, Wt, Y, col
    err = ctypes.c_int32(-1)
    D._check(lib.ddflb_nn_take_error(ctypes.byref(err), None))
    if rank != 0:
        return
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak, kind = float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        peak, kind = 1900.0, "fallback"
    agg = {k: v[0] / v[1] / 1e9 for k, v in tot.items()}
    # per shape, the roofline time: the larger of the tensor time at the BF16
    # peak and the HBM time of the compulsory bytes at the measured copy peak
    hbm, hbm_kind = peaks()
    t_roof = 0.0
    for r in rows:
        fl = 2.0 * r["pixels"] * r["N"] * 9 * r["C"]
        t = max(fl / (peak * 1e12), r["min_bytes"] / (hbm * 1e9)) * 1e3
        r["roofline_ms"] = round(t, 4)
        r["bound"] = "hbm" if r["min_bytes"] / (hbm * 1e9) * 1e12 > fl / peak else "tensor"
        r["frac_of_roofline"] = round(t / r["ms_implicit"], 3)
        t_roof += t
    print(json.dumps({
        "metric": "BF16 TFLOP/s, surrogate 3x3 convolutions (aggregate)",
        "value": round(agg["implicit"], 1), "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot["implicit"][1], 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": "U-Net 3x3 convolutions with >= 64 input channels, 256^2 level "
                               "sizes, batch 16, forward (BF16 out, leaky ReLU)",
                   "kernel": "implicit GEMM, tcgen05 + 4-D TMA (ddflb_nn_conv3x3) vs im2col + "
                             "tcgen05 GEMM"},
        "roofline": {"bound": "tensor", "achieved": round(agg["implicit"], 1), "peak": peak,
                     "unit": "TFLOP/s", "frac": round(agg["implicit"] / peak, 4), "peak_kind": kind,
                     # the layers' own roofline: sum over shapes of max(tensor time, HBM
                     # time of the compulsory bytes) against the measured total
                     "frac_of_layer_roofline": round(t_roof / tot["implicit"][1], 4),
                     "hbm_peak_gbs": hbm, "hbm_peak_kind": hbm_kind},
        "conv_path": args.conv_path,
        "im2col_gemm_tflops": round(agg["im2col"], 1), "device_error_word": err.value,
        "shapes": rows}))


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "batch":
        run_batch(args, world, rank, local)
    elif args.workload == "cavity":
        run_cavity(args, world, rank, local)
    elif args.workload == "surrogate":
        run_surrogate(args, world, rank, local)
    elif args.workload == "gemm":
        run_gemm(args, world, rank, local)
    elif args.workload == "sweep":
        run_sweep(args, world, rank, local)
    elif args.workload == "slabs":
        run_slabs(args, world, rank, local)
    elif args.workload == "conv":
        run_conv(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
