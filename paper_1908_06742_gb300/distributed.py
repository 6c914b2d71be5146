"""Host-side logic of multi-rank runs (one process per GPU).

The method's workloads split in two ways (no collective sits inside a time
step of one lattice unless the lattice itself is divided):

* independent instances -- the batched cavities and the surrogate's training
  and held-out cavities -- are partitioned over ranks (`shard_indices`); the
  per-instance results come back to rank 0 in global order (`gather_indexed`);
* data-parallel surrogate training averages the gradients of all ranks before
  each optimiser step (`average_gradients`), so every rank applies the same
  update and the weights stay identical;
* one lattice divided into y-slabs (the locality of the collide-and-stream
  update, Secs. 2-3) exchanges, once per time step, the populations that cross
  each slab face (`halo_exchange`), and reduces its conservation and residual
  sums in FP64 over all ranks (`allreduce_sums`).

Everything here goes through torch.distributed, so the same code runs with
NCCL on GPU tensors and with gloo on CPU tensors.  With a world size of 1
every function is the identity.
"""
from __future__ import annotations

from typing import Any, Dict, Iterable, List, Sequence, Tuple


def world_and_rank() -> Tuple[int, int]:
    """(world size, rank) of the initialised process group, or (1, 0)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(), dist.get_rank()
    return 1, 0


def shard_indices(n_items: int, rank: int, world: int) -> List[int]:
    """The items rank `rank` of `world` owns: rank, rank + world, ... (round
    robin, so instances of every size land on every rank).  Every item belongs
    to exactly one rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    return list(range(rank, n_items, world))


def gather_indexed(local: Dict[int, Any], world: int, dst: int = 0):
    """Per-instance results {global index: value} of every rank, merged on
    rank `dst` into a list ordered by global index (None on other ranks).
    Raises if two ranks report the same index."""
    import torch.distributed as dist
    if world == 1:
        return [local[k] for k in sorted(local)]
    parts: List[Any] = [None] * world
    dist.all_gather_object(parts, local)
    if dist.get_rank() != dst:
        return None
    merged: Dict[int, Any] = {}
    for part in parts:
        for k, v in part.items():
            if k in merged:
                raise ValueError(f"instance {k} reported by two ranks")
            merged[k] = v
    return [merged[k] for k in sorted(merged)]


def average_gradients(grads: Sequence, world: int) -> None:
    """In-place mean over ranks of a list of same-dtype tensors (one flat
    collective): with equal per-rank batches this is the gradient of the loss
    averaged over the global batch."""
    if world == 1 or not grads:
        return
    import torch
    import torch.distributed as dist
    flat = torch.cat([g.reshape(-1) for g in grads])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM)
    flat.div_(world)
    o = 0
    for g in grads:
        n = g.numel()
        g.copy_(flat[o:o + n].view_as(g))
        o += n


def allreduce_sums(values: Iterable[float], world: int, device=None) -> List[float]:
    """Sum of FP64 scalars over ranks (mass, scalar, residual sums of a
    divided lattice)."""
    vals = [float(v) for v in values]
    if world == 1:
        return vals
    import torch
    import torch.distributed as dist
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [float(v) for v in t.tolist()]


def slab_rows(ny: int, parts: int, k: int) -> Tuple[int, int]:
    """Rows [y0, y0 + h) of slab k when ny rows are cut into `parts` slabs
    (the first ny % parts slabs take one row more)."""
    if not 0 < parts <= ny or not 0 <= k < parts:
        raise ValueError(f"slab {k} of {parts} over {ny} rows")
    base, extra = divmod(ny, parts)
    y0 = k * base + min(k, extra)
    return y0, base + (1 if k < extra else 0)


def halo_exchange(send_down, send_up, world: int, rank: int, periodic: bool):
    """One face exchange of a y-slab decomposition, rank r owning slab r.

    send_down: what slab r passes to slab r - 1 (its bottom row's outgoing
    populations); send_up: what it passes to slab r + 1 (its top row's).
    Returns (from_below, from_above): slab r - 1's send_up and slab r + 1's
    send_down, or None at a wall face (periodic=False and r = 0 or
    r = world - 1).  Sends and receives are posted together (no ordering
    deadlock for any world size)."""
    import torch
    import torch.distributed as dist
    below = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    above = rank + 1 if rank < world - 1 else (0 if periodic else None)
    if world == 1:
        return (send_up if below is not None else None,
                send_down if above is not None else None)
    from_below = torch.empty_like(send_up) if below is not None else None
    from_above = torch.empty_like(send_down) if above is not None else None
    # Messages between one pair of ranks match in the order they are posted.
    # With two periodic slabs the neighbour below is also the neighbour above,
    # so every rank sends up before down and receives from below before from
    # above: the peer's up-message then lands in from_below, its down-message
    # in from_above.
    ops = []
    if above is not None:
        ops.append(dist.P2POp(dist.isend, send_up, above))
    if below is not None:
        ops.append(dist.P2POp(dist.isend, send_down, below))
    if below is not None:
        ops.append(dist.P2POp(dist.irecv, from_below, below))
    if above is not None:
        ops.append(dist.P2POp(dist.irecv, from_above, above))
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    return from_below, from_above
