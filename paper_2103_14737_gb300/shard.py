"""Event sharding across ranks (one process per GPU).

Events are independent: event e of a batch uses random-stream event number
first_event + e, so a batch split into contiguous event ranges, one per rank,
gives exactly the cells of the unsplit batch.  The forward needs no
data-path collective; ranks only agree on timing (the maximum over ranks).

The adjoint has one exchange.  A loss summed over events (and over random
streams, the seeds) has a gradient that is the sum of the per-event (per-seed)
gradients, so ranks that each ran fcs_simulate_backward on their own events
or seeds sum d_frac and d_shape_w over the ranks: allreduce_gradients.
"""
from __future__ import annotations


def shard_events(n_events: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous event range (first, count) of `rank` among `world` ranks;
    the first n_events % world ranks take one extra event."""
    if world < 1 or not (0 <= rank < world) or n_events < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_events, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def max_over_ranks(value: float) -> float:
    """Maximum of a float over the ranks of the default process group (the
    value itself when no group is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_gradients(*grads):
    """Sums gradient tensors in place over the ranks of the default process
    group (NCCL for CUDA tensors, gloo for CPU tensors) and returns them.

    Use after each rank's fcs_simulate_backward over its event range or its
    seeds: every rank then holds the gradient of the whole batch.  None
    entries are skipped; without a process group, or with one rank, nothing
    changes.  All ranks must pass tensors of the same shapes in the same
    order."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return grads
    for g in grads:
        if g is not None:
            dist.all_reduce(g, op=dist.ReduceOp.SUM)
    return grads
