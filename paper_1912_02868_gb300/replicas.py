"""Host-side logic of multi-GPU runs: independent replicas, no data-path collective.

Every solve is independent and a hierarchy's deflation space is read-only once
built, so N processes (one per GPU) each solve their own right-hand sides on
their own hierarchies.  The only cross-process steps are the barrier around the
timed region and the maximum of the per-rank times, both on the host side of
the measurement.  Rank r draws right-hand-side indices disjoint from every
other rank's, so the ranks' work is distinct.
"""
from __future__ import annotations

import os

RHS_STRIDE = 100000  # rank r uses right-hand-side indices [r * RHS_STRIDE, (r + 1) * RHS_STRIDE)


def rank_env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment (1 process when unset)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def rhs_index(rank: int, step: int) -> int:
    """Index of the right-hand side that rank `rank` solves at step `step`."""
    if not 0 <= step < RHS_STRIDE:
        raise ValueError(f"step {step} outside [0, {RHS_STRIDE})")
    return RHS_STRIDE * rank + step


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over all ranks (the value itself in a single process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None) -> None:
    """Barrier over all ranks (no-op in a single process)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        if device is not None and getattr(device, "type", "cpu") == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def total_units(world: int, steps: int, per_step: int) -> int:
    """Solves done by the whole job: every rank does `per_step` solves in each of `steps` steps."""
    return world * steps * per_step
