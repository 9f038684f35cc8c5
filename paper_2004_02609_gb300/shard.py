"""Capacitance extraction sharded over the ranks of a process group.

The unit-potential solves of the conductors (Eq. 8: one right-hand side
per conductor) are independent, so they split across GPUs with no exchange
during the solve: every rank sets up the same structure (replicated
spectra and preconditioner), solves a contiguous block of conductors, and
one all-gather of the m x m matrix's columns (m^2 doubles) assembles C on
every rank.  Batched independent structures split the same way.

The column solves of the library do not depend on which other columns share
their batch, so the assembled matrix equals the single-rank one bit for bit
when every rank runs the same product variant; ``pin_product_variant``
makes every rank use rank 0's.
"""
from __future__ import annotations

import numpy as np


def column_range(m: int, rank: int, world: int):
    """The contiguous block of conductors [j0, j1) that `rank` solves."""
    return (rank * m) // world, ((rank + 1) * m) // world


def _device_for(group):
    import torch
    import torch.distributed as dist
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
        else torch.device("cpu")


def gather_columns(block: np.ndarray, m: int, group=None) -> np.ndarray:
    """All-gather the column blocks ([m, j1 - j0] on each rank, in rank
    order) into the full [m, m] matrix on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    width = max(column_range(m, r, world)[1] - column_range(m, r, world)[0] for r in range(world))
    dev = _device_for(group)
    pad = torch.zeros((m, width), dtype=torch.float64, device=dev)
    if block.shape[1]:
        pad[:, :block.shape[1]] = torch.as_tensor(block, dtype=torch.float64, device=dev)
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    C = np.zeros((m, m))
    for r, p in enumerate(parts):
        j0, j1 = column_range(m, r, world)
        C[:, j0:j1] = p[:, :j1 - j0].cpu().numpy()
    return C


def capacitance_sharded(solve_columns, m: int, group=None) -> np.ndarray:
    """C [m, m] with this rank solving only its block of conductors:
    ``solve_columns(j0, j1)`` returns the [m, j1 - j0] columns."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    j0, j1 = column_range(m, rank, world)
    block = solve_columns(j0, j1) if j1 > j0 else np.zeros((m, 0))
    return gather_columns(np.asarray(block, dtype=np.float64), m, group)


def pin_product_variant(vc, group=None):
    """Make every rank run the FP32 products with rank 0's variant (the
    autotuner may pick differently on different GPUs, and variants round
    differently)."""
    import torch
    import torch.distributed as dist
    dev = _device_for(group)
    mine = torch.tensor([vc.set_product_path(-2), *vc.set_product_tiles(-2)], dtype=torch.int64, device=dev)
    dist.broadcast(mine, src=0, group=group)
    path, zo, zt, yf, yi = (int(v) for v in mine.cpu().tolist())
    if path == 0:
        vc.set_product_tiles(zo, zt, yf, yi)
    else:
        vc.set_product_path(path)


def capacitance_on_ranks(vc, tol: float, group=None) -> np.ndarray:
    """The capacitance matrix of the handle's structure with the conductors
    split over the group's ranks (one GPU each, every rank holding a handle
    of the same structure)."""
    pin_product_variant(vc, group)
    m = vc.n_conductors
    return capacitance_sharded(lambda j0, j1: vc.capacitance_columns(j0, j1, tol=tol)[0], m, group)
