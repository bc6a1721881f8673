"""Path-range sharding across ranks (one process per GPU).

The Monte Carlo estimate partitions over paths: rank r simulates a
contiguous, 64-path-aligned range with ``heston_mc_launch_tiles``; the
per-tile partial-sum rows of all ranks, concatenated in rank order, are
exactly the rows of the unsharded run, so ``heston_mc_reduce_tiles`` over
them gives bit-identical estimates on every rank.  The only exchange is one
gather of those rows (12 doubles per contract and 64-path tile), done here
with ``torch.distributed``.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import native

TILE = native.HESTON_TILE_PATHS


def shard_bounds(n_paths: int, world: int, rank: int, tile: int = TILE):
    """[begin, end) of rank's paths: contiguous, tile-aligned begins, the
    tiles spread as evenly as possible, covering [0, n_paths) exactly."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    n_tiles = -(-n_paths // tile)
    per, extra = divmod(n_tiles, world)
    t0 = rank * per + min(rank, extra)
    t1 = t0 + per + (1 if rank < extra else 0)
    return min(t0 * tile, n_paths), min(t1 * tile, n_paths)


def gather_tile_rows(local_rows: torch.Tensor, n_paths: int, world: int, group=None) -> torch.Tensor:
    """All-gather every rank's tile rows (shape (local_tiles, width)) and
    return the (n_tiles, width) concatenation in rank order."""
    width = local_rows.shape[1]
    counts = []
    for r in range(world):
        b, e = shard_bounds(n_paths, world, r)
        counts.append(-(-(e - b) // TILE))
    cap = max(counts)
    padded = torch.zeros((cap, width), dtype=local_rows.dtype, device=local_rows.device)
    padded[: local_rows.shape[0]] = local_rows
    bufs = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(bufs, padded, group=group)
    return torch.cat([bufs[r][: counts[r]] for r in range(world)], dim=0)


def _launch_tiles_native(params, contracts, path_begin, n, n_steps, rng_seed, options, rows):
    native.heston_mc_launch_tiles(params, contracts, path_begin, n, n_steps, rng_seed, options, rows)


def _reduce_tiles_native(rows, n_tiles, n_contracts, n_paths, device):
    ws_bytes = native.heston_mc_workspace_bytes(n_contracts, n_paths)
    ws = torch.empty(ws_bytes // 8 + 1, dtype=torch.float64, device=device)
    out = torch.empty(n_contracts * 12, dtype=torch.float64, device=device)
    native.heston_mc_reduce_tiles(rows, n_tiles, n_contracts, n_paths, ws, ws_bytes, out,
                                  torch.cuda.current_stream())
    return out


def price_greeks_sharded(params, contracts, n_paths, n_steps, rng_seed, options, group=None,
                         device=None, launch_tiles=None, reduce_tiles=None):
    """Estimate on this rank's path range, gather the tile rows, reduce them
    in the fixed order: every rank returns the single-GPU result (C, 12) as a
    host tensor (per contract: 6 estimates, then their 6 standard errors).

    device: where the rows live (default: the current CUDA device).
    launch_tiles(params, contracts, path_begin, n, n_steps, seed, options, rows)
    and reduce_tiles(rows, n_tiles, n_contracts, n_paths, device) -> (12 C,)
    default to the library's heston_mc_launch_tiles / heston_mc_reduce_tiles;
    host-only tests replace them."""
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device())
    launch_tiles = launch_tiles or _launch_tiles_native
    reduce_tiles = reduce_tiles or _reduce_tiles_native
    b, e = shard_bounds(n_paths, world, rank)
    nc = len(contracts)
    local_tiles = -(-(e - b) // TILE)
    local = torch.zeros((max(1, local_tiles), 12 * nc), dtype=torch.float64, device=device)
    if e > b:
        launch_tiles(params, contracts, b, e - b, n_steps, rng_seed, options, local)
    rows = gather_tile_rows(local[:local_tiles], n_paths, world, group) if world > 1 else local[:local_tiles]
    out = reduce_tiles(rows.contiguous(), rows.shape[0], nc, n_paths, device)
    if out.is_cuda:
        torch.cuda.current_stream().synchronize()
    return out.view(nc, 12).cpu()
