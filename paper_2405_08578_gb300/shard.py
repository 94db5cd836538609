"""Pair sharding across processes (one GPU each) for the all-pairs homography
matrix H_M of Sec. 4.

Image pairs are independent units: rank r of W takes pairs r, r + W, r + 2W, ...
of the pair list, runs them with lp_stitch_pairs on its own GPU, and one
all_gather assembles every rank's (H, n_in, valid) rows in pair order.  No
collective touches the data path; the gather moves P x 11 numbers.

The gather works on any torch.distributed backend (NCCL for device tensors,
gloo for host tensors), so the host logic is exercised on CPU processes.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def all_pairs(n: int) -> list[tuple[int, int]]:
    """(i, j), i < j, in row-major order: the order of lp_stitch_pairs' H_M."""
    return [(i, j) for i in range(n) for j in range(i + 1, n)]


def shard(num_pairs: int, world: int, rank: int) -> list[int]:
    """Indices of the pairs that rank `rank` of `world` processes."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    return list(range(rank, num_pairs, world))


def gather_rows(local_idx: list[int], local_rows: torch.Tensor, num_pairs: int, world: int) -> torch.Tensor:
    """Assemble per-pair rows (float64, shape [len(local_idx), C]) of every rank
    into one [num_pairs, C] tensor on every rank, in pair order."""
    cap = (num_pairs + world - 1) // world
    C = local_rows.shape[1]
    buf = torch.zeros((cap, C + 1), dtype=torch.float64, device=local_rows.device)
    buf[:, 0] = -1.0
    if len(local_idx):
        buf[: len(local_idx), 0] = torch.tensor(local_idx, dtype=torch.float64, device=local_rows.device)
        buf[: len(local_idx), 1:] = local_rows.to(torch.float64)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    out = torch.full((num_pairs, C), float("nan"), dtype=torch.float64, device=local_rows.device)
    for part in parts:
        keep = part[:, 0] >= 0
        out[part[keep, 0].long()] = part[keep, 1:]
    return out


def stitch_pairs_sharded(ctx, images, world: int, rank: int, pairs=None, stream=None):
    """H_M of a set of images with the pair list split across `world` ranks.

    images: list of (device uint8 tensor, H, W, pitch, channels) on this rank's GPU.
    Returns (HM [P, 3, 3] float64, n_in [P] int32, valid [P] uint8) on every rank."""
    pl = list(pairs) if pairs is not None else all_pairs(len(images))
    P = len(pl)
    mine = shard(P, world, rank)
    dev = images[0][0].device
    rows = torch.zeros((len(mine), 11), dtype=torch.float64, device=dev)
    if mine:
        HM = torch.zeros((len(mine), 9), dtype=torch.float64, device=dev)
        n_in = torch.zeros(len(mine), dtype=torch.int32, device=dev)
        valid = torch.zeros(len(mine), dtype=torch.uint8, device=dev)
        ctx.lp_stitch_pairs(images, HM, n_in, valid, pairs=[pl[q] for q in mine], stream=stream, pair_ids=mine)
        rows[:, :9] = HM
        rows[:, 9] = n_in.to(torch.float64)
        rows[:, 10] = valid.to(torch.float64)
    full = gather_rows(mine, rows, P, world)
    return full[:, :9].reshape(P, 3, 3), full[:, 9].to(torch.int32), full[:, 10].to(torch.uint8)
