"""One process per GPU for independent boxes.

Boxes are independent problems: ranks split them (longest-processing-time greedy on particle
count) and run with no collective on the data path.  A sub-workload keeps the identities its
particles and sources have in the full workload, so each box draws the same random numbers and
gives the same results on whichever rank it runs.  The only cross-rank steps are the timing
(maximum over ranks) and, when wanted, the photon budget (sum over ranks), both after the timed
region.  A single box does not split without a per-hop exchange, so for one box every rank runs
its own replica.
"""
from __future__ import annotations

import numpy as np


def partition_boxes(counts, world: int):
    """Deterministic LPT assignment of boxes to ranks: biggest first, each to the least-loaded
    rank (lowest rank on ties).  Returns one ascending array of box indices per rank."""
    counts = np.asarray(counts, dtype=np.int64)
    order = sorted(range(len(counts)), key=lambda b: (-int(counts[b]), b))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for b in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(b)
        load[r] += int(counts[b])
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def local_workload(wl: dict, boxes) -> dict:
    """The sub-workload made of the given boxes (particles, boxes and their sources)."""
    boxes = np.asarray(boxes, dtype=np.int64)
    off = wl["box_off"]
    idx = np.concatenate([np.arange(off[b], off[b + 1]) for b in boxes]) if len(boxes) else \
        np.zeros(0, np.int64)
    sizes = np.array([off[b + 1] - off[b] for b in boxes], dtype=np.int64)
    new_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    remap = {int(b): k for k, b in enumerate(boxes)}
    src_keep = np.array([int(b) in remap for b in wl["src_box"]], dtype=bool)
    nfs = wl["params"]["n_freq_src"]
    ndot = np.asarray(wl["src_ndot"]).reshape(len(wl["src_box"]), max(nfs, 1) if nfs else 0)
    out = dict(wl)
    # the identities of the boxes' particles and sources in the full workload: the random
    # streams of a box (rotations, packet identities) are then those it has there, and a rank
    # running its boxes repeats their results in the unsplit run
    first = np.asarray(wl.get("box_first_id", off[:-1]), dtype=np.int64)
    sids = np.asarray(wl.get("src_id", np.arange(len(wl["src_box"]))), dtype=np.int64)
    out.update(
        box_off=new_off, box_L=np.asarray(wl["box_L"])[boxes],
        src_box=np.array([remap[int(b)] for b in np.asarray(wl["src_box"])[src_keep]], np.int32),
        src_ndot=np.ascontiguousarray(ndot[src_keep]).reshape(-1),
        box_first_id=first[boxes], src_id=sids[src_keep])
    for k in ("x", "y", "z", "n_H", "N_H", "x_HI", "T"):
        out[k] = np.ascontiguousarray(np.asarray(wl[k])[idx])
    for k in ("src_x", "src_y", "src_z"):
        out[k] = np.ascontiguousarray(np.asarray(wl[k])[src_keep])
    return out


def max_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(arr, device=None) -> np.ndarray:
    import torch
    import torch.distributed as dist
    t = torch.tensor(np.asarray(arr, dtype=np.float64), device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()
