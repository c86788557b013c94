"""Multi-GPU form of the annealer: one process per GPU, states sharded.

The B states of an anneal are independent (the batch of Sec. IV.C), so they
split into contiguous index ranges, one per rank.  Each rank anneals its
range with the range's global offset as ``state0``: the random streams of a
state depend only on (seed, global state index), so the union of the shards
is exactly one anneal of all B states, whatever the number of ranks.  The
data path has no collective; the only exchange is the final choice of the
best state: every rank contributes its lowest (energy, global index) pair,
all ranks agree on the lexicographic minimum (lowest energy, ties to the
lowest index), and its owner broadcasts the winning bits.

``torch.distributed`` carries the exchange (gloo on CPU, NCCL on GPUs).
"""
from __future__ import annotations

import numpy as np


def shard_range(B: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous share of states [lo, hi) of `rank`: B // world each, the
    first B % world ranks one more."""
    if world < 1 or not 0 <= rank < world or B < 0:
        raise ValueError("bad shard arguments")
    q, r = divmod(B, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def local_best(bestE, lo: int) -> tuple[float, int, int]:
    """(energy, global index, local index) of the lowest energy of a shard,
    ties to the lowest index; (inf, -1, -1) for an empty shard."""
    E = np.asarray(bestE, dtype=np.float64).reshape(-1)
    if E.size == 0:
        return float("inf"), -1, -1
    k = int(np.argmin(E))          # first occurrence of the minimum
    return float(E[k]), lo + k, k


def global_best(E: float, index: int, x_words, W: int, group=None, device=None):
    """Agree on the lowest (energy, index) over the ranks and broadcast its
    packed bits (int32 [W]) from the owner.  Returns (E, index, bits as a
    numpy uint32 array)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return E, index, np.asarray(x_words, dtype=np.int32).view(np.uint32).copy()
    dev = torch.device("cpu") if device is None else device
    world = dist.get_world_size(group)
    mine = torch.tensor([E, float(index)], dtype=torch.float64, device=dev)
    allv = [torch.empty(2, dtype=torch.float64, device=dev) for _ in range(world)]
    dist.all_gather(allv, mine, group=group)
    pairs = [(float(v[0]), int(v[1]), r) for r, v in enumerate(t.cpu() for t in allv)]
    pairs = [p for p in pairs if p[1] >= 0]
    if not pairs:
        return float("inf"), -1, np.zeros(W, np.uint32)
    bE, bidx, owner = min(pairs, key=lambda p: (p[0], p[1]))
    buf = torch.zeros(W, dtype=torch.int32, device=dev)
    if dist.get_rank(group) == owner:
        buf.copy_(torch.as_tensor(np.asarray(x_words, dtype=np.int32).reshape(-1), device=dev))
    src = dist.get_global_rank(group, owner) if group is not None else owner
    dist.broadcast(buf, src=src, group=group)
    return bE, bidx, buf.cpu().numpy().view(np.uint32).copy()


def anneal_sharded(inst, seed: int, B: int, betas: np.ndarray, *, group=None, anneal_fn=None, device=None,
                   **kw) -> dict:
    """Anneal this rank's share of B states and agree on the overall best.

    anneal_fn(lo, hi) -> (bestX packed words [hi-lo, W], bestE [hi-lo]) runs
    the shard; by default it is ``inst.anneal(seed, hi - lo, betas,
    state0=lo, **kw)`` on the current GPU.  Returns the shard range, the
    shard's results and the overall best (energy, global index, bits)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        rank, world = dist.get_rank(group), dist.get_world_size(group)
    else:
        rank, world = 0, 1
    lo, hi = shard_range(B, rank, world)
    if anneal_fn is None:
        def anneal_fn(a, b):
            r = inst.anneal(seed, b - a, betas, state0=a, **kw)
            return r["bestX"].cpu().numpy(), r["bestE"].cpu().numpy()
    bx, be = anneal_fn(lo, hi)
    bx = np.asarray(bx)
    W = bx.shape[1] if bx.ndim == 2 and bx.shape[0] else (inst.N + 31) // 32
    E, gidx, k = local_best(be, lo)
    words = bx[k] if k >= 0 else np.zeros(W, np.int32)
    gE, gi, gx = global_best(E, gidx, words, W, group=group, device=device)
    return {"range": (lo, hi), "bestX": bx, "bestE": np.asarray(be), "best_E": gE, "best_index": gi,
            "best_X": gx}
