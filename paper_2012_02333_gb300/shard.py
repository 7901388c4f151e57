"""One reconstruction sharded over ranks (one process per GPU).

The paper's parallel processing (Sec. 4.2, Sec. 6.4) rests on there being no
data dependency between output entries or between Kronecker terms.  This
module partitions the output index space of one cut circuit into slabs by its
most significant bits: with G = 2^s ranks, rank r computes the 2^(n-s)
outputs whose top s bits read r (cutqc_reconstruct_fd_slab).  Every rank holds
the (small) subcircuit tensors in full and writes only its slab, so the only
exchange is an 8-byte FP64 all-reduce of the normalisation sum.  A
dynamic-definition recursion (Algorithm 1) shards the same way over its
active qubits: each rank bins its slab and ranks its own candidates, and the
ranks exchange 32 (index, FP64 value) pairs each to agree on the global top
list.  Partitioning the 4^K terms instead would need a reduce-scatter of all
2^n outputs, which is why the outputs are split.

Collectives go through torch.distributed (NCCL between GPUs, gloo on CPU);
no device memory of another rank is ever read directly.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import torch

from . import circuits


def slab_bits(world: int) -> int:
    """s with 2^s = world (the world size must be a power of two)."""
    if world < 1 or world & (world - 1):
        raise ValueError("the number of ranks must be a power of two")
    return world.bit_length() - 1


def allreduce_sum(x: torch.Tensor, group=None) -> torch.Tensor:
    """In-place sum of a float64 tensor over the ranks (the normalisation
    sum: 8 bytes per rank)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(x, op=dist.ReduceOp.SUM, group=group)
    return x


def topk_merge(idx: Sequence[int], val: Sequence[float], k: int, group=None) -> Tuple[List[int], List[float]]:
    """The global top-k from every rank's top-k (global bin indices, FP64
    values): an all-gather of k pairs per rank, ranked by value, ties to the
    lower index (the same order each rank's list uses).  Entries with index
    < 0 are padding."""
    import torch.distributed as dist
    pairs = [(float(v), int(i)) for i, v in zip(idx, val) if int(i) >= 0]
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        w = dist.get_world_size(group)
        mine_i = torch.full((k,), -1, dtype=torch.int64, device=dev)
        mine_v = torch.zeros(k, dtype=torch.float64, device=dev)
        for j, (v, i) in enumerate(pairs[:k]):
            mine_i[j] = i
            mine_v[j] = v
        all_i = [torch.empty_like(mine_i) for _ in range(w)]
        all_v = [torch.empty_like(mine_v) for _ in range(w)]
        dist.all_gather(all_i, mine_i, group=group)
        dist.all_gather(all_v, mine_v, group=group)
        pairs = [(float(v), int(i)) for ti, tv in zip(all_i, all_v)
                 for i, v in zip(ti.tolist(), tv.tolist()) if i >= 0]
    pairs.sort(key=lambda t: (-t[0], t[1]))
    pairs = pairs[:k]
    return [i for _, i in pairs] + [-1] * (k - len(pairs)), [v for v, _ in pairs] + [0.0] * (k - len(pairs))


def reconstruct_fd_sharded(cc: circuits.CutCircuit, tensors: Sequence[torch.Tensor], rank: int, world: int,
                           algo: str = "auto", out: Optional[torch.Tensor] = None, group=None, stream=None):
    """This rank's slab of the full definition and the global FP64 sum.
    Returns (slab, slab_bits, sum): slab[j] = p(rank * 2^(n - s) + j)."""
    from . import cutqc
    s = slab_bits(world)
    problem = cutqc.Problem.from_cut(cc, tensors)
    dev = tensors[0].device
    if out is None:
        out = torch.empty(2 ** (cc.n - s), dtype=problem.dtype, device=dev)
    sp = torch.empty(1, dtype=torch.float64, device=dev)
    cutqc.cutqc_reconstruct_fd_slab(problem, s, rank, out, algo, sp, stream)
    return out, s, allreduce_sum(sp, group)


def dd_roles_for_rank(roles: Sequence[int], rank: int, world: int) -> List[int]:
    """A recursion's roles for one rank: its s most significant active qubits
    (the lowest-numbered ones) fixed at the rank's bits, the rest unchanged."""
    s = slab_bits(world)
    out = list(roles)
    act = [q for q, r in enumerate(out) if r == 0]
    if s > len(act) - 1:
        raise ValueError("more slab bits than active qubits can spare")
    for j, q in enumerate(act[:s]):
        out[q] = 3 if (rank >> (s - 1 - j)) & 1 else 2
    return out


def reconstruct_dd_sharded(cc: circuits.CutCircuit, tensors: Sequence[torch.Tensor], roles: Sequence[int],
                           rank: int, world: int, topk: int = 32, algo: str = "auto", group=None, stream=None):
    """One dynamic-definition recursion sharded over the ranks: this rank's
    2^(#active - s) bins (the bins whose top s bits read the rank) and the
    global FP64-ranked top list (global bin indices)."""
    from . import cutqc
    s = slab_bits(world)
    na = sum(1 for r in roles if r == 0)
    mine = dd_roles_for_rank(roles, rank, world)
    problem = cutqc.Problem.from_cut(cc, tensors)
    bins = torch.empty(2 ** (na - s), dtype=problem.dtype, device=tensors[0].device)
    idx, val = cutqc.cutqc_reconstruct_dd(problem, mine, bins, topk, algo, stream)
    gidx = [(rank << (na - s)) | i if i >= 0 else -1 for i in idx]
    return bins, topk_merge(gidx, val, topk, group)
