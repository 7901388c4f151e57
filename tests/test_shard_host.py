"""The sharded reconstruction's host logic on CPU: two gloo ranks (127.0.0.1
rendezvous) each take one output slab (the most significant output bit fixed
at the rank), computed here by the FP64 oracle; the module's 8-byte FP64
all-reduce must give the unsharded sum and its all-gather merge of 32
candidates per rank the unsharded top-32, for the full definition and for a
dynamic-definition recursion sharded over its active qubits."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _top(vals, k, offset=0):
    order = sorted(range(len(vals)), key=lambda i: (-vals[i], i))[:k]
    return [offset + i for i in order], [float(vals[i]) for i in order]


def _rank_main(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from oracle import attribution as at
    from oracle import reconstruct as rc
    from paper_2012_02333_gb300 import circuits as C
    from paper_2012_02333_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cc = C.grid_blocks(3, 4, 8, 1, 1, 2, 6, 9)
    T = at.tensors(cc)
    s = shard.slab_bits(world)
    # full definition: this rank's slab = the outputs whose top s bits read rank
    roles = [(3 if (rank >> (s - 1 - q)) & 1 else 2) if q < s else 0 for q in range(cc.n)]
    slab = rc.dd_bins(cc.subs, T, cc.n, cc.n_cuts, roles)
    total = shard.allreduce_sum(torch.tensor([slab.sum()], dtype=torch.float64))
    li, lv = _top(slab, 32, rank << (cc.n - s))
    gi, gv = shard.topk_merge(li, lv, 32)
    # dynamic definition: recursion-1 roles with 5 active qubits, sharded over them
    droles = rc.initial_roles(cc.n, 5)
    mine = shard.dd_roles_for_rank(droles, rank, world)
    dbins = rc.dd_bins(cc.subs, T, cc.n, cc.n_cuts, mine)
    di, dv = _top(dbins, 8, rank << (5 - s))
    dgi, dgv = shard.topk_merge(di, dv, 8)
    q.put((rank, float(total.item()), gi, gv, slab.tolist(), dgi, dgv, dbins.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_unsharded_sum_and_top_lists():
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    from oracle import attribution as at
    from oracle import reconstruct as rc
    from paper_2012_02333_gb300 import circuits as C
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    cc = C.grid_blocks(3, 4, 8, 1, 1, 2, 6, 9)
    T = at.tensors(cc)
    full = rc.fd_full(cc.subs, T, cc.n, cc.n_cuts)
    want_i, want_v = _top(full, 32)
    dfull = rc.dd_bins(cc.subs, T, cc.n, cc.n_cuts, rc.initial_roles(cc.n, 5))
    dwant_i, dwant_v = _top(dfull, 8)
    # the slabs in rank order are the whole distribution
    assert np.allclose(np.concatenate([g[4] for g in got]), full, atol=1e-14)
    assert np.allclose(np.concatenate([g[7] for g in got]), dfull, atol=1e-14)
    for rank, total, gi, gv, _, dgi, dgv, _ in got:
        assert total == pytest.approx(full.sum(), abs=1e-13)
        assert gi == want_i and np.allclose(gv, want_v, atol=1e-14)
        assert dgi == dwant_i and np.allclose(dgv, dwant_v, atol=1e-14)


def test_slab_helpers():
    sys.path.insert(0, ROOT)
    from paper_2012_02333_gb300 import shard
    assert [shard.slab_bits(w) for w in (1, 2, 4, 8)] == [0, 1, 2, 3]
    with pytest.raises(ValueError):
        shard.slab_bits(3)
    roles = [1, 0, 0, 1, 0, 2]
    assert shard.dd_roles_for_rank(roles, 1, 2) == [1, 3, 0, 1, 0, 2]
    assert shard.dd_roles_for_rank(roles, 2, 4) == [1, 3, 2, 1, 0, 2]
    i, v = shard.topk_merge([5, 3, -1], [0.5, 0.5, 0.0], 4)     # no process group: local ranking only
    assert i == [3, 5, -1, -1] and v == [0.5, 0.5, 0.0, 0.0]
