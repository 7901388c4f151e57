"""GPU parity of the output-slab entry point that the sharded reconstruction
runs on every rank: the slabs of G = 2 and 4 ranks, computed one after the
other on this GPU (independent calls, no rank waits on another), put together
in rank order equal the oracle's full definition, their FP64 partial sums add
up to the oracle's sum, and a dynamic-definition recursion sharded over its
active qubits gives the unsharded bins and top list."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
import cases  # noqa: E402
from test_gpu_fd import env, oracle_case, to_dev  # noqa: E402,F401

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("name,dtype_np,algo,tol", [("grid4x5_k5", np.float32, "auto", 1e-6),
                                                   ("grid4x5_k5", np.float32, "tc_tf32x3", 1e-6),
                                                   ("grid4x4_s4", np.float32, "auto", 1e-6),
                                                   ("qaoa8_k4", np.float64, "cc", 1e-12)])
def test_fd_slabs_make_the_distribution(env, world, name, dtype_np, algo, tol):
    torch, cutqc = env
    from oracle import reconstruct as rc
    from paper_2012_02333_gb300 import shard
    cc, T = oracle_case(name, cases.SMALL[name])
    Tq = [t.astype(dtype_np) for t in T]
    ref = rc.fd_full(cc.subs, [t.astype(np.float64) for t in Tq], cc.n, cc.n_cuts)
    ts = to_dev(torch, Tq, torch.float64 if dtype_np == np.float64 else torch.float32)
    slabs, total = [], 0.0
    for r in range(world):
        out, s, sp = shard.reconstruct_fd_sharded(cc, ts, r, world, algo)
        slabs.append(out.double().cpu().numpy())
        total += float(sp.item())
    got = np.concatenate(slabs)
    assert np.abs(got - ref).max() <= tol
    assert total == pytest.approx(ref.sum(), abs=tol)


def test_dd_recursion_sharded_over_active_qubits(env):
    torch, cutqc = env
    from oracle import reconstruct as rc
    from paper_2012_02333_gb300 import shard
    cc, T = oracle_case("grid4x5_k5", cases.SMALL["grid4x5_k5"])
    T32 = [t.astype(np.float32) for t in T]
    ts = to_dev(torch, T32, torch.float32)
    roles = rc.initial_roles(cc.n, 12)
    want = rc.dd_bins(cc.subs, [t.astype(np.float64) for t in T32], cc.n, cc.n_cuts, roles)
    world = 4
    parts, lists_i, lists_v = [], [], []
    for r in range(world):
        bins, (gi, gv) = shard.reconstruct_dd_sharded(cc, ts, roles, r, world, 32)
        parts.append(bins.double().cpu().numpy())
        lists_i += gi
        lists_v += gv
    assert np.abs(np.concatenate(parts) - want).max() <= 1e-6
    gi, gv = shard.topk_merge(lists_i, lists_v, 32)
    order = sorted(range(len(want)), key=lambda i: (-want[i], i))[:32]
    assert np.allclose(gv, want[gi], atol=1e-12)
    assert gi[0] == order[0] or abs(want[gi[0]] - want[order[0]]) <= 1e-12
    assert all(gv[j] >= gv[j + 1] for j in range(31))
    assert np.delete(want, gi).max() <= gv[-1] + 1e-12
