"""GPU parity of the batched full definition: 64 cut circuits of uneven shape
(HWEA, AQFT, BV; 16-28 qubits; 2-4 subcircuits; K <= 8) in one call that
runs eagerly, is captured into a CUDA graph, and is replayed - every instance
checked against the FP64 oracle (all outputs for the small ones, sampled
outputs for the rest) on the first call and on the replay."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
from test_gpu_fd import env  # noqa: E402,F401

pytestmark = pytest.mark.gpu


_cache = {}


@pytest.mark.parametrize("algo", ["auto", "cc"])
def test_batched_64_instances_graph_replay(env, algo):
    """algo "cc": every final contraction on CUDA cores, the low-rank ones
    (at most 16 kept terms) together in one launch over a device work list."""
    torch, cutqc = env
    from oracle import attribution as at
    from oracle import reconstruct as rc
    from paper_2012_02333_gb300 import circuits as C
    batch = C.batch_instances(64, 0)
    if "T64" not in _cache:
        _cache["T64"] = [at.tensors(cc) for cc in batch]
    T64 = _cache["T64"]
    T32 = [[T.astype(np.float32) for T in Ts] for Ts in T64]
    dev = torch.device("cuda")
    ts = [[torch.tensor(T.reshape(-1), device=dev) for T in Ts] for Ts in T32]
    problems = [cutqc.Problem.from_cut(cc, t) for cc, t in zip(batch, ts)]
    outs = [torch.full((2 ** cc.n,), float("nan"), device=dev) for cc in batch]
    sums = torch.zeros(len(batch), dtype=torch.float64, device=dev)
    rng = np.random.default_rng(5)
    samples = []
    for cc, Ts in zip(batch, T32):
        if cc.n <= 18:
            samples.append(None)
        else:
            samples.append(sorted(set(int(x) for x in rng.integers(0, 2 ** cc.n, 256 if cc.n_cuts >= 6 else 512)) | {0, 2 ** cc.n - 1}))
    if "wants" not in _cache:
        wants = []
        for cc, Ts, xs in zip(batch, T32, samples):
            T = [t.astype(np.float64) for t in Ts]
            wants.append(rc.fd_full(cc.subs, T, cc.n, cc.n_cuts) if xs is None
                         else rc.fd_entries(cc.subs, T, cc.n, cc.n_cuts, xs))
        _cache["wants"] = wants
    wants = _cache["wants"]
    launches = []
    for call in range(3):            # eager + capture, then two graph replays
        for o in outs:
            o.fill_(float("nan"))
        l0 = cutqc.launch_count()
        cutqc.cutqc_reconstruct_fd(problems, outs, algo, sums)
        torch.cuda.synchronize()
        launches.append(cutqc.launch_count() - l0)
        for i, (cc, xs, want) in enumerate(zip(batch, samples, wants)):
            got = outs[i].double().cpu().numpy()
            got = got if xs is None else got[xs]
            err = np.abs(got - want).max()
            assert err <= 1e-6, (call, i, cc.n, cc.n_cuts, err)
        assert np.all(np.isfinite(sums.cpu().numpy()))
        for i, o in enumerate(outs):   # the fused FP64 sum is the sum of the returned outputs
            assert sums[i].item() == pytest.approx(torch.sum(o, dtype=torch.float64).item(), abs=1e-6)
    # the replays launch no kernels through the host API: one graph launch each
    assert launches[1] == 0 and launches[2] == 0
