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


_CACHE_RUN = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from oracle import attribution as at
from paper_2012_02333_gb300 import circuits as C, cutqc
full = C.batch_instances(64, 0)
batch = [full[i] for i in (8, 35, 46, 0, 7)]   # three 4-cut pairs (256 terms: the forms are timed) and two chains
ts = [[torch.tensor(T.reshape(-1).astype(np.float32), device="cuda") for T in at.tensors(cc)] for cc in batch]
problems = [cutqc.Problem.from_cut(cc, t) for cc, t in zip(batch, ts)]
outs = [torch.empty(2 ** cc.n, device="cuda") for cc in batch]
cutqc.cutqc_reconstruct_fd(problems, outs, "auto")
torch.cuda.synchronize()
np.save(sys.argv[1], np.concatenate([o[:4096].double().cpu().numpy() for o in outs]))
"""


def test_autotune_cache_file(env, tmp_path):
    """Under CUTQC_AUTOTUNE_CACHE the batch's measured form choices are written
    to the named file by one process and read back by the next, which gives
    the same outputs."""
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.txt"
    envv = dict(os.environ, CUTQC_AUTOTUNE_CACHE=str(cache))
    code = _CACHE_RUN.format(root=root)
    outs = []
    for k in range(2):
        f = tmp_path / f"out{k}.npy"
        r = subprocess.run([sys.executable, "-c", code, str(f)], env=envv, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-3000:]
        outs.append(np.load(f))
        if k == 0:
            lines = cache.read_text().splitlines()
            assert lines and all(l.split(" ", 1)[0] in ("0", "1") for l in lines)
            n_first = len(lines)
    assert len(cache.read_text().splitlines()) == n_first    # nothing measured again
    assert np.array_equal(outs[0], outs[1])
