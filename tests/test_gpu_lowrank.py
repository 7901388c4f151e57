"""GPU parity of single calls whose final contraction has at most 16 kept
terms (the streaming CUDA-core form: one-term outer products, one and two
cuts between the final groups, narrow and wide N sides) and of the shapes
around it (a final whose lowest output bits alternate between the groups,
group builds with a short side, operands of many short rows), each against
the FP64 oracle on sampled outputs, with the fused FP64 sum against the sum
of the returned outputs."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
from test_gpu_fd import env  # noqa: E402,F401

pytestmark = pytest.mark.gpu

# instances of the 64-instance batch (index: what the final contraction is)
CASES = {
    11: "28 qubits, one term (a disconnected subcircuit), 128-column N side",
    17: "28 qubits, four terms, 2^18-column N side",
    33: "28 qubits, sixteen terms",
    2: "24 qubits, K = 8: a group build with a 4-output side, then one term",
    13: "24 qubits, one term whose lowest output bits alternate between the groups",
    55: "18 qubits, K = 8, 16-column N side",
}


@pytest.mark.parametrize("idx", sorted(CASES))
def test_low_rank_single_calls(env, idx):
    torch, cutqc = env
    from oracle import attribution as at
    from oracle import reconstruct as rc
    from paper_2012_02333_gb300 import circuits as C
    cc = C.batch_instances(64, 0)[idx]
    T32 = [T.astype(np.float32) for T in at.tensors(cc)]
    dev = torch.device("cuda")
    ts = [torch.tensor(T.reshape(-1), device=dev) for T in T32]
    problem = cutqc.Problem.from_cut(cc, ts)
    out = torch.full((2 ** cc.n,), float("nan"), device=dev)
    sums = torch.zeros(1, dtype=torch.float64, device=dev)
    rng = np.random.default_rng(idx)
    n_s = 256 if cc.n_cuts >= 6 else 2048
    xs = sorted(set(int(x) for x in rng.integers(0, 2 ** cc.n, n_s)) | {0, 1, 2, 3, 2 ** cc.n - 1})
    want = rc.fd_entries(cc.subs, [T.astype(np.float64) for T in T32], cc.n, cc.n_cuts, xs)
    for algo in ("auto", "cc"):
        out.fill_(float("nan"))
        cutqc.cutqc_reconstruct_fd([problem], [out], algo, sums)
        torch.cuda.synchronize()
        assert not torch.isnan(out).any().item(), (idx, algo)
        got = out[torch.tensor(xs, device=dev)].double().cpu().numpy()
        assert np.abs(got - want).max() <= 1e-6, (idx, algo)
        assert sums.item() == pytest.approx(torch.sum(out, dtype=torch.float64).item(), abs=1e-6)
