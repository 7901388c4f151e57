"""Failure reporting without a GPU fault: a kernel whose bounded wait runs
out records a status word instead of hanging, and the host reports it.  The
self-test kernel waits on a flag nothing sets (limit 20 ms), then ends
normally; the context must stay usable afterwards."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
import cases  # noqa: E402
from test_gpu_fd import TOL32, env, oracle_case, to_dev  # noqa: E402,F401

pytestmark = pytest.mark.gpu


def test_status_clean_after_reconstruction(env):
    torch, cutqc = env
    cc, T = oracle_case("grid4x5_k5", cases.SMALL["grid4x5_k5"])
    cutqc.reconstruct_fd(cc, to_dev(torch, [t.astype(np.float32) for t in T], torch.float32), algo="tc_bf16x3")
    cutqc.device_status()


def test_timed_out_wait_is_reported_and_context_survives(env):
    torch, cutqc = env
    from oracle import reconstruct as rc
    cutqc.selftest_wait(20000)
    with pytest.raises(cutqc.CutQCError) as ei:
        cutqc.device_status()
    assert ei.value.status == cutqc.CUTQC_ERR_TIMEOUT
    cutqc.device_status()          # the record was cleared
    # the same context still computes correct results
    cc, T = oracle_case("grid4x5_k5", cases.SMALL["grid4x5_k5"])
    T32 = [t.astype(np.float32) for t in T]
    out, sp = cutqc.reconstruct_fd(cc, to_dev(torch, T32, torch.float32), algo="tc_bf16x3")
    cutqc.device_status()
    ref = rc.fd_full(cc.subs, [t.astype(np.float64) for t in T32], cc.n, cc.n_cuts)
    assert np.abs(out.double().cpu().numpy() - ref).max() <= TOL32


def test_synchronising_call_reports_the_timeout(env):
    """cutqc_reconstruct_dd synchronises to read its top list and reports a
    timeout recorded before it."""
    torch, cutqc = env
    from paper_2012_02333_gb300 import dd
    cc, T = oracle_case("grid4x4_s4", cases.SMALL["grid4x4_s4"])
    ts = to_dev(torch, [t.astype(np.float32) for t in T], torch.float32)
    cutqc.selftest_wait(20000)
    with pytest.raises(cutqc.CutQCError) as ei:
        dd.run(cc, ts, 3, 1, "bfs")
    assert ei.value.status == cutqc.CUTQC_ERR_TIMEOUT
    st = dd.run(cc, ts, 3, 1, "bfs")
    assert len(st.recursions) == 1


def test_selftest_rejects_bad_limit(env):
    torch, cutqc = env
    with pytest.raises(cutqc.CutQCError) as ei:
        cutqc.selftest_wait(-1)
    assert ei.value.status == cutqc.CUTQC_ERR_ARG
