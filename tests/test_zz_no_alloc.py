"""The allocation-free full-definition entry point (for callers that cannot
let the library call cudaMalloc: device memory reserved up front by another
allocator, or no device allocation allowed after start-up).

It must give what cutqc_reconstruct_fd gives with the CUDA-core form, within
the tolerances of the other parity tests (1e-6 for FP32, 1e-12 for FP64), on
two calls in a row that share its static scratch array - different problems,
so the second call cannot lean on what the first left behind.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if not os.path.exists(os.path.join(root, "paper_2012_02333_gb300", "libcutqc.so")):
        from paper_2012_02333_gb300 import build
        build.build()
    from paper_2012_02333_gb300 import cutqc
    return torch, cutqc


def _case(cutqc, torch, make, dtype):
    cc = make()
    ts = cutqc.simulate_tensors(cc, dtype, torch.device("cuda"))
    return cc, ts


def test_noalloc_matches_fd_on_two_calls_in_a_row(env):
    torch, cutqc = env
    from paper_2012_02333_gb300 import circuits as C
    runs = [
        (lambda: C.supremacy_4x6(0), torch.float32, 1e-6),     # the benchmark workload, K = 4
        (lambda: C.qaoa_2cluster(6, 1), torch.float64, 1e-12),  # a different shape and dtype, K = 4
    ]
    for make, dtype, tol in runs:
        cc, ts = _case(cutqc, torch, make, dtype)
        problem = cutqc.Problem.from_cut(cc, ts)
        ref = torch.empty(2 ** cc.n, dtype=dtype, device="cuda")
        ref_sum = torch.empty(1, dtype=torch.float64, device="cuda")
        cutqc.cutqc_reconstruct_fd([problem], [ref], "cc", ref_sum)
        got = torch.full((2 ** cc.n,), float("nan"), dtype=dtype, device="cuda")
        got_sum = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        cutqc.cutqc_reconstruct_fd_noalloc(problem, got, got_sum)
        torch.cuda.synchronize()
        err = (got.double() - ref.double()).abs().max().item()
        assert err <= tol, f"max abs difference {err:.3e}"
        assert abs(got_sum.item() - ref_sum.item()) <= max(tol, 1e-9)


def test_noalloc_rejects_problems_beyond_its_scratch(env):
    torch, cutqc = env
    import ctypes as C
    # two subcircuits joined by 10 cuts: the row maps alone exceed the 4 MiB array
    k = 10
    subs = (cutqc.cutqc_subcircuit * 2)()
    a_out, b_in = cutqc._i32(list(range(k))), cutqc._i32(list(range(k)))
    q0, q1 = cutqc._i32([0]), cutqc._i32([1])
    t0 = torch.zeros((4 ** k) * 2, device="cuda")
    t1 = torch.zeros((4 ** k) * 2, device="cuda")
    subs[0] = cutqc.cutqc_subcircuit(0, k, 1, None, a_out, q0, C.c_void_p(t0.data_ptr()))
    subs[1] = cutqc.cutqc_subcircuit(k, 0, 1, b_in, None, q1, C.c_void_p(t1.data_ptr()))
    prob = cutqc.cutqc_problem(2, k, 2, cutqc.CUTQC_F32, subs)
    out = torch.empty(4, device="cuda")
    st = cutqc._lib.cutqc_reconstruct_fd_noalloc(C.byref(prob), C.c_void_p(out.data_ptr()), None, None)
    assert st == cutqc.CUTQC_ERR_UNSUPPORTED
    assert "scratch" in cutqc.last_error()
