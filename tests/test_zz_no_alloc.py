"""The allocation-free full-definition entry point (for callers that cannot
let the library call cudaMalloc: device memory reserved up front by another
allocator, or no device allocation allowed after start-up).

Its outputs are compared with the FP64 oracle's plain sum on the same tensors
(oracle-simulated, rounded to FP32 for the FP32 cases) and with the
allocating entry point's (cutqc_reconstruct_fd, CUDA-core form) on the same
problem, within the tolerances of the other parity tests (1e-6 for FP32,
1e-12 for FP64), on two calls in a row that share its static scratch
array - different problems and dtypes, so
the second call cannot lean on what the first left behind - including a
K = 8 problem near the array's limit.  The same calls also run in a fresh
process that never touches the library's allocating entry points, where the
device's free memory must not change across repeated rounds of them.  This file is collected
last so that a run stopping at the first failure has already run every other
test; it also passes alone in a fresh process."""
import os
import subprocess
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
import cases  # noqa: E402

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(os.path.join(ROOT, "paper_2012_02333_gb300", "libcutqc.so")):
        from paper_2012_02333_gb300 import build
        build.build()
    from paper_2012_02333_gb300 import cutqc
    return torch, cutqc


# (case, dtype name, tolerance): the K = 8 pair needs 2.3 MB of the 4 MiB scratch
RUNS = [("k8_pair", "float32", 1e-6), ("qaoa8_k4", "float64", 1e-12), ("grid4x5_k5", "float32", 1e-6)]


def _make(name):
    return cases.k8_pair() if name == "k8_pair" else cases.SMALL[name]()


def _oracle(name, dtype_name):
    """(cut circuit, tensors in the call's dtype, the oracle's FP64 result on them)."""
    from oracle import attribution as at
    from oracle import reconstruct as rc
    cc = _make(name)
    T = [t.astype(np.float32 if dtype_name == "float32" else np.float64) for t in at.tensors(cc)]
    ref = rc.fd_full(cc.subs, [t.astype(np.float64) for t in T], cc.n, cc.n_cuts)
    return cc, T, ref


def test_noalloc_matches_oracle_on_calls_in_a_row(env):
    torch, cutqc = env
    prepared = []
    for name, dtn, tol in RUNS:
        cc, T, ref = _oracle(name, dtn)
        dt = getattr(torch, dtn)
        ts = [torch.tensor(t.reshape(-1), dtype=dt, device="cuda") for t in T]
        prepared.append((cutqc.Problem.from_cut(cc, ts), ts, dt, ref, tol, cc))
    # the allocating entry point's results on the same problems
    alloc = []
    for problem, ts, dt, ref, tol, cc in prepared:
        o = torch.full((2 ** cc.n,), float("nan"), dtype=dt, device="cuda")
        sp = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        cutqc.cutqc_reconstruct_fd([problem], [o], "cc", sp)
        torch.cuda.synchronize()
        alloc.append((o.double().cpu().numpy(), sp.item()))
    for _ in range(2):   # every problem twice, interleaved
        for (problem, ts, dt, ref, tol, cc), (a_out, a_sum) in zip(prepared, alloc):
            got = torch.full((2 ** cc.n,), float("nan"), dtype=dt, device="cuda")
            got_sum = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            cutqc.cutqc_reconstruct_fd_noalloc(problem, got, got_sum)
            torch.cuda.synchronize()
            g = got.double().cpu().numpy()
            err = np.abs(g - ref).max()
            assert err <= tol, f"{cc.n} qubits, K={cc.n_cuts}: max abs error {err:.3e}"
            assert abs(got_sum.item() - ref.sum()) <= max(tol, 1e-9)
            assert np.abs(g - a_out).max() <= tol, f"{cc.n} qubits: differs from cutqc_reconstruct_fd"
            assert abs(got_sum.item() - a_sum) <= max(tol, 1e-9)


_FRESH = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import test_zz_no_alloc as t
from paper_2012_02333_gb300 import cutqc
prepared = []
for name, dtn, tol in t.RUNS:
    cc, T, ref = t._oracle(name, dtn)
    dt = getattr(torch, dtn)
    ts = [torch.tensor(x.reshape(-1), dtype=dt, device="cuda") for x in T]
    out = torch.full((2 ** cc.n,), float("nan"), dtype=dt, device="cuda")
    sp = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    prepared.append((cutqc.Problem.from_cut(cc, ts), ts, out, sp, ref, tol))
torch.cuda.synchronize()
free = [torch.cuda.mem_get_info()[0]]
for rnd in range(3):
    for problem, ts, out, sp, ref, tol in prepared:
        cutqc.cutqc_reconstruct_fd_noalloc(problem, out, sp)
        torch.cuda.synchronize()
        err = np.abs(out.cpu().double().numpy() - ref).max()   # no device allocation between the readings
        assert err <= tol, ("round", rnd, err)
        assert abs(sp.item() - ref.sum()) <= max(tol, 1e-9)
    torch.cuda.synchronize()
    free.append(torch.cuda.mem_get_info()[0])
print("free bytes", free)
# after the first round (where the driver may still reserve memory of its
# own, such as local memory for kernels' stacks on their first launch) the
# calls change the device's free memory by nothing at all
assert free[1] == free[2] == free[3], free
print("NOALLOC_FRESH_OK")
"""


def test_noalloc_in_a_fresh_process_allocates_nothing(env):
    code = _FRESH.format(root=ROOT, tests=os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0 and "NOALLOC_FRESH_OK" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]


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


def test_noalloc_rejects_outputs_it_cannot_write(env):
    """Pageable host memory as out, or a host pointer as sum_p, is refused with
    CUTQC_ERR_ARG before anything is launched."""
    torch, cutqc = env
    import ctypes as C
    from oracle import attribution as at
    cc = cases.SMALL["hwea10_k1"]()
    ts = [torch.tensor(t.reshape(-1), dtype=torch.float64, device="cuda") for t in at.tensors(cc)]
    problem = cutqc.Problem.from_cut(cc, ts)
    torch.cuda.synchronize()
    n0 = cutqc.launch_count()
    host_out = torch.zeros(2 ** cc.n, dtype=torch.float64)          # pageable
    st = cutqc._lib.cutqc_reconstruct_fd_noalloc(C.byref(problem.c), C.c_void_p(host_out.data_ptr()), None, None)
    assert st == cutqc.CUTQC_ERR_ARG
    dev_out = torch.zeros(2 ** cc.n, dtype=torch.float64, device="cuda")
    host_sum = torch.zeros(1, dtype=torch.float64)
    st = cutqc._lib.cutqc_reconstruct_fd_noalloc(C.byref(problem.c), C.c_void_p(dev_out.data_ptr()),
                                                 C.c_void_p(host_sum.data_ptr()), None)
    assert st == cutqc.CUTQC_ERR_ARG
    assert cutqc.launch_count() == n0
    with pytest.raises(ValueError):   # a strided view of 2^n entries
        cutqc.cutqc_reconstruct_fd_noalloc(problem, torch.zeros(2 * 2 ** cc.n, dtype=torch.float64,
                                                                device="cuda")[::2])
