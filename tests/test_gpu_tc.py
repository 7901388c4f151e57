"""GPU parity of the tcgen05 split-precision contraction against the FP64
oracle (run on the same FP32 tensors).

BF16 x6 must meet 1e-6 max abs error everywhere; BF16 x3 must stay within its
a-priori bound 3 * 2^-18 * S + 1e-7 with S = 2^-K sum_e max|A_e| max|B_e|
(the bound the library's automatic choice uses); TF32 x3 within
3 * 2^-22 * S + 1e-7 and 1e-6; the automatic form must meet 1e-6
everywhere."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
import cases  # noqa: E402
from test_gpu_fd import env, oracle_case, to_dev  # noqa: E402,F401

pytestmark = pytest.mark.gpu

# shapes the tensor-core path takes: M = 2^fA >= 128 and N = 2^fB >= 256
TC_CASES = ["hwea16_s2", "grid4x5_k5"]


def split_bound(cc, T32):
    """S = 2^-K sum over non-zero terms e of max|A_e| * max|B_e| (two subcircuits)."""
    from oracle import reconstruct as rc
    mx = [np.abs(T.astype(np.float64)).reshape(T.shape[0] * T.shape[1], -1).max(axis=1) for T in T32]
    S = 0.0
    for e in range(4 ** cc.n_cuts):
        dg = [(e >> (2 * (cc.n_cuts - 1 - k))) & 3 for k in range(cc.n_cuts)]
        p = 1.0
        for s, m in zip(cc.subs, mx):
            p *= m[rc.row_of(s, dg)]
        S += p
    return S * 2.0 ** -cc.n_cuts


def run(env, name, algo):
    torch, cutqc = env
    from oracle import reconstruct as rc
    cc, Ts = oracle_case(name, cases.SMALL[name])
    T32 = [T.astype(np.float32) for T in Ts]
    ref = rc.fd_full(cc.subs, [T.astype(np.float64) for T in T32], cc.n, cc.n_cuts)
    out, sp = cutqc.reconstruct_fd(cc, to_dev(torch, T32, torch.float32), algo=algo)
    torch.cuda.synchronize()
    return cc, T32, ref, out.double().cpu().numpy(), float(sp.item()), cutqc.last_algo()


@pytest.mark.parametrize("name", TC_CASES)
def test_tc_bf16x3_within_bound(env, name):
    torch, cutqc = env
    cc, T32, ref, got, s, used = run(env, name, "tc_bf16x3")
    assert used == cutqc.CUTQC_TC_BF16X3
    bound = 3 * 2.0 ** -18 * split_bound(cc, T32) + 1e-7
    err = np.abs(got - ref).max()
    assert err <= bound, f"err {err:.3e} > bound {bound:.3e}"


@pytest.mark.parametrize("name", TC_CASES)
def test_tc_bf16x6_meets_1e6(env, name):
    torch, cutqc = env
    cc, T32, ref, got, s, used = run(env, name, "tc_bf16x6")
    assert used == cutqc.CUTQC_TC_BF16X6
    err = np.abs(got - ref).max()
    assert err <= 1e-6, f"err {err:.3e}"
    assert s == pytest.approx(ref.sum(), abs=1e-6)


@pytest.mark.parametrize("name", TC_CASES)
def test_tc_auto_meets_1e6(env, name):
    """The automatic form: the tensor-core path (x3 / x6 chosen on the
    device) for the 1024-term grid, the streaming CUDA-core form for the
    4-term chain (at most 16 terms: its output stream is all the work)."""
    torch, cutqc = env
    cc, T32, ref, got, s, used = run(env, name, "auto")
    assert used == (cutqc.CUTQC_CC if 4 ** cc.n_cuts <= 16 else cutqc.CUTQC_TC_BF16X3)
    err = np.abs(got - ref).max()
    assert err <= 1e-6, f"err {err:.3e}"


def test_tc_and_cc_agree_on_repeat(env):
    torch, cutqc = env
    cc, Ts = oracle_case("grid4x5_k5", cases.SMALL["grid4x5_k5"])
    ts = to_dev(torch, [T.astype(np.float32) for T in Ts], torch.float32)
    a, _ = cutqc.reconstruct_fd(cc, ts, algo="tc_bf16x6")
    b, _ = cutqc.reconstruct_fd(cc, ts, algo="tc_bf16x6")
    c, _ = cutqc.reconstruct_fd(cc, ts, algo="cc")
    assert torch.equal(a, b)
    assert (a.double() - c.double()).abs().max().item() <= 1e-6


@pytest.mark.parametrize("name", TC_CASES)
def test_tc_tf32x3_within_bound_and_1e6(env, name):
    """TF32 x3 (hi = tf32(x), lo = tf32(x - hi), products hh + hl + lh): the
    dropped lo*lo term and the rounding of lo bound the error per product by
    about 3 * 2^-22 |a||b|."""
    torch, cutqc = env
    cc, T32, ref, got, s, used = run(env, name, "tc_tf32x3")
    assert used == cutqc.CUTQC_TC_TF32X3
    bound = 3 * 2.0 ** -22 * split_bound(cc, T32) + 1e-7
    err = np.abs(got - ref).max()
    assert err <= min(bound, 1e-6), f"err {err:.3e} > bound {bound:.3e}"
    assert s == pytest.approx(ref.sum(), abs=1e-6)
    nseg, _ = cutqc.last_split()
    assert nseg == 3


def test_tc_tf32x3_more_accurate_than_bf16x3(env):
    """On the same shape TF32 x3 is at least as accurate as BF16 x3 (its
    dropped terms are 16 times smaller)."""
    torch, cutqc = env
    _, _, ref, g3, _, _ = run(env, "grid4x5_k5", "tc_bf16x3")
    _, _, _, gt, _, _ = run(env, "grid4x5_k5", "tc_tf32x3")
    assert np.abs(gt - ref).max() <= np.abs(g3 - ref).max() + 1e-12
