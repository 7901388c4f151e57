"""GPU parity of the adjoint (dL/dT for L = sum_x G(x) p(x)) against the FP64
oracle's chain rule, central differences, autograd, and the full-size QAOA
MaxCut workload (30 qubits, K = 4) on sampled gradient entries."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
import cases  # noqa: E402
from test_gpu_fd import env, oracle_case, to_dev  # noqa: E402,F401

pytestmark = pytest.mark.gpu

TWO_SUB = ["hwea10_k1", "bv6_k1", "grid3x4_k3", "qaoa8_k4", "hwea16_s2", "grid4x5_k5"]
# three and four subcircuits: each subcircuit against the group tensor of the
# others, rebuilt by the forward's group builds
MULTI_SUB = ["hwea9_s3", "grid4x4_s4"]


def rel_err(got, want):
    return np.abs(got - want).max() / max(1.0, np.abs(want).max())


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("name", TWO_SUB + MULTI_SUB)
def test_backward_explicit_G(env, name, dtype):
    torch, cutqc = env
    from oracle import reconstruct as rc
    cc, Ts = oracle_case(name, cases.SMALL[name])
    npdt, tdt, tol = (np.float64, torch.float64, 1e-12) if dtype == "f64" else (np.float32, torch.float32, 2e-6)
    Tq = [T.astype(npdt) for T in Ts]
    rng = np.random.default_rng(7)
    G = rng.uniform(-1, 1, 2 ** cc.n).astype(npdt)
    want = rc.grad(cc.subs, [T.astype(np.float64) for T in Tq], cc.n, cc.n_cuts, G.astype(np.float64))
    ts = to_dev(torch, Tq, tdt)
    problem = cutqc.Problem.from_cut(cc, ts)
    grads = [torch.empty_like(t) for t in ts]
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    cutqc.cutqc_reconstruct_backward(problem, grads, grad_out=torch.tensor(G, device="cuda"), loss_value=loss)
    for g, w in zip(grads, want):
        assert rel_err(g.double().cpu().numpy(), w.reshape(-1)) <= tol
    p = rc.fd_full(cc.subs, [T.astype(np.float64) for T in Tq], cc.n, cc.n_cuts)
    assert loss.item() == pytest.approx(float(G.astype(np.float64) @ p), abs=tol * max(1, np.abs(G).sum() * 1e-3))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("name", ["qaoa8_k4", "hwea10_k1", "grid3x4_k3"] + MULTI_SUB)
def test_backward_maxcut(env, name, dtype):
    torch, cutqc = env
    from oracle import reconstruct as rc
    from oracle import statevector as sv
    cc, Ts = oracle_case(name, cases.SMALL[name])
    edges = getattr(cc, "edges", None) or [(q, q + 1) for q in range(cc.n - 1)] + [(0, cc.n - 1)]
    npdt, tdt, tol = (np.float64, torch.float64, 1e-12) if dtype == "f64" else (np.float32, torch.float32, 2e-6)
    Tq = [T.astype(npdt) for T in Ts]
    Cx = rc.maxcut_values(cc.n, edges)
    want = rc.grad(cc.subs, [T.astype(np.float64) for T in Tq], cc.n, cc.n_cuts, Cx)
    ts = to_dev(torch, Tq, tdt)
    problem = cutqc.Problem.from_cut(cc, ts)
    grads = [torch.empty_like(t) for t in ts]
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    cutqc.cutqc_reconstruct_backward(problem, grads, edges=edges, loss_value=loss)
    for g, w in zip(grads, want):
        assert rel_err(g.double().cpu().numpy(), w.reshape(-1)) <= tol
    brute = float(Cx @ sv.probabilities(cc.circuit))
    assert loss.item() == pytest.approx(brute, abs=1e-5 if dtype == "f32" else 1e-11)


@pytest.mark.parametrize("name", ["qaoa8_k4", "grid4x4_s4"])
def test_backward_central_differences_fp64(env, name):
    """L is linear in each tensor: FP64 central differences (h = 1e-6) of the
    library's own loss value match its gradient."""
    torch, cutqc = env
    cc, Ts = oracle_case(name, cases.SMALL[name])
    ts = to_dev(torch, Ts, torch.float64)
    edges = getattr(cc, "edges", None) or [(q, q + 1) for q in range(cc.n - 1)] + [(0, cc.n - 1)]

    def loss_of(tensors):
        problem = cutqc.Problem.from_cut(cc, tensors)
        grads = [torch.empty_like(t) for t in tensors]
        lv = torch.empty(1, dtype=torch.float64, device="cuda")
        cutqc.cutqc_reconstruct_backward(problem, grads, edges=edges, loss_value=lv)
        return lv.item(), grads

    L0, grads = loss_of(ts)
    h = 1e-6
    rng = np.random.default_rng(1)
    for c in range(len(ts)):
        for i in rng.choice(ts[c].numel(), 6, replace=False):
            tp = [t.clone() for t in ts]
            tm = [t.clone() for t in ts]
            tp[c][i] += h
            tm[c][i] -= h
            fd = (loss_of(tp)[0] - loss_of(tm)[0]) / (2 * h)
            assert grads[c][i].item() == pytest.approx(fd, abs=1e-8)


def test_autograd_functions(env):
    torch, cutqc = env
    from paper_2012_02333_gb300.autograd import MaxCutExpectation, Reconstruct
    from oracle import reconstruct as rc
    cc, Ts = oracle_case("qaoa8_k4", cases.SMALL["qaoa8_k4"])
    ts = [t.requires_grad_(True) for t in to_dev(torch, Ts, torch.float64)]
    Cx = torch.tensor(rc.maxcut_values(cc.n, cc.edges), device="cuda")
    p = Reconstruct.apply(cc, "cc", *ts)
    L1 = (p * Cx).sum()
    g1 = torch.autograd.grad(L1, ts)
    L2 = MaxCutExpectation.apply(cc, cc.edges, *ts)
    g2 = torch.autograd.grad(L2, ts)
    assert L1.item() == pytest.approx(L2.item(), abs=1e-12)
    for a, b in zip(g1, g2):
        assert (a - b).abs().max().item() <= 1e-12


def test_qaoa30_maxcut_full_size(env):
    """The 30-qubit QAOA MaxCut workload (two 15-node clusters, 2 bridges,
    K = 4; the oracle's simulated tensors rounded to FP32 for both sides): 64
    sampled gradient entries per subcircuit against the oracle's chain rule,
    Euler's identity L = sum T * dL/dT for each side, and FP64 central
    differences of the loss."""
    torch, cutqc = env
    from oracle import reconstruct as rc
    from paper_2012_02333_gb300 import circuits as C
    cc, Ts = oracle_case("qaoa30", lambda: C.qaoa_2cluster(15, 0))
    assert cc.n == 30 and cc.n_cuts == 4
    ts = to_dev(torch, [T.astype(np.float32) for T in Ts], torch.float32)
    problem = cutqc.Problem.from_cut(cc, ts)
    grads = [torch.empty_like(t) for t in ts]
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    cutqc.cutqc_reconstruct_backward(problem, grads, edges=cc.edges, loss_value=loss)
    T64 = [t.double().cpu().numpy().reshape(4 ** s.k_in, 4 ** s.k_out, -1) for t, s in zip(ts, cc.subs)]
    g64 = [g.double().cpu().numpy() for g in grads]
    L = loss.item()
    assert 0 < L < len(cc.edges)
    for T, g in zip(T64, g64):
        assert float(T.reshape(-1) @ g) == pytest.approx(L, rel=1e-5)
    f = rc.maxcut_of(cc.n, cc.edges)
    rng = np.random.default_rng(3)
    for c, s in enumerate(cc.subs):
        rows = 4 ** (s.k_in + s.k_out)
        for _ in range(64):
            r, x = int(rng.integers(rows)), int(rng.integers(2 ** s.n_eff))
            want = rc.grad_entry(cc.subs, T64, cc.n, cc.n_cuts, c, r, x, f)
            got = g64[c][r * 2 ** s.n_eff + x]
            assert got == pytest.approx(want, abs=2e-6 * max(1.0, abs(want)))
    # central differences in FP64 on a few entries
    t64 = [t.double() for t in ts]

    def loss_of(tensors):
        pr = cutqc.Problem.from_cut(cc, tensors)
        gs = [torch.empty_like(t) for t in tensors]
        lv = torch.empty(1, dtype=torch.float64, device="cuda")
        cutqc.cutqc_reconstruct_backward(pr, gs, edges=cc.edges, loss_value=lv)
        return lv.item(), gs

    L64, gs64 = loss_of(t64)
    h = 1e-6
    for c in range(2):
        for i in rng.choice(t64[c].numel(), 3, replace=False):
            tp = [t.clone() for t in t64]
            tm = [t.clone() for t in t64]
            tp[c][i] += h
            tm[c][i] -= h
            fd = (loss_of(tp)[0] - loss_of(tm)[0]) / (2 * h)
            assert gs64[c][i].item() == pytest.approx(fd, abs=1e-6)
