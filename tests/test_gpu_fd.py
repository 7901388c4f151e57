"""GPU parity of the full-definition reconstruction and of the GPU subcircuit
simulator against the FP64 oracle, through the C ABI.

Tolerances: the FP64 CUDA-core path must agree with the oracle to 1e-12 (only
rounding order differs); every FP32 path must agree to 1e-6 max abs error
(the target stated for this reconstruction) with the oracle run on the same
FP32-rounded tensors promoted to FP64, which isolates reconstruction error."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
import cases  # noqa: E402

pytestmark = pytest.mark.gpu

TOL32 = 1e-6
TOL64 = 1e-12


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


_cache = {}


def oracle_case(name, make):
    if name not in _cache:
        from oracle import attribution as at
        cc = make()
        _cache[name] = (cc, at.tensors(cc))
    return _cache[name]


def to_dev(torch, Ts, dtype):
    return [torch.tensor(np.ascontiguousarray(T).reshape(-1), dtype=dtype, device="cuda") for T in Ts]


@pytest.mark.parametrize("name", list(cases.SMALL))
def test_fd_cc_fp64(env, name):
    torch, cutqc = env
    from oracle import reconstruct as rc
    cc, Ts = oracle_case(name, cases.SMALL[name])
    ref = rc.fd_full(cc.subs, Ts, cc.n, cc.n_cuts)
    out, sp = cutqc.reconstruct_fd(cc, to_dev(torch, Ts, torch.float64), algo="cc")
    got = out.cpu().numpy()
    assert np.abs(got - ref).max() <= TOL64
    assert float(sp.item()) == pytest.approx(ref.sum(), abs=1e-12)


@pytest.mark.parametrize("algo", ["cc", "auto"])
@pytest.mark.parametrize("name", list(cases.SMALL))
def test_fd_fp32(env, name, algo):
    torch, cutqc = env
    from oracle import reconstruct as rc
    cc, Ts = oracle_case(name, cases.SMALL[name])
    T32 = [T.astype(np.float32) for T in Ts]
    ref = rc.fd_full(cc.subs, [T.astype(np.float64) for T in T32], cc.n, cc.n_cuts)
    out, sp = cutqc.reconstruct_fd(cc, to_dev(torch, T32, torch.float32), algo=algo)
    got = out.double().cpu().numpy()
    err = np.abs(got - ref).max()
    assert err <= TOL32, f"max abs err {err:.3e}"
    assert float(sp.item()) == pytest.approx(ref.sum(), abs=TOL32)


@pytest.mark.parametrize("name", ["hwea10_k1", "qaoa8_k4", "grid4x4_s4", "aqft8_k4", "bv6_k1"])
def test_gpu_simulator_matches_oracle(env, name):
    torch, cutqc = env
    cc, Ts = oracle_case(name, cases.SMALL[name])
    for sub, T in zip(cc.subs, Ts):
        g = cutqc.cutqc_simulate_subcircuit(sub, torch.float64).cpu().numpy()
        assert np.abs(g - T.reshape(-1)).max() < 1e-12
        g32 = cutqc.cutqc_simulate_subcircuit(sub, torch.float32).cpu().numpy()
        assert np.abs(g32 - T.reshape(-1).astype(np.float32)).max() <= 2 * np.finfo(np.float32).eps * max(1.0, np.abs(T).max())


def test_repeated_calls_reuse_plan_and_agree(env):
    torch, cutqc = env
    cc, Ts = oracle_case("grid4x4_s4", cases.SMALL["grid4x4_s4"])
    ts = to_dev(torch, [T.astype(np.float32) for T in Ts], torch.float32)
    a, _ = cutqc.reconstruct_fd(cc, ts, algo="cc")
    b, _ = cutqc.reconstruct_fd(cc, ts, algo="cc")
    assert torch.equal(a, b)        # deterministic: stable compaction, fixed order


def test_host_tensors_end_to_end(env):
    torch, cutqc = env
    from oracle import reconstruct as rc
    cc, Ts = oracle_case("grid3x4_k3", cases.SMALL["grid3x4_k3"])
    host = [torch.tensor(T.reshape(-1).astype(np.float32)).pin_memory() for T in Ts]
    out, sp = cutqc.reconstruct_fd(cc, host)
    ref = rc.fd_full(cc.subs, [T.astype(np.float32).astype(np.float64) for T in Ts], cc.n, cc.n_cuts)
    assert np.abs(out.double().cpu().numpy() - ref).max() <= TOL32


@pytest.fixture(scope="module")
def sup(env):
    """The 24-qubit 4x6 supremacy workload at full size: oracle tensors (FP64
    CPU simulation), rounded to FP32 for both sides."""
    cc, Ts = oracle_case("sup4x6", cases.supremacy_4x6)
    return cc, [T.astype(np.float32) for T in Ts]


def test_misaligned_output_is_rejected(env, sup):
    """A device output one element off the 16-byte grid (a tensor view) is an
    argument error before anything is launched; the vector stores never see
    it.  A 16-byte aligned view that is not 32-byte aligned is accepted and
    gives the same result as a fresh buffer: on the 4x6 workload the
    tensor-core epilogue writes 8 consecutive outputs per 32-byte store, and
    falls back to 16-byte stores for that view."""
    torch, cutqc = env
    cc, T32 = sup
    ts = to_dev(torch, T32, torch.float32)
    ref, _ = cutqc.reconstruct_fd(cc, ts, algo="tc_bf16x3")
    big = torch.full((2 ** cc.n + 8,), -1.0, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    n0 = cutqc.launch_count()
    with pytest.raises(cutqc.CutQCError, match="16-byte"):
        cutqc.reconstruct_fd(cc, ts, algo="tc_bf16x3", out=big[1:1 + 2 ** cc.n])
    assert cutqc.launch_count() == n0
    view = big[4:4 + 2 ** cc.n]
    assert view.data_ptr() % 32 == 16
    o, _ = cutqc.reconstruct_fd(cc, ts, algo="tc_bf16x3", out=view)
    torch.cuda.synchronize()
    assert torch.equal(view, ref)
    assert torch.all(big[:4] == -1.0) and torch.all(big[4 + 2 ** cc.n:] == -1.0)


_sup_ref = {}


@pytest.mark.parametrize("algo", ["cc", "auto", "tc_bf16x3", "tc_bf16x6", "tc_tf32x3"])
def test_supremacy_4x6_full_size(env, sup, algo):
    """Full size (2^24 outputs, the launch configuration the benchmark times):
    every output against the oracle's plain FP64 sum over all 256 Kronecker
    terms on the same FP32 tensors, plus the FP64 sum against the closed form
    over the FP32 tensors.  On this shape the bf16 forms prepare their
    operands in one pass (one block per term, 176 of 256 kept, zero rows up to
    the end of the last stage) and the contraction cuts its last round of
    tiles into 128-column halves over more CTAs; those outputs are among the
    ones compared."""
    torch, cutqc = env
    from oracle import reconstruct as rc
    cc, T32 = sup
    if "ref" not in _sup_ref:
        _sup_ref["ref"] = rc.fd_full(cc.subs, [T.astype(np.float64) for T in T32], cc.n, cc.n_cuts)
    ref = _sup_ref["ref"]
    out, sp = cutqc.reconstruct_fd(cc, to_dev(torch, T32, torch.float32), algo=algo)
    got = out.double().cpu().numpy()
    err = np.abs(got - ref).max()
    assert err <= TOL32, f"max abs err {err:.3e}"
    # the fused FP64 sum is the sum of the returned outputs
    assert float(sp.item()) == pytest.approx(got.sum(), abs=1e-9)
    # closed form: sum_x p(x) = 2^-K sum_e prod_c sum_x T_c[e|c][x], within the
    # aggregate error bound (3 * 2^-18 split + K_eff * 2^-23 FP32 accumulation)
    # * sum_x S_x, where sum_x S_x = 2^-K sum_e prod_c ||T_c[e|c]||_1
    rows = [T.astype(np.float64).reshape(T.shape[0] * T.shape[1], -1) for T in T32]
    sums = [r.sum(axis=1) for r in rows]
    l1 = [np.abs(r).sum(axis=1) for r in rows]
    total, s_l1, k_eff = 0.0, 0.0, 0
    for e in range(4 ** cc.n_cuts):
        dg = [(e >> (2 * (cc.n_cuts - 1 - k))) & 3 for k in range(cc.n_cuts)]
        prod, pl1 = 1.0, 1.0
        for s, v, a in zip(cc.subs, sums, l1):
            r = rc.row_of(s, dg)
            prod *= v[r]
            pl1 *= a[r]
        total += prod
        s_l1 += pl1
        k_eff += pl1 > 0
    total *= 2.0 ** -cc.n_cuts
    s_l1 *= 2.0 ** -cc.n_cuts
    tol = (3 * 2.0 ** -18 + k_eff * 2.0 ** -23) * s_l1 + 1e-9   # covers every split form
    assert abs(float(sp.item()) - total) <= tol, (float(sp.item()) - total, tol)
    assert abs(float(sp.item()) - 1.0) <= tol + 1e-6    # trace preservation of the uncut circuit


@pytest.mark.parametrize("algo", ["tc_bf16x3", "tc_bf16x6", "tc_tf32x3"])
def test_large_output_sampled(env, algo):
    """2^26 outputs (256 MiB of FP32, larger than L2): a 26-qubit HWEA chain
    cut once into two 13-qubit halves.  At this size the tensor-core epilogue
    restages its blocks through shared memory and stores them in output-address
    order; 4096 sampled outputs are checked against the oracle's plain sum and
    the fused FP64 sum against the sum of the returned outputs."""
    torch, cutqc = env
    from oracle import reconstruct as rc
    cc, Ts = oracle_case("hwea26_s2", cases.hwea26_chain)
    T32 = [T.astype(np.float32) for T in Ts]
    out, sp = cutqc.reconstruct_fd(cc, to_dev(torch, T32, torch.float32), algo=algo)
    assert cutqc.last_algo() == cutqc.ALGOS[algo]
    got = out.double().cpu().numpy()
    rng = np.random.default_rng(12)
    xs = sorted(set(int(x) for x in rng.integers(0, 2 ** cc.n, 4096)) | {0, 1, 2, 3, 2 ** cc.n - 1})
    want = rc.fd_entries(cc.subs, [T.astype(np.float64) for T in T32], cc.n, cc.n_cuts, xs)
    err = np.abs(got[xs] - want).max()
    assert err <= TOL32, f"max abs err {err:.3e}"
    assert float(sp.item()) == pytest.approx(got.sum(), abs=1e-9)
    assert float(sp.item()) == pytest.approx(1.0, abs=1e-5)
    del out
    torch.cuda.empty_cache()


def test_supremacy_gpu_simulated_inputs(env, sup):
    """The benchmark's own input preparation (GPU simulator) reproduces the
    oracle's FP32 tensors of the full-size workload."""
    torch, cutqc = env
    cc, T32 = sup
    for s, T in zip(cc.subs, T32):
        g = cutqc.cutqc_simulate_subcircuit(s, torch.float32).cpu().numpy()
        assert np.abs(g - T.reshape(-1)).max() <= 1e-6


@pytest.mark.parametrize("algo", ["cc", "tc_bf16x3"])
def test_output_into_pinned_host_memory(env, algo):
    """out may be pinned host memory: the contraction writes the probabilities
    into it directly; the result equals the device-output call exactly (the
    same kernels and summation order), and the FP64 sum matches."""
    torch, cutqc = env
    cc, Ts = oracle_case("hwea26_s2", cases.hwea26_chain)
    ts = to_dev(torch, [T.astype(np.float32) for T in Ts], torch.float32)
    dev_out, dev_sp = cutqc.reconstruct_fd(cc, ts, algo=algo)
    host_out = torch.full((2 ** cc.n,), -1.0, dtype=torch.float32).pin_memory()
    o, sp = cutqc.reconstruct_fd(cc, ts, algo=algo, out=host_out)
    torch.cuda.synchronize()
    assert o.data_ptr() == host_out.data_ptr()
    assert torch.equal(host_out, dev_out.cpu())
    assert float(sp.item()) == pytest.approx(float(dev_sp.item()), abs=1e-9)


def test_unregistered_host_output_is_rejected(env):
    """Pageable host memory is refused before anything is launched."""
    torch, cutqc = env
    cc, Ts = oracle_case("hwea10_k1", cases.SMALL["hwea10_k1"])
    p = cutqc.Problem.from_cut(cc, to_dev(torch, Ts, torch.float64))
    buf = np.zeros(2 ** cc.n, dtype=np.float64)
    arr = (cutqc.C.c_void_p * 1)(buf.ctypes.data)
    st = cutqc._lib.cutqc_reconstruct_fd(cutqc.C.byref(p.c), 1, arr, cutqc.CUTQC_AUTO, None,
                                          cutqc._stream_ptr(None))
    assert st == cutqc.CUTQC_ERR_ARG
    assert "pinned" in cutqc._lib.cutqc_last_error().decode()


@pytest.mark.parametrize("make,D,nC", [(lambda C: C.hwea(10, 4), 6, 2), (lambda C: C.bv(8, 3), 5, 2),
                                       (lambda C: C.hwea(9, 5), 4, 3)])
def test_reconstruction_of_searched_cuts(env, make, D, nC):
    """End to end from the cut searcher (Sec. 4.1): the least-cost cut of the
    circuit, its subcircuits' tensors (oracle simulation), the GPU
    reconstruction in FP64 (CUDA core) and FP32 (automatic form), against the
    statevector of the uncut circuit (exactness, Sec. 3.2.3)."""
    torch, cutqc = env
    from oracle import attribution as at
    from oracle import statevector as sv
    from paper_2012_02333_gb300 import circuits as C
    circ = make(C)
    r = cutqc.cut_search(circ, D, nC)
    cc = C.cut_from_clusters(circ, r["gate_cluster"], max_width=D)
    assert cc.n_cuts == r["K"] and max(s.d for s in cc.subs) <= D
    T = at.tensors(cc)
    truth = sv.probabilities(cc.circuit)
    out64, _ = cutqc.reconstruct_fd(cc, to_dev(torch, T, torch.float64), algo="cc")
    assert np.abs(out64.cpu().numpy() - truth).max() <= 1e-12
    out32, _ = cutqc.reconstruct_fd(cc, to_dev(torch, [t.astype(np.float32) for t in T], torch.float32))
    assert np.abs(out32.double().cpu().numpy() - truth).max() <= TOL32


@pytest.mark.parametrize("algo", ["cc", "auto"])
def test_single_row_operands_of_long_rows(env, algo):
    """Two uncut blocks of 20 and 4 qubits (K = 0: one Kronecker term, both
    operands a single row, one of 2^20 entries): the row statistics split the
    long row over many blocks and combine the chunks; all 2^24 outputs against
    the oracle."""
    torch, cutqc = env
    from oracle import reconstruct as rc
    from paper_2012_02333_gb300 import circuits as C
    cc, Ts = oracle_case("hwea24_k0", lambda: C.cut_circuit(C.hwea(24, 3), [0] * 20 + [1] * 4, max_cuts=0))
    assert cc.n_cuts == 0 and len(cc.subs) == 2
    T32 = [T.astype(np.float32) for T in Ts]
    ref = rc.fd_full(cc.subs, [T.astype(np.float64) for T in T32], cc.n, cc.n_cuts)
    out, sp = cutqc.reconstruct_fd(cc, to_dev(torch, T32, torch.float32), algo=algo)
    assert np.abs(out.double().cpu().numpy() - ref).max() <= TOL32
    assert float(sp.item()) == pytest.approx(ref.sum(), abs=TOL32)


@pytest.mark.parametrize("algo", ["tc_bf16x3", "tc_tf32x3", "tc_bf16x6"])
def test_qaoa30_forward_full_size(env, algo):
    """The 30-qubit QAOA workload's forward (2^30 outputs, 32768 tiles: 215
    per CTA, the epilogue restaged through shared memory) in every split form:
    4096 sampled outputs against the oracle's plain sum (oracle-simulated
    tensors rounded to FP32), and the fused FP64 sum against the sum of the
    outputs."""
    torch, cutqc = env
    from oracle import reconstruct as rc
    from paper_2012_02333_gb300 import circuits as C
    cc, Ts = oracle_case("qaoa30", lambda: C.qaoa_2cluster(15, 0))
    T32 = [T.astype(np.float32) for T in Ts]
    out, sp = cutqc.reconstruct_fd(cc, to_dev(torch, T32, torch.float32), algo=algo)
    assert cutqc.last_algo() == cutqc.ALGOS[algo]
    rng = np.random.default_rng(30)
    xs = sorted(set(int(x) for x in rng.integers(0, 2 ** cc.n, 4096)) | {0, 2 ** cc.n - 1})
    got = out[torch.tensor(xs, device="cuda")].double().cpu().numpy()
    want = rc.fd_entries(cc.subs, [T.astype(np.float64) for T in T32], cc.n, cc.n_cuts, xs)
    err = np.abs(got - want).max()
    assert err <= TOL32, f"max abs err {err:.3e}"
    assert float(sp.item()) == pytest.approx(torch.sum(out, dtype=torch.float64).item(), abs=1e-6)
    del out
    torch.cuda.empty_cache()
