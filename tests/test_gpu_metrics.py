"""GPU parity of the Eq. 16 chi^2 loss, the total variation and
inverse-transform sampling against the FP64 oracle.  Distances: relative
1e-12 for FP64 inputs, 1e-6 for FP32 (the oracle sums the FP32-rounded
inputs in FP64).  Sampling returns indices: where the uniform does not fall
within 1e-11 of the total of a boundary of the cumulative sums the index must
equal the oracle's; every draw must be a valid inverse-transform outcome (its
interval of the exact FP64 cumulative sums, widened by that tolerance,
contains u * total) with positive weight."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
import cases  # noqa: E402
from test_gpu_fd import env, oracle_case, to_dev  # noqa: E402,F401

pytestmark = pytest.mark.gpu


def dist_pair(rng, n, zeros=False, negative=False):
    a = rng.random(n) ** 2
    b = rng.random(n) ** 2
    if zeros:
        z = rng.random(n) < 0.3
        a[z] = 0.0
        b[z] = 0.0
    if negative:
        a[rng.random(n) < 0.05] = -1e-9
    return a / a.sum(), b / b.sum()


@pytest.mark.parametrize("n", [1, 7, 1000, 4096, (1 << 20) + 3])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_distance_parity(env, n, dtype):
    torch, cutqc = env
    from oracle import metrics as mt
    rng = np.random.default_rng(n)
    for zeros, negative in [(False, False), (True, False), (True, True)]:
        a, b = dist_pair(rng, n, zeros, negative)
        if dtype == "f32":
            a, b = a.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
            tdt, tol = torch.float32, 1e-6
        else:
            tdt, tol = torch.float64, 1e-12
        chi, tv = cutqc.cutqc_distance(torch.tensor(a, dtype=tdt, device="cuda"),
                                       torch.tensor(b, dtype=tdt, device="cuda"))
        want_chi, want_tv = mt.chi_square(a, b), mt.total_variation(a, b)
        assert chi.item() == pytest.approx(want_chi, rel=tol, abs=1e-300)
        assert tv.item() == pytest.approx(want_tv, rel=tol, abs=1e-300)


def test_distance_of_reconstruction_to_ground_truth(env):
    """The reconstructed distribution of a cut circuit against the statevector
    ground truth of the uncut circuit (Fig. 2a): chi^2 equals the oracle's on
    the same two vectors, and is tiny (the reconstruction is exact up to
    FP32 / split-precision rounding, Sec. 3.2.3)."""
    torch, cutqc = env
    from oracle import metrics as mt
    from oracle import statevector as sv
    cc, T = oracle_case("grid4x5_k5", cases.SMALL["grid4x5_k5"])
    out, _ = cutqc.reconstruct_fd(cc, to_dev(torch, [t.astype(np.float32) for t in T], torch.float32))
    truth = sv.probabilities(cc.circuit)
    a = out.double().cpu().numpy()
    chi, tv = cutqc.cutqc_distance(out, torch.tensor(truth, dtype=torch.float32, device="cuda"))
    b32 = truth.astype(np.float32).astype(np.float64)
    assert chi.item() == pytest.approx(mt.chi_square(a, b32), rel=1e-5, abs=1e-12)
    assert tv.item() == pytest.approx(mt.total_variation(a, b32), rel=1e-5, abs=1e-12)
    assert chi.item() < 1e-6 and tv.item() < 1e-4


def blocked_cumulative(p64, block=1024):
    """The oracle's C_x = sum_{i <= x} max(p_i, 0) with less rounding for large
    inputs: pairwise block sums, their running sum, and running sums inside
    each block (a sequential sum over 2^28 values drifts by more than the
    tolerance of these checks)."""
    w = np.maximum(p64, 0.0)
    n = len(w)
    pad = (-n) % block
    wb = np.concatenate([w, np.zeros(pad)]).reshape(-1, block)
    starts = np.concatenate([[0.0], np.cumsum(wb.sum(axis=1))[:-1]])
    return (starts[:, None] + np.cumsum(wb, axis=1)).reshape(-1)[:n]


def check_draws(p64, u, got, tol_rel=1e-11):
    from oracle import metrics as mt
    C = mt.cumulative(p64) if len(p64) <= (1 << 21) else blocked_cumulative(p64)
    total = C[-1]
    t_all = u * total
    want = np.minimum(np.searchsorted(C, t_all, side="right"), len(C) - 1) if len(p64) > (1 << 21) \
        else mt.sample(p64, u)
    t = u * total
    tol = tol_rel * total
    w = np.maximum(p64, 0.0)
    assert (got >= 0).all() and (got < len(p64)).all()
    assert (w[got] > 0).all()
    lo = np.where(got > 0, C[np.maximum(got - 1, 0)], 0.0)
    hi = C[got]
    assert ((lo - tol <= t) & (t <= hi + tol)).all()
    # away from boundaries the draw is the oracle's
    prev = np.where(want > 0, C[np.maximum(want - 1, 0)], 0.0)
    clear = (np.abs(t - prev) > tol) & (np.abs(C[want] - t) > tol)
    assert (got[clear] == want[clear]).all()
    assert clear.mean() > 0.99


def test_sampling_from_unaligned_view(env):
    """FP32 weights that are element- but not 16-byte aligned (a view one
    entry into a buffer): whole chunks then come in by scalar loads instead of
    16-byte loads; the draws obey the same parity rule."""
    torch, cutqc = env
    n = (1 << 16) + 300
    rng = np.random.default_rng(77)
    p = rng.random(n) ** 3
    p[rng.random(n) < 0.3] = 0.0
    p /= p.sum()
    buf = torch.zeros(n + 1, dtype=torch.float32, device="cuda")
    buf[1:] = torch.tensor(p, dtype=torch.float32, device="cuda")
    view = buf[1:]
    assert view.data_ptr() % 16 == 4
    u = rng.random(50000)
    got = cutqc.cutqc_sample(view, torch.tensor(u, device="cuda")).cpu().numpy()
    check_draws(view.double().cpu().numpy(), u, got)


@pytest.mark.parametrize("n", [1, 5, 1024, 1025, 3000, (1 << 20) + 7])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_sampling_parity(env, n, dtype):
    torch, cutqc = env
    rng = np.random.default_rng(100 + n)
    p = rng.random(n) ** 4
    p[rng.random(n) < 0.2] = 0.0
    p[rng.random(n) < 0.02] = -1e-9
    if p.max() <= 0:
        p[0] = 1.0
    p /= np.maximum(p, 0).sum()
    tdt = torch.float64 if dtype == "f64" else torch.float32
    p_t = torch.tensor(p, dtype=tdt, device="cuda")
    p64 = p_t.double().cpu().numpy()
    u = rng.random(20000)
    u[:3] = [0.0, 0.5, np.nextafter(1.0, 0.0)]
    got = cutqc.cutqc_sample(p_t, torch.tensor(u, device="cuda")).cpu().numpy()
    check_draws(p64, u, got)


def test_sampling_special_cases(env):
    torch, cutqc = env
    u = torch.tensor(np.linspace(0.0, 0.999, 101), device="cuda")
    # a point mass in the last of several empty chunks
    p = torch.zeros(5000, device="cuda")
    p[4999] = 0.3
    assert (cutqc.cutqc_sample(p, u) == 4999).all()
    # only the first entry
    p = torch.zeros(5000, dtype=torch.float64, device="cuda")
    p[0] = 2.0
    assert (cutqc.cutqc_sample(p, u) == 0).all()
    # nothing has weight: -1
    p = torch.full((3000,), -1e-12, device="cuda")
    assert (cutqc.cutqc_sample(p, u) == -1).all()
    # no draws requested
    assert cutqc.cutqc_sample(p, torch.empty(0, dtype=torch.float64, device="cuda")).numel() == 0


def test_sampling_a_reconstruction(env):
    """Draws from the 2^24-entry reconstruction of the benchmark circuit:
    every draw valid against the exact cumulative sums of the returned FP32
    probabilities."""
    torch, cutqc = env
    from paper_2012_02333_gb300 import circuits as C
    cc = C.supremacy_4x6(0)
    ts = cutqc.simulate_tensors(cc, torch.float32)
    out, _ = cutqc.reconstruct_fd(cc, ts)
    rng = np.random.default_rng(9)
    u = rng.random(100000)
    got = cutqc.cutqc_sample(out, torch.tensor(u, device="cuda")).cpu().numpy()
    check_draws(out.double().cpu().numpy(), u, got)


def test_distance_benchmark_size_properties(env):
    """2^30 entries (the benchmark's size): properties that hold at any size
    -- chi^2(a, a) = 0, symmetry, chi^2 <= 2 and TV <= 1 for distributions,
    and the sum over a split of the index range equals the whole (the first
    2^20 entries checked against the oracle as well)."""
    torch, cutqc = env
    from oracle import metrics as mt
    n = 1 << 30
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    a = torch.rand(n, generator=g, device="cuda")
    a /= a.sum()
    b = torch.rand(n, generator=g, device="cuda")
    b /= b.sum()
    c0, t0 = cutqc.cutqc_distance(a, a)
    assert c0.item() == 0.0 and t0.item() == 0.0
    cab, tab = cutqc.cutqc_distance(a, b)
    cba, tba = cutqc.cutqc_distance(b, a)
    assert cab.item() == pytest.approx(cba.item(), rel=1e-6)
    assert tab.item() == pytest.approx(tba.item(), rel=1e-6)
    assert 0.0 < cab.item() <= 2.0 and 0.0 < tab.item() <= 1.0
    h = n // 2
    c1, t1 = cutqc.cutqc_distance(a[:h], b[:h])
    c2, t2 = cutqc.cutqc_distance(a[h:], b[h:])
    assert c1.item() + c2.item() == pytest.approx(cab.item(), rel=1e-6)
    assert t1.item() + t2.item() == pytest.approx(tab.item(), rel=1e-6)
    k = 1 << 20
    ck, tk = cutqc.cutqc_distance(a[:k], b[:k])
    aa, bb = a[:k].double().cpu().numpy(), b[:k].double().cpu().numpy()
    assert ck.item() == pytest.approx(mt.chi_square(aa, bb), rel=1e-6)
    assert tk.item() == pytest.approx(mt.total_variation(aa, bb), rel=1e-6)


def test_sampling_2e28_entries(env):
    """Draws from a 2^28-entry distribution with zero and negative runs, every
    draw valid against the exact FP64 cumulative sums."""
    torch, cutqc = env
    n = 1 << 28
    g = torch.Generator(device="cuda")
    g.manual_seed(4)
    p = torch.rand(n, generator=g, device="cuda") ** 8
    p[: 1 << 20] = 0.0
    p[1 << 25: (1 << 25) + 4096] = -1e-9
    u = np.random.default_rng(5).random(50000)
    got = cutqc.cutqc_sample(p, torch.tensor(u, device="cuda")).cpu().numpy()
    check_draws(p.double().cpu().numpy(), u, got)
