"""GPU parity of the attribution entry point (Sec. 3.2.2, Eq. 2 then Eq. 3):
variant distributions -> Pauli-indexed subcircuit tensors, against the FP64
oracle's einsum form of the same equations, element by element.  Inputs: the
oracle's own simulated variant distributions of the test circuits, and seeded
random distributions (any non-negative numbers normalised per variant, as from
shot counts) so that every sign and coefficient is exercised with values the
physics would not produce."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
import cases  # noqa: E402
from test_gpu_fd import env  # noqa: E402,F401

pytestmark = pytest.mark.gpu

NAMES = ["hwea10_k1", "bv6_k1", "grid3x4_k3", "qaoa8_k4", "aqft8_k4", "grid4x4_s4", "grid4x5_k5", "hwea14_skinny",
         "nocut6"]   # k_in 0..4 (4: the single-kernel form), k_out 0..4


def subcircuits():
    for name in NAMES:
        cc = cases.SMALL[name]()
        for i, s in enumerate(cc.subs):
            yield f"{name}/{i}", s


@pytest.mark.parametrize("label,sub", list(subcircuits()), ids=lambda v: v if isinstance(v, str) else "")
def test_attribute_simulated_variants(env, label, sub):
    torch, cutqc = env
    from oracle import attribution as at
    p = at.variant_probabilities(sub)
    want = at.attribute(sub, p).reshape(-1)
    got64 = cutqc.cutqc_attribute(sub, torch.tensor(p.reshape(-1), dtype=torch.float64, device="cuda"))
    assert np.abs(got64.cpu().numpy() - want).max() <= 1e-12
    p32 = p.astype(np.float32)
    want32 = at.attribute(sub, p32.astype(np.float64)).reshape(-1)
    got32 = cutqc.cutqc_attribute(sub, torch.tensor(p32.reshape(-1), device="cuda"))
    assert np.abs(got32.double().cpu().numpy() - want32).max() <= 1e-6


@pytest.mark.parametrize("name", ["qaoa8_k4", "grid4x5_k5", "aqft8_k4"])
def test_attribute_random_distributions(env, name):
    torch, cutqc = env
    from oracle import attribution as at
    rng = np.random.default_rng(7)
    for sub in cases.SMALL[name]().subs:
        shape = (4 ** sub.k_in, 3 ** sub.k_out, 2 ** sub.d)
        p = rng.random(shape)
        p /= p.sum(axis=2, keepdims=True)
        want = at.attribute(sub, p).reshape(-1)
        got = cutqc.cutqc_attribute(sub, torch.tensor(p.reshape(-1), device="cuda"))
        assert np.abs(got.cpu().numpy() - want).max() <= 1e-12


def test_attribute_matches_the_simulator_path(env):
    """Attributing the oracle's variant distributions on the GPU gives the
    tensors the GPU simulator produces (its own attribution) for the
    benchmark circuit's two subcircuits."""
    torch, cutqc = env
    from oracle import attribution as at
    cc = cases.supremacy_4x6()
    for sub in cc.subs:
        p = torch.tensor(at.variant_probabilities(sub).reshape(-1), device="cuda")
        got = cutqc.cutqc_attribute(sub, p)
        sim = cutqc.cutqc_simulate_subcircuit(sub, torch.float64)
        assert torch.abs(got - sim).max().item() <= 1e-12


def synthetic_sub(d, k_in, k_out, seed):
    """A subcircuit layout without gates (the attribution only needs the slot
    and output qubits): random distinct local qubits for the measured slots."""
    from types import SimpleNamespace
    rng = np.random.default_rng(seed)
    perm = [int(q) for q in rng.permutation(d)]
    meas = perm[:k_out]
    outs = sorted(perm[k_out:])
    return SimpleNamespace(d=d, k_in=k_in, k_out=k_out, n_eff=d - k_out,
                           in_slots=[(q, i) for i, q in enumerate(perm[:k_in])],
                           out_slots=[(q, i) for i, q in enumerate(meas)],
                           outputs=[(q, q) for q in outs])


@pytest.mark.parametrize("d,k_in,k_out", [(8, 1, 5), (9, 0, 6), (7, 4, 1), (6, 5, 0), (5, 2, 4), (3, 0, 2),
                                         (7, 2, 2), (6, 1, 1), (5, 2, 0), (4, 0, 1), (9, 2, 1), (3, 1, 2)])
def test_attribute_all_kernel_forms(env, d, k_in, k_out):
    """Slot counts that select each form: k_out > 4 (outcome gather), k_in > 3
    (single kernel), n_eff < 2, the variant-centred form for one to four
    measurement slots and zero to three init slots; random layouts of the
    measured qubits among the local qubits."""
    torch, cutqc = env
    from oracle import attribution as at
    rng = np.random.default_rng(d * 100 + k_in * 10 + k_out)
    sub = synthetic_sub(d, k_in, k_out, seed=d + k_in + k_out)
    p = rng.random((4 ** k_in, 3 ** k_out, 2 ** d))
    p /= p.sum(axis=2, keepdims=True)
    want = at.attribute(sub, p).reshape(-1)
    got = cutqc.cutqc_attribute(sub, torch.tensor(p.reshape(-1), device="cuda"))
    assert np.abs(got.cpu().numpy() - want).max() <= 1e-12
    got32 = cutqc.cutqc_attribute(sub, torch.tensor(p.reshape(-1), dtype=torch.float32, device="cuda"))
    want32 = at.attribute(sub, p.astype(np.float32).astype(np.float64)).reshape(-1)
    assert np.abs(got32.double().cpu().numpy() - want32).max() <= 1e-6


def test_attribute_into_unaligned_output(env):
    """An output that is not 16-byte aligned takes the scalar-store form."""
    torch, cutqc = env
    from oracle import attribution as at
    sub = cases.SMALL["qaoa8_k4"]().subs[0]
    p = at.variant_probabilities(sub)
    n = (4 ** sub.k_in) * (4 ** sub.k_out) * (2 ** sub.n_eff)
    buf = torch.zeros(n + 1, dtype=torch.float32, device="cuda")
    out = buf[1:]
    cutqc.cutqc_attribute(sub, torch.tensor(p.reshape(-1), dtype=torch.float32, device="cuda"), out=out)
    want = at.attribute(sub, p.astype(np.float32).astype(np.float64)).reshape(-1)
    assert np.abs(out.double().cpu().numpy() - want).max() <= 1e-6
    assert buf[0].item() == 0.0


def test_attribute_benchmark_size(env):
    """The benchmark's attribution workload itself: both QAOA-30 subcircuits
    (17 qubits, 2 init + 2 measurement slots) from seeded synthetic variant
    distributions, every entry against the oracle."""
    torch, cutqc = env
    from oracle import attribution as at
    from paper_2012_02333_gb300 import circuits as C
    cc = C.qaoa_2cluster(15, 0)
    rng = np.random.default_rng(21)
    for sub in cc.subs:
        p = rng.random(((4 ** sub.k_in) * (3 ** sub.k_out), 2 ** sub.d)).astype(np.float32)
        p /= p.sum(axis=1, keepdims=True)
        got = cutqc.cutqc_attribute(sub, torch.tensor(p.reshape(-1), device="cuda"))
        want = at.attribute(sub, p.astype(np.float64).reshape(4 ** sub.k_in, 3 ** sub.k_out, 2 ** sub.d))
        assert np.abs(got.double().cpu().numpy() - want.reshape(-1)).max() <= 1e-6


# ---- merged tensors of a dynamic-definition recursion from the variants ----

def _synthetic_sub(d, k_in, k_out):
    """A subcircuit whose measured cut qubits are its first local qubits and
    whose outputs are the rest, global qubit = local qubit: the roles below
    then put the merged outputs exactly where each merge form needs them."""
    from paper_2012_02333_gb300 import circuits as C
    return C.Subcircuit(d=d, gates=[], in_slots=[(j, j) for j in range(k_in)],
                        out_slots=[(j, j) for j in range(k_out)], outputs=[(lq, lq) for lq in range(k_out, d)])


# roles of outputs 2..11 of a 12-qubit subcircuit with 2 measured cut qubits
MERGE_FORMS = {
    "run_dense": [0] * 6 + [1] * 4,            # merged = the lowest 4 index bits, kept bits right above
    "run_zoomed": [0, 0, 3, 0, 2, 0, 1, 1, 1, 1],
    # block form: every index bit below the highest merged one merged or kept, at most two kept
    "block_low2": [0, 0, 0, 0, 1, 1, 1, 1, 0, 0],      # merged 2-5, kept 0-1
    "block_zoom": [0, 3, 0, 0, 0, 1, 1, 1, 0, 1],      # merged 0, 2-4, kept 1, bit 8 zoomed
    "block_split": [0, 0, 0, 1, 0, 1, 1, 1, 0, 1],     # merged 0, 2-4, 6, kept 1 and 5
    "warp": [0, 1, 1, 1, 0, 1, 1, 1, 0, 0],    # 6 merged values, not on the lowest bits
    "thread": [0, 1, 0, 0, 2, 0, 1, 0, 0, 0],  # 2 merged values
    "zoom_only": [0, 3, 0, 2, 0, 0, 3, 0, 0, 0],
    "all_active": [0] * 10,
}


@pytest.mark.parametrize("form", list(MERGE_FORMS))
def test_attribute_merged_forms(env, form):
    """Every merge form (contiguous runs, blocks with one or two kept bits
    among the merged ones, warp and thread per output, zoom only, nothing
    merged) against
    the oracle's attribute-then-merge, FP64 and FP32, on seeded random variant
    distributions."""
    torch, cutqc = env
    from oracle import attribution as at
    sub = _synthetic_sub(12, 2, 2)
    roles = [0, 0] + MERGE_FORMS[form]
    rng = np.random.default_rng(31)
    V = (4 ** sub.k_in) * (3 ** sub.k_out)
    p = rng.random((V, 2 ** sub.d))
    p /= p.sum(axis=1, keepdims=True)
    want = at.attribute_merged(sub, p, roles).reshape(-1)
    got = cutqc.cutqc_attribute_merged(sub, torch.tensor(p.reshape(-1), device="cuda"), roles)
    assert got.numel() == want.size
    assert np.abs(got.cpu().numpy() - want).max() <= 1e-12
    p32 = p.astype(np.float32)
    want32 = at.attribute_merged(sub, p32.astype(np.float64), roles).reshape(-1)
    got32 = cutqc.cutqc_attribute_merged(sub, torch.tensor(p32.reshape(-1), device="cuda"), roles)
    assert np.abs(got32.double().cpu().numpy() - want32).max() <= 1e-6


@pytest.mark.parametrize("name", ["qaoa8_k4", "grid4x5_k5", "hwea10_k1", "aqft8_k4"])
def test_attribute_merged_simulated_variants(env, name):
    """Physical variant distributions of the test circuits, roles cycling
    through active / merged / zoomed over the global qubits."""
    torch, cutqc = env
    from oracle import attribution as at
    cc = cases.SMALL[name]()
    for pattern in [(0, 1, 2, 3), (1, 0, 1, 3, 0), (1, 1, 0)]:
        roles = [pattern[q % len(pattern)] for q in range(cc.n)]
        for sub in cc.subs:
            if sub.k_out == 0 and not any(roles[g] == 0 for _, g in sub.outputs):
                continue   # nothing left to attribute (rejected, see the host tests)
            p = at.variant_probabilities(sub)
            want = at.attribute_merged(sub, p, roles).reshape(-1)
            got = cutqc.cutqc_attribute_merged(sub, torch.tensor(p.reshape(-1), dtype=torch.float64,
                                                                 device="cuda"), roles)
            assert np.abs(got.cpu().numpy() - want).max() <= 1e-12, (pattern, sub.d)


def test_attribute_merged_benchmark_size(env):
    """Both QAOA-30 subcircuits (17 qubits, 2 + 2 slots) with the roles of a
    first recursion of 20 active qubits, FP32 synthetic variant distributions,
    every entry against the oracle."""
    torch, cutqc = env
    from oracle import attribution as at
    from paper_2012_02333_gb300 import circuits as C
    cc = C.qaoa_2cluster(15, 0)
    roles = [0 if q < 20 else 1 for q in range(cc.n)]
    rng = np.random.default_rng(23)
    for sub in cc.subs:
        p = rng.random(((4 ** sub.k_in) * (3 ** sub.k_out), 2 ** sub.d)).astype(np.float32)
        p /= p.sum(axis=1, keepdims=True)
        got = cutqc.cutqc_attribute_merged(sub, torch.tensor(p.reshape(-1), device="cuda"), roles)
        want = at.attribute_merged(sub, p.astype(np.float64), roles)
        assert np.abs(got.double().cpu().numpy() - want.reshape(-1)).max() <= 1e-6
