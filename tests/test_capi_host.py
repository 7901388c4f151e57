"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, it exports every function include/cutqc.h declares, and argument /
shape errors come back as statuses before anything is launched."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2012_02333_gb300", "libcutqc.so")


@pytest.fixture(scope="module")
def capi():
    if not os.path.exists(LIB):
        from paper_2012_02333_gb300 import build
        build.build()
    from paper_2012_02333_gb300 import cutqc
    return cutqc


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cutqc.h")).read()
    return sorted(set(re.findall(r"CUTQC_API\s+[\w\s\*]+?\b(cutqc_\w+)\s*\(", src)))


def test_header_declares_the_entry_points():
    fns = declared_functions()
    for want in ("cutqc_reconstruct_fd", "cutqc_reconstruct_dd", "cutqc_reconstruct_backward",
                 "cutqc_last_error", "cutqc_release", "cutqc_simulate_subcircuit"):
        assert want in fns


def test_library_exports_every_declared_symbol(capi):
    lib = C.CDLL(LIB)
    for fn in declared_functions():
        assert hasattr(lib, fn), fn


def _problem(capi, subs_spec, n_qubits, n_cuts, dtype=1):
    keep = []
    arr = (capi.cutqc_subcircuit * len(subs_spec))()
    for i, (kin, kout, neff, ic, oc, oq) in enumerate(subs_spec):
        a, b, c = capi._i32(ic), capi._i32(oc), capi._i32(oq)
        keep += [a, b, c]
        # a non-null placeholder that is never dereferenced: every call below
        # fails validation on the host before any device work
        arr[i] = capi.cutqc_subcircuit(kin, kout, neff, a, b, c, C.c_void_p(0x1000))
    p = capi.cutqc_problem(n_qubits, n_cuts, len(subs_spec), dtype, arr)
    return p, keep, arr


def _fd(capi, p):
    out = (C.c_void_p * 1)(C.c_void_p(0x2000))
    return capi._lib.cutqc_reconstruct_fd(C.byref(p), 1, out, 0, None, None)


GOOD = [(0, 1, 5, [], [0], [0, 1, 2, 3, 4]), (1, 0, 5, [0], [], [5, 6, 7, 8, 9])]


@pytest.mark.parametrize("mutate,status", [
    (lambda s: s.__setitem__(1, (1, 0, 5, [1], [], [5, 6, 7, 8, 9])), "CUTQC_ERR_SHAPE"),    # cut id out of range
    (lambda s: s.__setitem__(1, (1, 0, 5, [0], [], [4, 6, 7, 8, 9])), "CUTQC_ERR_SHAPE"),    # qubit twice
    (lambda s: s.__setitem__(1, (1, 0, 4, [0], [], [5, 6, 7, 8])), "CUTQC_ERR_SHAPE"),       # qubit missing
    (lambda s: s.__setitem__(0, (0, 0, 5, [], [], [0, 1, 2, 3, 4])), "CUTQC_ERR_SHAPE"),     # cut without upstream
])
def test_shape_errors(capi, mutate, status):
    spec = list(GOOD)
    mutate(spec)
    p, keep, arr = _problem(capi, spec, 10, 1)
    st = _fd(capi, p)
    assert st == getattr(capi, status), capi.last_error()
    assert capi.last_error()


def test_limits_and_arguments(capi):
    p, keep, arr = _problem(capi, GOOD, 10, 13)
    assert _fd(capi, p) == capi.CUTQC_ERR_UNSUPPORTED          # K > 12
    p, keep, arr = _problem(capi, GOOD, 10, 1, dtype=7)
    assert _fd(capi, p) == capi.CUTQC_ERR_ARG                  # bad dtype
    assert capi._lib.cutqc_reconstruct_fd(None, 1, None, 0, None, None) == capi.CUTQC_ERR_ARG
    big = [(0, 1, 20, [], [0], list(range(20))), (1, 0, 20, [0], [], list(range(20, 40)))]
    p, keep, arr = _problem(capi, big, 40, 1)
    assert _fd(capi, p) == capi.CUTQC_ERR_UNSUPPORTED          # FD beyond 2^34
    p, keep, arr = _problem(capi, GOOD, 10, 1)
    out = (C.c_void_p * 1)(C.c_void_p(0x2000))
    assert capi._lib.cutqc_reconstruct_fd(C.byref(p), 1, out, 9, None, None) == capi.CUTQC_ERR_ARG  # algo


def test_simulator_argument_errors(capi):
    g = (capi.cutqc_gate * 1)(capi.cutqc_gate(13, 0, 0, 0.0))   # CZ on one qubit twice
    t = C.c_void_p(0x3000)
    st = capi._lib.cutqc_simulate_subcircuit(g, 1, 2, None, 0, None, 0, capi._i32([0, 1]), 2, 1, t, None)
    assert st == capi.CUTQC_ERR_SHAPE
    st = capi._lib.cutqc_simulate_subcircuit(g, 1, 40, None, 0, None, 0, capi._i32([0]), 1, 1, t, None)
    assert st == capi.CUTQC_ERR_UNSUPPORTED


def test_attribution_argument_errors(capi):
    p, t = C.c_void_p(0x2000), C.c_void_p(0x3000)
    i32 = capi._i32
    # 3 local qubits: one measured cut qubit and two outputs
    ok_args = (p, 3, 1, i32([2]), 1, i32([0, 1]), 2, capi.CUTQC_F32, t, None)
    bad = [
        ((p, 3, 1, i32([2]), 1, i32([0, 1]), 1, capi.CUTQC_F32, t, None), capi.CUTQC_ERR_SHAPE),   # a qubit unassigned
        ((p, 3, 1, i32([1]), 1, i32([0, 1]), 2, capi.CUTQC_F32, t, None), capi.CUTQC_ERR_SHAPE),   # qubit used twice
        ((p, 3, 1, i32([3]), 1, i32([0, 1]), 2, capi.CUTQC_F32, t, None), capi.CUTQC_ERR_SHAPE),   # out of range
        ((p, 3, 7, i32([2]), 6, i32([0, 1]), 2, capi.CUTQC_F32, t, None), capi.CUTQC_ERR_SHAPE),   # K > 12 slots
        ((None, 3, 1, i32([2]), 1, i32([0, 1]), 2, capi.CUTQC_F32, t, None), capi.CUTQC_ERR_ARG),
        ((p, 3, 1, i32([2]), 1, i32([0, 1]), 2, 7, t, None), capi.CUTQC_ERR_ARG),                   # dtype
        ((p, 31, 0, None, 0, i32(list(range(31))), 31, capi.CUTQC_F32, t, None), capi.CUTQC_ERR_UNSUPPORTED),
    ]
    for args, status in bad:
        assert capi._lib.cutqc_attribute(*args) == status, args
    assert ok_args[1] == 3


def test_distance_and_sampling_argument_errors(capi):
    a, b = C.c_void_p(0x2000), C.c_void_p(0x3000)
    f = capi._lib
    assert f.cutqc_distance(a, None, 8, capi.CUTQC_F32, a, b, None) == capi.CUTQC_ERR_ARG
    assert f.cutqc_distance(a, b, 0, capi.CUTQC_F32, a, b, None) == capi.CUTQC_ERR_UNSUPPORTED
    assert f.cutqc_distance(a, b, 8, 5, a, b, None) == capi.CUTQC_ERR_ARG
    assert f.cutqc_sample(None, 8, capi.CUTQC_F32, a, 4, b, None) == capi.CUTQC_ERR_ARG
    assert f.cutqc_sample(a, 8, capi.CUTQC_F32, None, 4, b, None) == capi.CUTQC_ERR_ARG
    assert f.cutqc_sample(a, 8, capi.CUTQC_F32, a, -1, b, None) == capi.CUTQC_ERR_ARG
    assert f.cutqc_sample(a, 1 << 41, capi.CUTQC_F32, a, 4, b, None) == capi.CUTQC_ERR_UNSUPPORTED


def test_misaligned_pointers_are_rejected(capi):
    """Device arrays are accessed with 16-byte vector loads and stores, so a
    pointer off that grid is an argument error on the host, never a fault."""
    f, i32, ARG = capi._lib, capi._i32, capi.CUTQC_ERR_ARG
    # a subcircuit tensor 4 bytes off
    spec = list(GOOD)
    p, keep, arr = _problem(capi, spec, 10, 1)
    arr[1].tensor = C.c_void_p(0x1004)
    assert _fd(capi, p) == ARG and "16-byte" in capi.last_error()
    # the full-definition output and its FP64 sum
    p, keep, arr = _problem(capi, GOOD, 10, 1)
    out = (C.c_void_p * 1)(C.c_void_p(0x2008))
    assert f.cutqc_reconstruct_fd(C.byref(p), 1, out, 0, None, None) == ARG
    out = (C.c_void_p * 1)(C.c_void_p(0x2000))
    assert f.cutqc_reconstruct_fd(C.byref(p), 1, out, 0, C.c_void_p(0x3004), None) == ARG
    assert "sum_p" in capi.last_error()
    assert f.cutqc_reconstruct_fd_noalloc(C.byref(p), C.c_void_p(0x2004), None, None) == ARG
    # dynamic-definition bins
    role = (C.c_int8 * 10)(*([0] * 10))
    assert f.cutqc_reconstruct_dd(C.byref(p), role, C.c_void_p(0x2004), 0, None, None, 0, None) == ARG
    assert "bins" in capi.last_error()
    # adjoint gradients
    grads = (C.c_void_p * 2)(C.c_void_p(0x4000), C.c_void_p(0x5002))
    assert f.cutqc_reconstruct_backward(C.byref(p), C.c_void_p(0x6000), None, grads, None, None) == ARG
    # attribution and simulation
    # (element alignment: these kernels choose vector or scalar accesses)
    args = [C.c_void_p(0x2002), 3, 1, i32([2]), 1, i32([0, 1]), 2, capi.CUTQC_F32, C.c_void_p(0x3000), None]
    assert f.cutqc_attribute(*args) == ARG
    args[0], args[8] = C.c_void_p(0x2000), C.c_void_p(0x3004)
    args[7] = capi.CUTQC_F64
    assert f.cutqc_attribute(*args) == ARG
    g = (capi.cutqc_gate * 1)(capi.cutqc_gate(0, 0, 0, 0.0))
    st = f.cutqc_simulate_subcircuit(g, 1, 2, None, 0, None, 0, i32([0, 1]), 2, 1, C.c_void_p(0x3002), None)
    assert st == ARG
    # distance and sampling take element-aligned arrays, scalars need 8 bytes
    a, b = C.c_void_p(0x2000), C.c_void_p(0x3000)
    assert f.cutqc_distance(C.c_void_p(0x2002), b, 8, capi.CUTQC_F32, a, b, None) == ARG
    assert f.cutqc_distance(a, C.c_void_p(0x3004), 8, capi.CUTQC_F64, a, b, None) == ARG
    assert f.cutqc_distance(a, b, 8, capi.CUTQC_F32, C.c_void_p(0x2004), b, None) == ARG
    assert f.cutqc_sample(a, 8, capi.CUTQC_F32, C.c_void_p(0x2004), 4, b, None) == ARG
    assert f.cutqc_sample(a, 8, capi.CUTQC_F32, a, 4, C.c_void_p(0x3002), None) == ARG


def test_attribute_merged_argument_errors(capi):
    p, t = C.c_void_p(0x2000), C.c_void_p(0x3000)
    i32, f = capi._i32, capi._lib
    roles = lambda r: (C.c_int8 * len(r))(*r)
    # 3 local qubits: one measured cut qubit (2) and two outputs (0, 1)
    base = [p, 3, 1, i32([2]), 1, i32([0, 1]), 2, roles([0, 1]), capi.CUTQC_F32, t, None]
    for idx, val, status in [
        (7, roles([0, 4]), capi.CUTQC_ERR_ARG),             # role out of range
        (7, None, capi.CUTQC_ERR_ARG),                      # no roles for the outputs
        (5, i32([0, 2]), capi.CUTQC_ERR_SHAPE),             # an output on the measured qubit
        (1, 31, capi.CUTQC_ERR_UNSUPPORTED),                # d > 30
    ]:
        args = list(base)
        args[idx] = val
        assert f.cutqc_attribute_merged(*args) == status, (idx, capi.last_error())
    # nothing left to attribute: no measured cut qubit, every output merged or zoomed
    st = f.cutqc_attribute_merged(p, 2, 1, None, 0, i32([0, 1]), 2, roles([1, 3]), capi.CUTQC_F32, t, None)
    assert st == capi.CUTQC_ERR_UNSUPPORTED and "left to attribute" in capi.last_error()
