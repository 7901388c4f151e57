"""Python binding of the C ABI in include/cutqc.h (ctypes, argument
marshalling only: every step of the reconstruction runs in the library's CUDA
kernels).  PyTorch provides device memory and streams.

Loading fails loudly when libcutqc.so is missing: there is no CPU fallback.
Build it with ``python -c "import __graft_entry__ as g; g.build()"``.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence, Tuple

import torch

from . import circuits

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcutqc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first (paper_2012_02333_gb300.build)")
_lib = C.CDLL(LIB_PATH)

# ---------------------------------------------------------------- constants
CUTQC_OK = 0
CUTQC_ERR_ARG = -1
CUTQC_ERR_SHAPE = -2
CUTQC_ERR_OOM = -3
CUTQC_ERR_CUDA = -4
CUTQC_ERR_UNSUPPORTED = -5
CUTQC_ERR_TIMEOUT = -6
CUTQC_ERR_DEVICE = -7
CUTQC_F64 = 0
CUTQC_F32 = 1
CUTQC_AUTO = 0
CUTQC_CC = 1
CUTQC_TC_BF16X3 = 2
CUTQC_TC_BF16X6 = 3
CUTQC_TC_TF32X3 = 4
ALGOS = {"auto": CUTQC_AUTO, "cc": CUTQC_CC, "tc_bf16x3": CUTQC_TC_BF16X3, "tc_bf16x6": CUTQC_TC_BF16X6,
         "tc_tf32x3": CUTQC_TC_TF32X3}
CUTQC_LOSS_NONE = 0
CUTQC_LOSS_MAXCUT = 1

GATE_OPS = {name: i for i, name in enumerate(
    ["h", "x", "y", "z", "s", "sdg", "t", "sx", "sy", "sw", "rx", "ry", "rz", "cz", "cx", "cp"])}


class cutqc_subcircuit(C.Structure):
    _fields_ = [("k_in", C.c_int32), ("k_out", C.c_int32), ("n_eff", C.c_int32),
                ("in_cut", C.POINTER(C.c_int32)), ("out_cut", C.POINTER(C.c_int32)),
                ("out_qubit", C.POINTER(C.c_int32)), ("tensor", C.c_void_p)]


class cutqc_problem(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("n_cuts", C.c_int32), ("n_sub", C.c_int32),
                ("dtype", C.c_int32), ("sub", C.POINTER(cutqc_subcircuit))]


class cutqc_loss(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_edges", C.c_int32), ("edges", C.POINTER(C.c_int32))]


class cutqc_gate(C.Structure):
    _fields_ = [("op", C.c_int32), ("q0", C.c_int32), ("q1", C.c_int32), ("param", C.c_double)]


_lib.cutqc_reconstruct_fd.argtypes = [C.POINTER(cutqc_problem), C.c_int32, C.POINTER(C.c_void_p), C.c_int32,
                                      C.c_void_p, C.c_void_p]
_lib.cutqc_reconstruct_dd.argtypes = [C.POINTER(cutqc_problem), C.POINTER(C.c_int8), C.c_void_p, C.c_int32,
                                      C.POINTER(C.c_int64), C.POINTER(C.c_double), C.c_int32, C.c_void_p]
_lib.cutqc_reconstruct_backward.argtypes = [C.POINTER(cutqc_problem), C.c_void_p, C.POINTER(cutqc_loss),
                                            C.POINTER(C.c_void_p), C.c_void_p, C.c_void_p]
_lib.cutqc_simulate_subcircuit.argtypes = [C.POINTER(cutqc_gate), C.c_int32, C.c_int32, C.POINTER(C.c_int32),
                                           C.c_int32, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_int32),
                                           C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]
_lib.cutqc_reconstruct_fd_noalloc.argtypes = [C.POINTER(cutqc_problem), C.c_void_p, C.c_void_p, C.c_void_p]
_lib.cutqc_reconstruct_fd_slab.argtypes = [C.POINTER(cutqc_problem), C.c_int32, C.c_int64, C.c_void_p, C.c_int32,
                                           C.c_void_p, C.c_void_p]
_lib.cutqc_profile.argtypes = [C.c_int32]
_lib.cutqc_last_split.argtypes = [C.POINTER(C.c_int32), C.POINTER(C.c_double)]
_lib.cutqc_profile_read.argtypes = [C.POINTER(C.c_int64), C.POINTER(C.c_double)]
_lib.cutqc_device_status.argtypes = [C.c_void_p]
_lib.cutqc_cut_search.argtypes = [C.POINTER(cutqc_gate), C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int64,
                                  C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                  C.POINTER(C.c_double)]
_lib.cutqc_distance.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
_lib.cutqc_sample.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
_lib.cutqc_attribute.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_int32), C.c_int32,
                                 C.POINTER(C.c_int32), C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]
_lib.cutqc_attribute_merged.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_int32), C.c_int32,
                                        C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_int8), C.c_int32,
                                        C.c_void_p, C.c_void_p]
_lib.cutqc_selftest_wait.argtypes = [C.c_int32, C.c_void_p]
_lib.cutqc_last_error.restype = C.c_char_p
_lib.cutqc_launch_count.restype = C.c_int64
_lib.cutqc_last_algo.restype = C.c_int32
for _f in ("cutqc_reconstruct_fd", "cutqc_reconstruct_fd_slab", "cutqc_reconstruct_dd", "cutqc_reconstruct_backward",
           "cutqc_simulate_subcircuit", "cutqc_profile", "cutqc_profile_read", "cutqc_last_split",
           "cutqc_reconstruct_fd_noalloc", "cutqc_device_status", "cutqc_selftest_wait", "cutqc_attribute",
           "cutqc_attribute_merged", "cutqc_distance", "cutqc_sample", "cutqc_cut_search"):
    getattr(_lib, _f).restype = C.c_int


class CutQCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cutqc status {status}: {msg}")
        self.status = status


def _check(status: int) -> None:
    if status != CUTQC_OK:
        raise CutQCError(status, _lib.cutqc_last_error().decode())


def last_error() -> str:
    return _lib.cutqc_last_error().decode()


def launch_count() -> int:
    return int(_lib.cutqc_launch_count())


def last_algo() -> int:
    """cutqc_algo of the last full-definition call's final contraction."""
    return int(_lib.cutqc_last_algo())


def last_split():
    """(split products 3 or 6, a-priori magnitude S) of the last tensor-core
    contraction on this thread (synchronises its stream)."""
    n = C.c_int32()
    b = C.c_double()
    _check(_lib.cutqc_last_split(C.byref(n), C.byref(b)))
    return int(n.value), float(b.value)


def release() -> None:
    _lib.cutqc_release()


def profile(enable: bool) -> None:
    """Bracket every main-contraction launch with CUDA events (cutqc_profile)."""
    _check(_lib.cutqc_profile(1 if enable else 0))


def profile_read():
    """(launches, total milliseconds) of the bracketed main-kernel launches."""
    n = C.c_int64()
    ms = C.c_double()
    _check(_lib.cutqc_profile_read(C.byref(n), C.byref(ms)))
    return int(n.value), float(ms.value)


def _i32(xs: Sequence[int]):
    arr = (C.c_int32 * max(len(xs), 1))(*[int(x) for x in xs])
    return arr


def _dist_dtype(t: torch.Tensor) -> int:
    if not t.is_cuda or not t.is_contiguous() or t.dtype not in (torch.float32, torch.float64):
        raise ValueError("expected a contiguous CUDA float32 / float64 tensor")
    return CUTQC_F64 if t.dtype == torch.float64 else CUTQC_F32


def cutqc_distance(a: torch.Tensor, b: torch.Tensor, stream=None):
    """Binding of cutqc_distance: (chi^2 of Eq. 16, total variation) of two
    distributions as CUDA float64 scalars (no host synchronisation)."""
    dt = _dist_dtype(a)
    if _dist_dtype(b) != dt or a.numel() != b.numel():
        raise ValueError("a and b must have the same dtype and size")
    out = torch.empty(2, dtype=torch.float64, device=a.device)
    _check(_lib.cutqc_distance(C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), a.numel(), dt,
                               C.c_void_p(out.data_ptr()), C.c_void_p(out.data_ptr() + 8), _stream_ptr(stream)))
    return out[0], out[1]


def cutqc_sample(p: torch.Tensor, u: torch.Tensor, stream=None) -> torch.Tensor:
    """Binding of cutqc_sample: one outcome index (int64) per uniform in u
    (CUDA float64, values in [0, 1))."""
    dt = _dist_dtype(p)
    if not u.is_cuda or u.dtype != torch.float64 or not u.is_contiguous():
        raise ValueError("u must be a contiguous CUDA float64 tensor")
    out = torch.empty(u.numel(), dtype=torch.int64, device=p.device)
    _check(_lib.cutqc_sample(C.c_void_p(p.data_ptr()), p.numel(), dt, C.c_void_p(u.data_ptr()), u.numel(),
                             C.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def cut_search(circ: circuits.Circuit, max_width: int, max_subcircuits: int, max_nodes: int = 10 ** 8) -> dict:
    """Binding of cutqc_cut_search: the least-cost cut (Eqs. 4-15) of `circ`
    for devices of max_width qubits and at most max_subcircuits subcircuits.
    Returns {"gate_cluster": {gate index: subcircuit}, "assign": [...] per
    multi-qubit gate in order, "K": cuts, "cost": Eq. 14}."""
    gates = (cutqc_gate * max(len(circ.gates), 1))()
    for i, g in enumerate(circ.gates):
        q1 = g.qubits[1] if len(g.qubits) > 1 else -1
        gates[i] = cutqc_gate(GATE_OPS[g.name], g.qubits[0], q1, g.params[0] if g.params else 0.0)
    cl = (C.c_int32 * max(len(circ.gates), 1))()
    nv, k = C.c_int32(), C.c_int32()
    cost = C.c_double()
    _check(_lib.cutqc_cut_search(gates, len(circ.gates), circ.n, max_width, max_subcircuits, max_nodes, cl,
                                 C.byref(nv), C.byref(k), C.byref(cost)))
    assign = [int(cl[v]) for v in range(nv.value)]
    verts = [gi for gi, g in enumerate(circ.gates) if len(g.qubits) > 1]
    return {"gate_cluster": dict(zip(verts, assign)), "assign": assign, "K": int(k.value), "cost": cost.value}


def device_status(stream=None) -> None:
    """Synchronise `stream` and raise CutQCError if a kernel since the last
    check recorded a timed-out bounded wait (CUTQC_ERR_TIMEOUT) or a failed
    device-side check (CUTQC_ERR_DEVICE); the record is cleared either way."""
    _check(_lib.cutqc_device_status(_stream_ptr(stream)))


def selftest_wait(limit_us: int, stream=None) -> None:
    """Launch the bounded-wait self-test (a wait nothing satisfies, limited to
    `limit_us` microseconds); device_status() then reports the timeout."""
    _check(_lib.cutqc_selftest_wait(int(limit_us), _stream_ptr(stream)))


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


# ------------------------------------------------------------------ problems

class Problem:
    """Marshals one cut circuit (structure from ``circuits.CutCircuit`` or
    anything with the same fields) and its device tensors into a
    ``cutqc_problem``.  Keeps every ctypes array alive while it lives."""

    def __init__(self, n_qubits: int, n_cuts: int, subs, tensors: Sequence[torch.Tensor]):
        if len(subs) != len(tensors):
            raise ValueError("one tensor per subcircuit")
        dts = {t.dtype for t in tensors}
        if len(dts) != 1 or dts.pop() not in (torch.float32, torch.float64):
            raise ValueError("tensors must all be float32 or all float64")
        self.dtype = tensors[0].dtype
        self.tensors = list(tensors)
        self._keep = []
        arr = (cutqc_subcircuit * len(subs))()
        for i, (s, t) in enumerate(zip(subs, tensors)):
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("tensors must be contiguous CUDA tensors")
            want = (4 ** s.k_in) * (4 ** s.k_out) * (2 ** s.n_eff)
            if t.numel() != want:
                raise ValueError(f"tensor {i} has {t.numel()} entries, expected {want}")
            ic, oc, oq = _i32(s.in_cut), _i32(s.out_cut), _i32(s.out_qubit)
            self._keep += [ic, oc, oq]
            arr[i] = cutqc_subcircuit(s.k_in, s.k_out, s.n_eff, ic, oc, oq, C.c_void_p(t.data_ptr()))
        self._subs = arr
        self.n_qubits, self.n_cuts = n_qubits, n_cuts
        self.c = cutqc_problem(n_qubits, n_cuts, len(subs),
                               CUTQC_F64 if self.dtype == torch.float64 else CUTQC_F32, arr)

    @classmethod
    def from_cut(cls, cc: circuits.CutCircuit, tensors: Sequence[torch.Tensor]) -> "Problem":
        return cls(cc.n, cc.n_cuts, cc.subs, tensors)


# ------------------------------------------------------------------ entry points

def cutqc_reconstruct_fd(problems: Sequence[Problem], outs: Sequence[torch.Tensor], algo: str = "auto",
                         sum_p: Optional[torch.Tensor] = None, stream=None) -> None:
    """Binding of cutqc_reconstruct_fd (full definition, Sec. 4.2)."""
    n = len(problems)
    parr = (cutqc_problem * n)(*[p.c for p in problems])
    optr = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    for p, o in zip(problems, outs):
        if o.dtype != p.dtype or o.numel() != 2 ** p.n_qubits or not (o.is_cuda or o.is_pinned()):
            raise ValueError("out must be a CUDA or pinned CPU tensor of 2^n entries in the tensors' dtype")
    sp = None
    if sum_p is not None:
        if sum_p.dtype != torch.float64 or sum_p.numel() < n or not sum_p.is_cuda:
            raise ValueError("sum_p must be a CUDA float64 tensor of n_problems entries")
        sp = sum_p.data_ptr()
    _check(_lib.cutqc_reconstruct_fd(parr, n, optr, ALGOS[algo], sp, _stream_ptr(stream)))


def cutqc_reconstruct_fd_slab(problem: Problem, slab_bits: int, slab_index: int, out: torch.Tensor,
                              algo: str = "auto", sum_p: Optional[torch.Tensor] = None, stream=None) -> None:
    """Binding of cutqc_reconstruct_fd_slab: the 2^(n - slab_bits) outputs whose
    slab_bits most significant bits read slab_index, and their FP64 sum."""
    if out.dtype != problem.dtype or out.numel() != 2 ** (problem.n_qubits - slab_bits) or \
            not out.is_contiguous() or not (out.is_cuda or out.is_pinned()):
        raise ValueError("out must be a contiguous CUDA or pinned tensor of 2^(n - slab_bits) entries")
    sp = None
    if sum_p is not None:
        if sum_p.dtype != torch.float64 or not sum_p.is_cuda:
            raise ValueError("sum_p must be a CUDA float64 tensor")
        sp = sum_p.data_ptr()
    _check(_lib.cutqc_reconstruct_fd_slab(C.byref(problem.c), int(slab_bits), int(slab_index),
                                          C.c_void_p(out.data_ptr()), ALGOS[algo], sp, _stream_ptr(stream)))


def reconstruct_fd(cc: circuits.CutCircuit, tensors: Sequence[torch.Tensor], algo: str = "auto",
                   out: Optional[torch.Tensor] = None, with_sum: bool = True, stream=None,
                   device: Optional[torch.device] = None):
    """Full-definition reconstruction of one cut circuit.  Tensors on the host
    are copied to the device first (pinned, on `stream`).  `out` may be a CUDA
    tensor or a pinned CPU tensor of 2^n entries; in the second case the
    kernels write the probabilities straight into it (no separate copy).
    Returns (out, FP64 sum on the device or None)."""
    dev = device or (tensors[0].device if tensors[0].is_cuda else torch.device("cuda", torch.cuda.current_device()))
    s = stream or torch.cuda.current_stream(dev)
    with torch.cuda.stream(s):
        dts = [t if t.is_cuda else t.to(dev, non_blocking=True) for t in tensors]
        if out is None:
            out = torch.empty(2 ** cc.n, dtype=dts[0].dtype, device=dev)
        elif out.dtype != dts[0].dtype or out.numel() != 2 ** cc.n or not out.is_contiguous() or \
                not (out.is_cuda or out.is_pinned()):
            raise ValueError("out must be a contiguous CUDA or pinned CPU tensor of 2^n entries in the tensors' dtype")
        sp = torch.empty(1, dtype=torch.float64, device=dev) if with_sum else None
    p = Problem.from_cut(cc, dts)
    cutqc_reconstruct_fd([p], [out], algo, sp, s)
    return out, sp


def cutqc_reconstruct_fd_noalloc(problem: Problem, out: torch.Tensor, sum_p: Optional[torch.Tensor] = None,
                                 stream=None) -> None:
    """Binding of cutqc_reconstruct_fd_noalloc: the two-subcircuit CUDA-core
    full definition with its scratch in the library's static device array (for
    callers that cannot let the library allocate device memory)."""
    here = torch.device("cuda", torch.cuda.current_device())
    if out.dtype != problem.dtype or out.numel() != 2 ** problem.n_qubits or not out.is_contiguous() or \
            not ((out.is_cuda and out.device == here) or out.is_pinned()):
        raise ValueError("out must be a contiguous tensor of 2^n entries in the tensors' dtype, on the current "
                         "CUDA device or in pinned host memory")
    sp = None
    if sum_p is not None:
        if sum_p.dtype != torch.float64 or not sum_p.is_cuda or sum_p.device != here:
            raise ValueError("sum_p must be a float64 tensor on the current CUDA device")
        sp = sum_p.data_ptr()
    _check(_lib.cutqc_reconstruct_fd_noalloc(C.byref(problem.c), C.c_void_p(out.data_ptr()), sp,
                                             _stream_ptr(stream)))


def cutqc_reconstruct_backward(problem: Problem, grads: Sequence[torch.Tensor], grad_out: Optional[torch.Tensor] = None,
                               edges: Optional[Sequence[Tuple[int, int]]] = None,
                               loss_value: Optional[torch.Tensor] = None, stream=None) -> None:
    """Binding of cutqc_reconstruct_backward: grads[c] <- dL/dT_c for
    L = sum_x G(x) p(x), with G = grad_out (2^n entries) or, when `edges` is
    given, the MaxCut cut count of each bit string generated on the fly.
    loss_value (CUDA float64, 1 entry) receives L."""
    if len(grads) != len(problem.tensors):
        raise ValueError("one gradient per subcircuit")
    for g, t in zip(grads, problem.tensors):
        if g.dtype != t.dtype or g.numel() != t.numel() or not g.is_cuda or not g.is_contiguous():
            raise ValueError("each gradient must be a contiguous CUDA tensor shaped like its tensor")
    gptr = (C.c_void_p * len(grads))(*[g.data_ptr() for g in grads])
    loss = None
    keep = None
    if edges is not None:
        flat = [int(q) for e in edges for q in e]
        keep = _i32(flat)
        loss = cutqc_loss(CUTQC_LOSS_MAXCUT, len(edges), keep)
    elif grad_out is None:
        raise ValueError("need grad_out or edges")
    if grad_out is not None and (grad_out.dtype != problem.dtype or grad_out.numel() != 2 ** problem.n_qubits):
        raise ValueError("grad_out must have 2^n entries in the tensors' dtype")
    lv = None
    if loss_value is not None:
        if loss_value.dtype != torch.float64 or not loss_value.is_cuda:
            raise ValueError("loss_value must be a CUDA float64 tensor")
        lv = loss_value.data_ptr()
    _check(_lib.cutqc_reconstruct_backward(C.byref(problem.c),
                                           C.c_void_p(grad_out.data_ptr()) if grad_out is not None else None,
                                           C.byref(loss) if loss is not None else None, gptr, lv,
                                           _stream_ptr(stream)))


def cutqc_reconstruct_dd(problem: Problem, roles: Sequence[int], bins: torch.Tensor, topk: int = 0,
                         algo: str = "auto", stream=None):
    """Binding of cutqc_reconstruct_dd (one dynamic-definition recursion,
    Algorithm 1).  roles[q]: 0 active, 1 merged, 2 zoomed at 0, 3 zoomed at 1.
    Fills `bins` (2^#active entries, the tensors' dtype) and returns the topk
    heaviest bins ranked in FP64 as (indices, values)."""
    n_act = sum(1 for r in roles if r == 0)
    if len(roles) != problem.n_qubits:
        raise ValueError("one role per qubit")
    if bins.dtype != problem.dtype or bins.numel() != 2 ** n_act or not bins.is_cuda:
        raise ValueError("bins must be a CUDA tensor of 2^#active entries in the tensors' dtype")
    r = (C.c_int8 * len(roles))(*[int(x) for x in roles])
    ti = (C.c_int64 * max(topk, 1))()
    tv = (C.c_double * max(topk, 1))()
    _check(_lib.cutqc_reconstruct_dd(C.byref(problem.c), r, C.c_void_p(bins.data_ptr()), topk, ti, tv,
                                     ALGOS[algo], _stream_ptr(stream)))
    return [int(ti[j]) for j in range(topk)], [float(tv[j]) for j in range(topk)]


def cutqc_simulate_subcircuit(sub: circuits.Subcircuit, dtype=torch.float32, device=None, stream=None,
                              out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Binding of cutqc_simulate_subcircuit: the attributed tensor of one
    subcircuit, simulated on the GPU (input preparation)."""
    dev = device or torch.device("cuda", torch.cuda.current_device())
    gates = (cutqc_gate * max(len(sub.gates), 1))()
    for i, g in enumerate(sub.gates):
        q1 = g.qubits[1] if len(g.qubits) > 1 else -1
        gates[i] = cutqc_gate(GATE_OPS[g.name], g.qubits[0], q1, g.params[0] if g.params else 0.0)
    n_out = (4 ** sub.k_in) * (4 ** sub.k_out) * (2 ** sub.n_eff)
    if out is None:
        out = torch.empty(n_out, dtype=dtype, device=dev)
    elif out.numel() != n_out or out.dtype != dtype or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous CUDA tensor of 4^k_in*4^k_out*2^n_eff entries in dtype")
    s = stream or torch.cuda.current_stream(dev)
    _check(_lib.cutqc_simulate_subcircuit(
        gates, len(sub.gates), sub.d, _i32([q for q, _ in sub.in_slots]), sub.k_in,
        _i32([q for q, _ in sub.out_slots]), sub.k_out, _i32([q for q, _ in sub.outputs]), sub.n_eff,
        CUTQC_F64 if dtype == torch.float64 else CUTQC_F32, C.c_void_p(out.data_ptr()), s.cuda_stream))
    return out


def cutqc_attribute(sub: circuits.Subcircuit, variant_probs: torch.Tensor, out: Optional[torch.Tensor] = None,
                    stream=None) -> torch.Tensor:
    """Binding of cutqc_attribute: the attributed tensor of one subcircuit from
    the output distributions of its variants, a CUDA tensor of
    4^k_in * 3^k_out * 2^d entries ([s][mb][y], see the C header)."""
    n_in = (4 ** sub.k_in) * (3 ** sub.k_out) * (2 ** sub.d)
    if not variant_probs.is_cuda or not variant_probs.is_contiguous() or variant_probs.numel() != n_in or \
            variant_probs.dtype not in (torch.float32, torch.float64):
        raise ValueError("variant_probs must be a contiguous CUDA float tensor of 4^k_in*3^k_out*2^d entries")
    n_out = (4 ** sub.k_in) * (4 ** sub.k_out) * (2 ** sub.n_eff)
    if out is None:
        out = torch.empty(n_out, dtype=variant_probs.dtype, device=variant_probs.device)
    elif out.numel() != n_out or out.dtype != variant_probs.dtype or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous CUDA tensor of 4^k_in*4^k_out*2^n_eff entries")
    s = stream or torch.cuda.current_stream(variant_probs.device)
    _check(_lib.cutqc_attribute(
        C.c_void_p(variant_probs.data_ptr()), sub.d, sub.k_in, _i32([q for q, _ in sub.out_slots]), sub.k_out,
        _i32([q for q, _ in sub.outputs]), sub.n_eff,
        CUTQC_F64 if variant_probs.dtype == torch.float64 else CUTQC_F32, C.c_void_p(out.data_ptr()),
        s.cuda_stream))
    return out


def cutqc_attribute_merged(sub: circuits.Subcircuit, variant_probs: torch.Tensor, roles: Sequence[int],
                           out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Binding of cutqc_attribute_merged: the merged tensor of one recursion of
    the dynamic definition, [4^k_in * 4^k_out][2^a], straight from the
    variants' output distributions.  roles[q] over global qubits: 0 active,
    1 merged, 2 zoomed at 0, 3 zoomed at 1."""
    n_in = (4 ** sub.k_in) * (3 ** sub.k_out) * (2 ** sub.d)
    if not variant_probs.is_cuda or not variant_probs.is_contiguous() or variant_probs.numel() != n_in or \
            variant_probs.dtype not in (torch.float32, torch.float64):
        raise ValueError("variant_probs must be a contiguous CUDA float tensor of 4^k_in*3^k_out*2^d entries")
    role_out = [int(roles[g]) for _, g in sub.outputs]
    a = sum(1 for r in role_out if r == 0)
    n_out = (4 ** sub.k_in) * (4 ** sub.k_out) * (2 ** a)
    if out is None:
        out = torch.empty(n_out, dtype=variant_probs.dtype, device=variant_probs.device)
    elif out.numel() != n_out or out.dtype != variant_probs.dtype or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous CUDA tensor of 4^k_in*4^k_out*2^a entries")
    s = stream or torch.cuda.current_stream(variant_probs.device)
    _check(_lib.cutqc_attribute_merged(
        C.c_void_p(variant_probs.data_ptr()), sub.d, sub.k_in, _i32([q for q, _ in sub.out_slots]), sub.k_out,
        _i32([q for q, _ in sub.outputs]), sub.n_eff, (C.c_int8 * max(1, len(role_out)))(*role_out),
        CUTQC_F64 if variant_probs.dtype == torch.float64 else CUTQC_F32, C.c_void_p(out.data_ptr()),
        s.cuda_stream))
    return out


def simulate_tensors(cc: circuits.CutCircuit, dtype=torch.float32, device=None) -> List[torch.Tensor]:
    """GPU-simulated tensors of every subcircuit of a cut circuit."""
    return [cutqc_simulate_subcircuit(s, dtype, device) for s in cc.subs]
