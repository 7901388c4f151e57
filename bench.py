#!/usr/bin/env python
"""Benchmark: full-definition reconstruction of a 24-qubit supremacy circuit.

Workload: a 4x6 supremacy-style grid circuit of depth 8 (seed 0), cut into
its left and right halves for a 15-qubit device (two subcircuits of 15 and
13 qubits, K = 4 wire cuts, 4^4 = 256 Kronecker terms, 2^12 outputs each):
the paper's Figure 12 setting.  Subcircuit tensors are FP32, produced by the
library's GPU subcircuit simulator before timing.  One step = one call of the
C ABI's cutqc_reconstruct_fd over the whole path (early-termination row
checks, compaction, operand preparation, the contraction into all 2^24
probabilities, the FP64 sum).

Metric: reconstructed probabilities per second (whole job, all ranks).  The
L2 is flushed (256 MiB written, then read back) before each timed step; each step is timed with
CUDA events on its stream; the max over ranks is reported.  With --gpus N
under torchrun every rank reconstructs its own replica (weak scaling, no
collective on the data path).

Each line reports the median step time (best and mean beside it), a
back-to-back steady-state timing with no flush, the dominant kernel's
roofline fraction, and, on rank 0 at N = 1, the FP64 oracle timed on the host
cores on the same input tensors (cpu_baseline) with the error of the timed
output against it (error_vs_oracle).  With --gpus N outside torchrun the
script starts the N ranks itself.

--impl reference times the FP64 CPU oracle on the workload: every step is the
plain sum over all 256 Kronecker terms for all 2^24 outputs.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "reconstructed probs/sec & % roofline at ≤1e-6 max abs err vs FP64 oracle"
UNIT = "probs/s"
WORKLOAD = "supremacy_4x6_depth8_K4_fd_fp32"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# DRAM traffic (read + write bytes) of one k_tc_gemm launch on this workload from
# the ncu capture summarised in profiles/k_tc_gemm_supremacy_4x6_k4.md, valid while
# the kernel source is unchanged (first 16 hex digits of its SHA-256)
TRAFFIC_TC = {"sha256_16": "c250ed940ba927e3", "bytes": 10.288e6}
# Library peaks of the machine's GB300 beside the driver's BF16 and copy figures,
# measured with `python bench.py --workload peaks --steps 10 --warmup 3`
# (torch.matmul 8192^3, best of 10): TF32 tensor cores, FP32 without TF32
# (CUDA cores) and FP64; summarised in profiles/peaks_gb300.md
LIBRARY_PEAKS = {"tf32_tflops": 1053.7, "fp32_tflops": 69.96, "fp64_tflops": 1.101}
FP32_ALU_TFLOPS = LIBRARY_PEAKS["fp32_tflops"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--algo", default="auto", choices=["auto", "cc", "tc_bf16x3", "tc_bf16x6", "tc_tf32x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="supremacy_4x6",
                    choices=["supremacy_4x6", "hwea10", "batch64", "qaoa30", "dd80", "attr_qaoa30", "attr_merged_qaoa30",
                             "metrics_qaoa30", "sim_supremacy4x6", "peaks"],
                    help="supremacy_4x6 is the benchmark line; the others time the other configurations")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return dict(FALLBACK_PEAKS), "fallback"


def tc_peak(pk, pk_src, algo):
    """Tensor peak for the split form that ran: the measured BF16 burst peak,
    or for TF32 the measured TF32 peak (the peaks file's if it has one, else
    the library peak measured on this machine)."""
    from paper_2012_02333_gb300 import cutqc
    if algo == getattr(cutqc, "CUTQC_TC_TF32X3", -1):
        if "tf32_tflops" in pk:
            return pk["tf32_tflops"], f"{pk_src} tf32"
        return LIBRARY_PEAKS["tf32_tflops"], "measured tf32 (torch.matmul, LIBRARY_PEAKS)"
    return pk["bf16_tflops"], f"{pk_src} bf16 burst"


def workload():
    from paper_2012_02333_gb300 import circuits
    return circuits.supremacy_4x6(0)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed
    region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """The maximum of a per-rank number over all ranks (the job's time is its
    slowest rank's); CUDA tensors under NCCL, host tensors under gloo."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n_out_per_rank, world, ms):
    """Whole-job throughput: every rank reconstructs its own replica (weak
    scaling, no collective on the data path), so the job processes
    world * n_out probabilities in the slowest rank's time."""
    return world * n_out_per_rank / (ms / 1e3)


def kept_terms(cc, tensors):
    """The algorithmic work: Kronecker terms whose factor rows are all
    non-zero (early termination, Sec. 4.2), counted on the host."""
    import numpy as np
    from itertools import product
    rows_nz = []
    for s, t in zip(cc.subs, tensors):
        v = t.cpu().numpy().reshape(4 ** s.k_in * 4 ** s.k_out, -1)
        rows_nz.append(np.any(v != 0, axis=1))
    k_eff = 0
    for dg in product(range(4), repeat=cc.n_cuts):
        ok = True
        for s, nz in zip(cc.subs, rows_nz):
            a = 0
            for c in s.in_cut:
                a = 4 * a + dg[c]
            b = 0
            for c in s.out_cut:
                b = 4 * b + dg[c]
            ok &= bool(nz[a * 4 ** s.k_out + b])
        k_eff += ok
    return k_eff


def step_ms(ts):
    """Median, best and mean of per-step times (ms); the median is the figure
    the line reports."""
    return {"median": statistics.median(ts), "best": min(ts), "mean": statistics.mean(ts)}


def error_stats(got, want, what):
    """Max-abs and total-variation error of a result against the oracle's."""
    import numpy as np
    d = np.asarray(got, np.float64) - np.asarray(want, np.float64)
    return {"max_abs_err": float(np.abs(d).max()), "tv": float(0.5 * np.abs(d).sum()),
            "entries_compared": int(d.size), "compared": what, "tol": 1e-6,
            "within_tol": bool(np.abs(d).max() <= 1e-6)}


def product_bins(rng, cc, roles, n_bins):
    """About n_bins distinct bin indices of a dynamic-definition recursion,
    drawn from a product of small per-subcircuit sets of active-output values,
    so each subcircuit's merged tensor is needed at only a few active values."""
    active = [q for q in range(cc.n) if roles[q] == 0]
    rank = {q: i for i, q in enumerate(active)}
    na = len(active)
    per = []
    for s in cc.subs:
        qs = [q for q in s.out_qubit if roles[q] == 0]
        per.append((qs, rng.choice(2 ** len(qs), size=min(2 ** len(qs), 32), replace=False) if qs else [0]))
    combos = set()
    tries = 0
    while len(combos) < n_bins and tries < 20 * n_bins:
        tries += 1
        b = 0
        for qs, vals in per:
            a = int(vals[rng.integers(len(vals))])
            for j, q in enumerate(qs):
                b |= ((a >> (len(qs) - 1 - j)) & 1) << (na - 1 - rank[q])
        combos.add(b)
    return sorted(combos)


def device_slab(torch, cc, ts, roles):
    """slab(c, a) for the oracle's selected-bin sum (dd_entries): gathers, on
    the device, the tensor entries of subcircuit c whose active outputs read
    `a` and zoomed outputs their fixed bits, and hands them to the host in row
    pieces of at most 512 MiB (data movement only; the sums are the oracle's)."""
    def slab(c, a):
        s = cc.subs[c]
        T = ts[c].view(4 ** s.k_in * 4 ** s.k_out, 2 ** s.n_eff)
        base = 0
        act = [i for i, q in enumerate(s.out_qubit) if roles[q] == 0]
        mrg = [i for i, q in enumerate(s.out_qubit) if roles[q] == 1]
        for j, i in enumerate(act):
            base |= ((a >> (len(act) - 1 - j)) & 1) << (s.n_eff - 1 - i)
        for i, q in enumerate(s.out_qubit):
            if roles[q] == 3:
                base |= 1 << (s.n_eff - 1 - i)
        m = torch.arange(2 ** len(mrg), device=T.device, dtype=torch.int64)
        cols = torch.full_like(m, base)
        for j, i in enumerate(mrg):
            cols |= ((m >> (len(mrg) - 1 - j)) & 1) << (s.n_eff - 1 - i)
        step = max(1, (1 << 27) // cols.numel())
        for r0 in range(0, T.shape[0], step):
            yield r0, T[r0:r0 + step].index_select(1, cols).cpu().numpy()
    return slab


def oracle_fd_leg(cc, host64, got_fn, n_sample=None, rng=None):
    """The cpu_baseline leg of a full-definition workload: the FP64 oracle's
    plain sum on the workload's own tensors, timed on the host cores, and the
    error of the GPU result against it.  With n_sample set, the oracle
    evaluates that many sampled outputs one by one (all 4^K terms each)
    instead of all 2^n.  got_fn(xs or None) returns the GPU result (all, or at
    xs) as a numpy array."""
    import numpy as np
    from oracle import reconstruct as rc
    t0 = time.perf_counter()
    if n_sample is None:
        want = rc.fd_full(cc.subs, host64, cc.n, cc.n_cuts)
        xs = None
    else:
        xs = sorted(set(int(x) for x in rng.integers(0, 2 ** cc.n, n_sample)))
        want = rc.fd_entries(cc.subs, host64, cc.n, cc.n_cuts, xs)
    dt = time.perf_counter() - t0
    n_units = 2 ** cc.n if xs is None else len(xs)
    what = (f"all 2^{cc.n} outputs" if xs is None else f"{len(xs)} sampled outputs of 2^{cc.n}")
    cpu = {"value": n_units / dt, "unit": "probs/s", "cores": 1, "kind": "oracle",
           "sample": f"{what}, every one of the 4^{cc.n_cuts} Kronecker terms, FP64 numpy oracle (no scaling)",
           "sample_seconds": dt, "host_cpus": os.cpu_count()}
    return cpu, error_stats(got_fn(xs), want, what + " vs the FP64 oracle on the same input tensors"), want


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands, timed on the host
    cores.  One step = the oracle's plain sum over all 256 Kronecker terms for
    all 2^24 outputs of the benchmark workload (nothing scaled)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    from oracle import attribution as at
    from oracle import reconstruct as rc
    cc = workload()
    T64 = [T.astype(np.float32).astype(np.float64) for T in at.tensors(cc)]
    W, K = args.warmup, args.steps
    times = []
    for i in range(W + K):
        t0 = time.perf_counter()
        rc.fd_full(cc.subs, T64, cc.n, cc.n_cuts)
        dt = time.perf_counter() - t0
        if i >= W:
            times.append(1e3 * dt)
    st = step_ms(times)
    ms = st["median"]
    value = 2 ** cc.n / (ms / 1e3)
    desc = (f"all 2^{cc.n} outputs of the workload, every one of the {4 ** cc.n_cuts} Kronecker terms, FP64 numpy "
            f"oracle on the oracle-simulated tensors rounded to FP32")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": ms, "ms_best": st["best"], "ms_mean": st["mean"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_qubits": cc.n, "n_cuts": cc.n_cuts},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    from paper_2012_02333_gb300 import cutqc

    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    cc = workload()
    n_out = 2 ** cc.n
    # input preparation (untimed): GPU-simulated FP32 subcircuit tensors
    tensors = cutqc.simulate_tensors(cc, torch.float32, dev)
    host = [t.cpu().pin_memory() for t in tensors]
    k_eff = kept_terms(cc, host)
    out = torch.empty(n_out, dtype=torch.float32, device=dev)
    sum_p = torch.empty(1, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    flush_sink = torch.empty((), dtype=torch.float32, device=dev)

    def flush_l2():
        # evict everything: write 256 MiB, then read it back so the dirty lines
        # are written back to HBM before the timed region starts
        flush.fill_(1.0)
        torch.sum(flush, dim=0, out=flush_sink)
    stream = torch.cuda.current_stream(dev)
    problem = cutqc.Problem.from_cut(cc, tensors)

    def step():
        cutqc.cutqc_reconstruct_fd([problem], [out], args.algo, sum_p, stream)

    for _ in range(max(args.warmup, 3)):
        flush_l2()
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clk = Clocks(dev.index)
    barrier(world)
    torch.cuda.synchronize()
    clk.start()
    l0 = cutqc.launch_count()
    for a, b in evs:
        flush_l2()
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    launches = cutqc.launch_count() - l0
    # steady state: the same steps back to back with no flush in between, so
    # each step also pays for writing the previous step's output back to HBM
    sa, sb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sa.record(stream)
    for _ in range(args.steps):
        step()
    sb.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    st = step_ms([a.elapsed_time(b) for a, b in evs])
    ms_steady = max_over_ranks(sa.elapsed_time(sb) / args.steps, world)
    # the dominant kernel alone: the same steps again with its launches
    # bracketed by events on its stream (this separates it from the kernels
    # before it, which otherwise overlap its start), flushed and back to back
    cutqc.profile_read()        # discard
    cutqc.profile(True)
    for _ in range(args.steps):
        flush_l2()
        step()
    torch.cuda.synchronize()
    n_main, main_ms = cutqc.profile_read()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    cutqc.profile(False)
    n_main2, main_ms2 = cutqc.profile_read()
    ms = max_over_ranks(st["median"], world)
    value = job_value(n_out, world, ms)
    kern_ms = main_ms / max(n_main, 1)
    kern_ms_steady = main_ms2 / max(n_main2, 1)

    # end to end through the public API: pinned host tensors in, probabilities out
    out_host = torch.empty(n_out, dtype=torch.float32).pin_memory()
    sum_host = torch.empty(1, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush_l2()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        # the contraction writes the probabilities straight into the pinned
        # host buffer (device -> host over the host link inside the call)
        o, sp = cutqc.reconstruct_fd(cc, host, algo=args.algo, out=out_host, stream=stream, device=dev)
        sum_host.copy_(sp, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
    e2e = max_over_ranks(statistics.median(e2e_ms), world)
    h2d = sum(t.numel() * t.element_size() for t in host)
    d2h = n_out * 4 + 8

    pk, pk_src = peaks()
    used_tc = cutqc.last_algo() != cutqc.CUTQC_CC
    flops1 = 2.0 * k_eff * n_out
    bytes_alg = n_out * 4 + sum(t.numel() * 4 for t in tensors)

    def roof_of(kms):
        t_s = kms / 1e3
        hbm = {"bytes_per_launch": bytes_alg, "achieved_gbs": bytes_alg / t_s / 1e9, "peak_gbs": pk["hbm_gbs"],
               "frac": bytes_alg / t_s / 1e9 / pk["hbm_gbs"], "t_roof_us": bytes_alg / (pk["hbm_gbs"] * 1e9) * 1e6}
        if used_tc:
            s, split_S = cutqc.last_split()
            peak_t, src = tc_peak(pk, pk_src, cutqc.last_algo())
            comp = {"flops_per_launch": s * flops1, "split_products": s, "split_bound_S": split_S,
                    "achieved_tflops": s * flops1 / t_s / 1e12, "peak_tflops": peak_t,
                    "frac": s * flops1 / t_s / 1e12 / peak_t, "peak_source": src,
                    "frac_single_product": flops1 / t_s / 1e12 / peak_t,
                    "t_roof_us": s * flops1 / (peak_t * 1e12) * 1e6}
            cbound = "tensor"
        else:
            comp = {"flops_per_launch": flops1, "achieved_tflops": flops1 / t_s / 1e12,
                    "peak_tflops": FP32_ALU_TFLOPS, "frac": flops1 / t_s / 1e12 / FP32_ALU_TFLOPS,
                    "peak_source": "measured fp32 CUDA-core matmul (LIBRARY_PEAKS)",
                    "t_roof_us": flops1 / (FP32_ALU_TFLOPS * 1e12) * 1e6}
            cbound = "alu"
        if comp["t_roof_us"] >= hbm["t_roof_us"]:
            r = {"bound": cbound, "achieved": comp["achieved_tflops"], "peak": comp["peak_tflops"],
                 "unit": "TFLOP/s", "frac": comp["frac"]}
        else:
            r = {"bound": "hbm", "achieved": hbm["achieved_gbs"], "peak": hbm["peak_gbs"], "unit": "GB/s",
                 "frac": hbm["frac"]}
        r.update({"t_roof_us": max(comp["t_roof_us"], hbm["t_roof_us"]), "compute": comp, "hbm": hbm})
        return r
    # the reported fraction is the lower of the two regimes: flushed L2 (inputs
    # from HBM, the output absorbed by L2) and back to back (the previous
    # output's write-back inside the launch)
    r_fl, r_st = roof_of(kern_ms), roof_of(kern_ms_steady)
    roof = dict(r_fl if r_fl["frac"] <= r_st["frac"] else r_st)
    roof["regime"] = "flushed" if r_fl["frac"] <= r_st["frac"] else "back_to_back"
    traffic = None
    if used_tc:
        import hashlib
        src = os.path.join(ROOT, "paper_2012_02333_gb300", "csrc", "k_tc.cu")
        if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == TRAFFIC_TC["sha256_16"]:
            traffic = TRAFFIC_TC["bytes"]
    roof.update({"traffic": traffic, "kernel_ms": kern_ms if roof["regime"] == "flushed" else kern_ms_steady,
                 "kernel_ms_flushed": kern_ms, "kernel_ms_back_to_back": kern_ms_steady,
                 "frac_flushed": r_fl["frac"], "frac_back_to_back": r_st["frac"], "peak_file": pk_src})

    dtype = {cutqc.CUTQC_CC: "f32"}.get(cutqc.last_algo(), None)
    if dtype is None:
        s, _ = cutqc.last_split()
        dtype = ("tf32" if cutqc.last_algo() == getattr(cutqc, "CUTQC_TC_TF32X3", -1) else "bf16") + f"x{s}-f32acc"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "ms_best": st["best"], "ms_mean": st["mean"],
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_qubits": cc.n, "n_cuts": cc.n_cuts,
                       "kronecker_terms": 4 ** cc.n_cuts, "nonzero_terms": k_eff,
                       "subcircuits": [[s.d, s.k_in, s.k_out, s.n_eff] for s in cc.subs],
                       "algo": args.algo, "inputs": "FP32 tensors from the GPU subcircuit simulator, seed 0",
                       "l2": "flushed before every timed step: 256 MiB written then read back (outside the timed region)",
                       "parallelism": f"replicas x{world}"},
            "steady_state": {"ms_per_step": ms_steady, "value": job_value(n_out, world, ms_steady),
                             "l2": "no flush: steps back to back, each pays the previous output's write-back"},
            "roofline": roof,
            "e2e": {"value": world * n_out / (e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e,
                    "path": "pinned host tensors in (copied on the stream), probabilities written by the "
                            "contraction straight into pinned host memory, FP64 sum copied back"},
            "gpu_launches": launches, "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        host64 = [t.numpy().astype(np.float64) for t in host]
        cpu, err, want = oracle_fd_leg(cc, host64, lambda xs: out.double().cpu().numpy())
        err["sum_p"] = float(sum_p.item())
        err["sum_p_minus_oracle_sum"] = float(sum_p.item() - want.sum())
        line["cpu_baseline"] = cpu
        line["error_vs_oracle"] = err
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_other(args):
    """Timings of the other configurations (not the benchmark line): the 10-qubit
    HWEA in FP64 (CUDA core), the 64-instance batch (graph replay), the 30-qubit
    QAOA MaxCut forward and adjoint, one 80-qubit dynamic-definition recursion
    with 30 active qubits.  Inputs come from the GPU subcircuit simulator."""
    import torch

    from paper_2012_02333_gb300 import circuits, cutqc, dd

    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    sink = torch.empty((), dtype=torch.float32, device=dev)

    def flush_l2():
        flush.fill_(1.0)
        torch.sum(flush, dim=0, out=sink)

    stats = {}

    def timed(step, key="main"):
        """Median step time (ms) over args.steps flushed steps; median, best and
        mean are kept under `key`."""
        for _ in range(max(args.warmup, 3)):
            flush_l2()
            step()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            flush_l2()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        stats[key] = step_ms(ts)
        return max_over_ranks(stats[key]["median"], world)

    import numpy as np
    rng = np.random.default_rng(2012)
    check = rank == 0 and world == 1 and not args.no_cpu_baseline
    extra = {}
    w = args.workload
    if w == "hwea10":
        cc = circuits.hwea_10q_k1(0)
        ts = cutqc.simulate_tensors(cc, torch.float64, dev)
        problem = cutqc.Problem.from_cut(cc, ts)
        out = torch.empty(2 ** cc.n, dtype=torch.float64, device=dev)
        ms = timed(lambda: cutqc.cutqc_reconstruct_fd([problem], [out], "cc"))
        if check:
            cpu, err, _ = oracle_fd_leg(cc, [t.cpu().numpy() for t in ts], lambda xs: out.cpu().numpy())
            extra.update({"cpu_baseline": cpu, "error_vs_oracle": err})
        units, unit, dtype = 2 ** cc.n, "probs/s", "f64"
        cfg = {"workload": "hwea10_K1_fd_fp64", "n_qubits": cc.n, "n_cuts": cc.n_cuts}
    elif w == "batch64":
        batch = circuits.batch_instances(64, 0)
        tss = [cutqc.simulate_tensors(cc, torch.float32, dev) for cc in batch]
        problems = [cutqc.Problem.from_cut(cc, t) for cc, t in zip(batch, tss)]
        outs = [torch.empty(2 ** cc.n, device=dev) for cc in batch]
        sums = torch.empty(len(batch), dtype=torch.float64, device=dev)
        ms = timed(lambda: cutqc.cutqc_reconstruct_fd(problems, outs, "auto", sums))
        # HBM roofline of the batch: every output written once, every
        # subcircuit tensor read once (group builds and operand pieces stay in L2
        # or are counted as overhead)
        bytes_alg = sum(o.numel() * 4 for o in outs) + sum(t.numel() * 4 for ts in tss for t in ts)
        pk, pk_src = peaks()
        gbs = bytes_alg / (ms / 1e3) / 1e9
        # the instances whose final contraction takes the tensor cores (a
        # single call in the automatic form chooses them), as a batch of their
        # own: the split-precision form against the FP32 CUDA-core form
        tc_idx = []
        for i, (p, o) in enumerate(zip(problems, outs)):
            cutqc.cutqc_reconstruct_fd([p], [o], "auto", sums[i:i + 1])
            if cutqc.last_algo() != cutqc.CUTQC_CC:
                tc_idx.append(i)
        tp, to = [problems[i] for i in tc_idx], [outs[i] for i in tc_idx]
        tc_sub = {}
        if tc_idx:
            tc_sub = {"instances": tc_idx, "n_outputs": sum(2 ** batch[i].n for i in tc_idx),
                      "split_ms": timed(lambda: cutqc.cutqc_reconstruct_fd(tp, to, "auto", sums[:len(tp)]),
                                        "tc_subset"),
                      "cc_ms": timed(lambda: cutqc.cutqc_reconstruct_fd(tp, to, "cc", sums[:len(tp)]),
                                     "tc_subset_cc"),
                      "what": "the instances whose final contraction has more than 16 kept terms (the "
                              "tensor-core form), as one graph-captured batch: automatic split-precision "
                              "form against every contraction on the FP32 CUDA-core form"}
            tc_sub["speedup_vs_cc"] = tc_sub["cc_ms"] / tc_sub["split_ms"]
        extra = {"cc_only_ms": timed(lambda: cutqc.cutqc_reconstruct_fd(problems, outs, "cc", sums), "cc"),
                 "cc_only": "every instance on the FP32 CUDA-core form, same graph replay",
                 "tensor_core_subset": tc_sub,
                 "roofline": {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                              "frac": gbs / pk["hbm_gbs"], "traffic": None, "algorithmic_bytes": bytes_alg,
                              "peak_file": pk_src}}
        if check:
            # 64 sampled outputs of every instance, each by all of its 4^K terms,
            # against the automatic form's outputs (the timed line's)
            cutqc.cutqc_reconstruct_fd(problems, outs, "auto", sums)
            cpu_s, n_cpu, gots = 0.0, 0, []
            for cc, t, o in zip(batch, tss, outs):
                cpu, err, want = oracle_fd_leg(
                    cc, [x.double().cpu().numpy() for x in t],
                    lambda xs, o=o: o[torch.tensor(xs, device=dev)].double().cpu().numpy(), 64, rng)
                cpu_s += cpu["sample_seconds"]
                n_cpu += err["entries_compared"]
                gots.append(err["max_abs_err"])
            extra["cpu_baseline"] = {"value": n_cpu / cpu_s, "unit": "probs/s", "cores": 1, "kind": "oracle",
                                     "sample": "64 sampled outputs of each of the 64 instances, every one of "
                                               "its 4^K Kronecker terms, FP64 numpy oracle (no scaling)",
                                     "sample_seconds": cpu_s}
            extra["error_vs_oracle"] = {"max_abs_err": max(gots), "entries_compared": n_cpu, "tol": 1e-6,
                                        "within_tol": max(gots) <= 1e-6,
                                        "compared": "64 sampled outputs per instance vs the FP64 oracle on the "
                                                    "same input tensors"}
        units, unit, dtype = sum(2 ** cc.n for cc in batch), "probs/s", "f32 (per instance cc or bf16x3/x6)"
        cfg = {"workload": "batch64_hwea_aqft_bv_fd_fp32", "instances": len(batch),
               "n_qubits": [cc.n for cc in batch], "n_cuts": [cc.n_cuts for cc in batch],
               "subcircuits": [len(cc.subs) for cc in batch], "launch": "CUDA graph replay"}
    elif w == "qaoa30":
        cc = circuits.qaoa_2cluster(15, 0)
        ts = cutqc.simulate_tensors(cc, torch.float32, dev)
        problem = cutqc.Problem.from_cut(cc, ts)
        out = torch.empty(2 ** cc.n, device=dev)
        sp = torch.empty(1, dtype=torch.float64, device=dev)
        ms = timed(lambda: cutqc.cutqc_reconstruct_fd([problem], [out], "auto", sp))
        grads = [torch.empty_like(t) for t in ts]
        loss = torch.empty(1, dtype=torch.float64, device=dev)
        ms_bwd = timed(lambda: cutqc.cutqc_reconstruct_backward(problem, grads, edges=cc.edges, loss_value=loss),
                       "bwd")
        extra = {"adjoint_ms": ms_bwd, "adjoint": "MaxCut loss and dL/dT of both subcircuits",
                 "expected_cut": float(loss.item()),
                 "cc_only_ms": timed(lambda: cutqc.cutqc_reconstruct_fd([problem], [out], "cc", sp), "cc"),
                 "cc_only": "forward on the FP32 CUDA-core form"}
        # roofline of the forward step: the slower of the split products at the
        # BF16 peak and the output plus tensors at the HBM rate
        cutqc.cutqc_reconstruct_fd([problem], [out], "auto", sp)
        nseg, _ = cutqc.last_split()
        k_eff = kept_terms(cc, ts)
        pk, pk_src = peaks()
        t_tc = nseg * 2.0 * k_eff * 2 ** cc.n / (pk["bf16_tflops"] * 1e12)
        b_alg = 2 ** cc.n * 4 + sum(t.numel() * 4 for t in ts)
        t_hbm = b_alg / (pk["hbm_gbs"] * 1e9)
        if t_tc >= t_hbm:
            roof = {"bound": "tensor", "achieved": nseg * 2.0 * k_eff * 2 ** cc.n / (ms / 1e3) / 1e12,
                    "peak": pk["bf16_tflops"], "unit": "TFLOP/s"}
        else:
            roof = {"bound": "hbm", "achieved": b_alg / (ms / 1e3) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s"}
        roof.update({"frac": max(t_tc, t_hbm) / (ms / 1e3), "traffic": None, "split_products": nseg,
                     "kept_terms": k_eff, "t_roof_us": 1e6 * max(t_tc, t_hbm), "peak_file": pk_src,
                     "of": "the whole forward step (preparation and contraction)"})
        extra["roofline"] = roof
        # the adjoint's HBM roofline: both tensors read once, both gradients
        # written once (the row sums, keys and tables are a few MB in L2)
        b_bwd = 2 * sum(t.numel() * 4 for t in ts)
        extra["adjoint_roofline"] = {"bound": "hbm", "achieved": b_bwd / (ms_bwd / 1e3) / 1e9,
                                     "peak": pk["hbm_gbs"], "unit": "GB/s",
                                     "frac": b_bwd / (ms_bwd / 1e3) / 1e9 / pk["hbm_gbs"],
                                     "algorithmic_bytes": b_bwd, "traffic": None, "peak_file": pk_src}
        if check:
            cutqc.cutqc_reconstruct_fd([problem], [out], "auto", sp)
            cpu, err, _ = oracle_fd_leg(cc, [t.double().cpu().numpy() for t in ts],
                                        lambda xs: out[torch.tensor(xs, device=dev)].double().cpu().numpy(),
                                        4096, rng)
            extra.update({"cpu_baseline": cpu, "error_vs_oracle": err})
        units, unit, dtype = 2 ** cc.n, "probs/s", "bf16x3/x6-f32acc"
        cfg = {"workload": "qaoa30_maxcut_K4_fd_fp32", "n_qubits": cc.n, "n_cuts": cc.n_cuts}
    elif w == "sim_supremacy4x6":
        # the GPU subcircuit simulator (input preparation, here timed): every
        # variant of both subcircuits of the 4x6 supremacy workload simulated
        # in complex FP64, attributed (Eq. 3, Eq. 2) into the FP32 tensors
        cc = circuits.supremacy_4x6(0)
        outs = [torch.empty((4 ** s.k_in) * (4 ** s.k_out) * (2 ** s.n_eff), device=dev) for s in cc.subs]
        # FP64 work as applied: the init variants (4^k_in states of 2^d
        # amplitudes) go through every gate (dense complex matrices: 14 flops
        # per amplitude for a 1-qubit gate, 30 for a 2-qubit one), then each
        # of the 3^k_out measurement bases rotates its X- and Y-measured
        # qubits (14 flops per amplitude each); the attribution's few flops
        # per output are not counted
        flops = 0
        for sub in cc.subs:
            nv, dim = 4 ** sub.k_in, 2 ** sub.d
            per = sum(30 if len(g.qubits) == 2 else 14 for g in sub.gates)
            rot = sub.k_out * 2 * 3 ** max(sub.k_out - 1, 0)
            flops += nv * dim * (per + 14 * rot)

        def sim_step():
            for sub, o in zip(cc.subs, outs):
                cutqc.cutqc_simulate_subcircuit(sub, torch.float32, dev, out=o)
        ms = timed(sim_step)
        units, unit, dtype = sum(o.numel() for o in outs), "tensor entries/s", "complex f64 state, f32 tensors"
        extra = {"gates": sum(len(sub.gates) for sub in cc.subs),
                 "roofline": {"bound": "alu", "achieved": flops / (ms / 1e3) / 1e12,
                              "peak": LIBRARY_PEAKS["fp64_tflops"], "unit": "TFLOP/s",
                              "frac": flops / (ms / 1e3) / 1e12 / LIBRARY_PEAKS["fp64_tflops"],
                              "traffic": None, "algorithmic_flops": flops,
                              "peak_file": "measured FP64 (torch.matmul, LIBRARY_PEAKS)",
                              "note": "FP64-equivalent flops of the dense gate matrices as applied (the gates "
                                      "run in double-float on the FP32 pipes, so this is the fraction of the "
                                      "FP64 peak the FP64 form would need); the states (2 and 8 MB) stay in L2"}}
        cfg = {"workload": "sim_supremacy4x6_fp64_state", "subcircuits": [[s.d, s.k_in, s.k_out, s.n_eff]
                                                                          for s in cc.subs],
               "step": "simulate every variant of both subcircuits and attribute (input preparation; each call "
                       "ends with a stream synchronisation; its scratch is kept per device)"}
    elif w == "metrics_qaoa30":
        # Eq. 16 chi^2 and total variation between the split-precision and the
        # FP32 CUDA-core reconstructions of QAOA-30 (2^30 entries each), and
        # 2^20 draws from the first (uniforms from a seeded generator)
        cc = circuits.qaoa_2cluster(15, 0)
        ts = cutqc.simulate_tensors(cc, torch.float32, dev)
        pa, _ = cutqc.reconstruct_fd(cc, ts, algo="auto")
        pb, _ = cutqc.reconstruct_fd(cc, ts, algo="cc")
        del ts
        ms = timed(lambda: cutqc.cutqc_distance(pa, pb))
        chi, tv = cutqc.cutqc_distance(pa, pb)
        gen = torch.Generator(device=dev)
        gen.manual_seed(0)
        u = torch.rand(1 << 20, dtype=torch.float64, generator=gen, device=dev)
        ms_s = timed(lambda: cutqc.cutqc_sample(pa, u), "sample")
        bytes_alg = 2 * pa.numel() * 4
        pk, pk_src = peaks()
        extra = {"roofline": {"bound": "hbm", "achieved": bytes_alg / (ms / 1e3) / 1e9, "peak": pk["hbm_gbs"],
                              "unit": "GB/s", "frac": bytes_alg / (ms / 1e3) / 1e9 / pk["hbm_gbs"], "traffic": None,
                              "algorithmic_bytes": bytes_alg, "peak_file": pk_src},
                 "chi2_tc_vs_cc": chi.item(), "tv_tc_vs_cc": tv.item(),
                 "sample_ms": ms_s, "samples": u.numel(),
                 "sample_rate_per_s": u.numel() / (ms_s / 1e3)}
        units, unit, dtype = pa.numel(), "entries/s", "f32 in, compensated f32 sums, f64 total"
        cfg = {"workload": "metrics_qaoa30_fp32", "n": pa.numel(),
               "step": "chi^2 (Eq. 16) and total variation of two 2^30-entry distributions; sampling timed beside it"}
        del pb
    elif w == "attr_merged_qaoa30":
        # the merged tensors of a first dynamic-definition recursion (20 of 30
        # qubits active, the rest merged) of both QAOA-30 subcircuits, straight
        # from seeded synthetic variant distributions
        cc = circuits.qaoa_2cluster(15, 0)
        roles = [0 if q < 20 else 1 for q in range(cc.n)]
        gen = torch.Generator(device=dev)
        gen.manual_seed(0)
        probs, outs = [], []
        for sub in cc.subs:
            v = torch.rand((4 ** sub.k_in) * (3 ** sub.k_out), 2 ** sub.d, generator=gen, device=dev)
            probs.append((v / v.sum(dim=1, keepdim=True)).reshape(-1).contiguous())
            outs.append(cutqc.cutqc_attribute_merged(sub, probs[-1], roles))

        def attr_step():
            for sub, p, o in zip(cc.subs, probs, outs):
                cutqc.cutqc_attribute_merged(sub, p, roles, o)
        ms = timed(attr_step)
        bytes_alg = sum(p.numel() * 4 + o.numel() * 4 for p, o in zip(probs, outs))
        pk, pk_src = peaks()
        extra = {"roofline": {"bound": "hbm", "achieved": bytes_alg / (ms / 1e3) / 1e9, "peak": pk["hbm_gbs"],
                              "unit": "GB/s", "frac": bytes_alg / (ms / 1e3) / 1e9 / pk["hbm_gbs"],
                              "traffic": None, "algorithmic_bytes": bytes_alg, "peak_file": pk_src}}
        if check:
            from oracle import attribution as at
            t0 = time.perf_counter()
            wants = [at.attribute_merged(sub, p.double().cpu().numpy().reshape((4 ** sub.k_in) * (3 ** sub.k_out), -1),
                                         roles) for sub, p in zip(cc.subs, probs)]
            dt = time.perf_counter() - t0
            extra["cpu_baseline"] = {"value": sum(p.numel() for p in probs) / dt, "unit": "variant outcomes/s",
                                     "cores": 1, "kind": "oracle", "sample_seconds": dt,
                                     "sample": "both subcircuits' merged tensors in full, FP64 numpy oracle"}
            extra["error_vs_oracle"] = error_stats(
                np.concatenate([o.double().cpu().numpy() for o in outs]),
                np.concatenate([w.reshape(-1) for w in wants]), "every merged tensor entry vs the FP64 oracle")
        units, unit, dtype = sum(p.numel() for p in probs), "variant outcomes/s", "f32 in, compensated f32 sums"
        cfg = {"workload": "attr_merged_qaoa30_fp32", "roles": "qubits 0-19 active, 20-29 merged",
               "subcircuits": [[s.d, s.k_in, s.k_out, s.n_eff] for s in cc.subs],
               "merged_tensor_entries": [o.numel() for o in outs],
               "inputs": "seeded uniform variant distributions normalised per variant (synthetic shot frequencies)",
               "step": "merge the variant distributions over the merged outputs, then Eq. 3 and Eq. 2, both "
                       "subcircuits"}
    elif w == "attr_qaoa30":
        # attribution of both QAOA-30 subcircuits from seeded synthetic variant
        # distributions (uniform numbers normalised per variant, the shape of
        # shot-count frequencies): 4^2 x 3^2 variants of 2^17 outcomes each
        cc = circuits.qaoa_2cluster(15, 0)
        gen = torch.Generator(device=dev)
        gen.manual_seed(0)
        probs, outs = [], []
        for sub in cc.subs:
            v = torch.rand((4 ** sub.k_in) * (3 ** sub.k_out), 2 ** sub.d, generator=gen, device=dev)
            probs.append((v / v.sum(dim=1, keepdim=True)).reshape(-1).contiguous())
            outs.append(torch.empty((4 ** sub.k_in) * (4 ** sub.k_out) * (2 ** sub.n_eff), device=dev))

        def attr_step():
            for sub, p, o in zip(cc.subs, probs, outs):
                cutqc.cutqc_attribute(sub, p, o)
        ms = timed(attr_step)
        bytes_alg = sum(p.numel() * 4 + o.numel() * 4 for p, o in zip(probs, outs))
        pk, pk_src = peaks()
        extra = {"roofline": {"bound": "hbm", "achieved": bytes_alg / (ms / 1e3) / 1e9, "peak": pk["hbm_gbs"],
                              "unit": "GB/s", "frac": bytes_alg / (ms / 1e3) / 1e9 / pk["hbm_gbs"],
                              "traffic": None, "algorithmic_bytes": bytes_alg, "peak_file": pk_src}}
        if check:
            from oracle import attribution as at
            t0 = time.perf_counter()
            wants = [at.attribute(sub, p.double().cpu().numpy().reshape((4 ** sub.k_in) * (3 ** sub.k_out), -1))
                     for sub, p in zip(cc.subs, probs)]
            dt = time.perf_counter() - t0
            extra["cpu_baseline"] = {"value": sum(o.numel() for o in outs) / dt, "unit": "tensor entries/s",
                                     "cores": 1, "kind": "oracle", "sample_seconds": dt,
                                     "sample": "both subcircuits' tensors in full, FP64 numpy oracle (Eq. 3, Eq. 2)"}
            extra["error_vs_oracle"] = error_stats(
                np.concatenate([o.double().cpu().numpy() for o in outs]),
                np.concatenate([w.reshape(-1) for w in wants]), "every tensor entry vs the FP64 oracle")
        units, unit, dtype = sum(o.numel() for o in outs), "tensor entries/s", "f32 in, compensated f32 sums"
        cfg = {"workload": "attr_qaoa30_fp32", "subcircuits": [[s.d, s.k_in, s.k_out, s.n_eff] for s in cc.subs],
               "inputs": "seeded uniform variant distributions normalised per variant (synthetic shot frequencies)",
               "step": "Eq. 3 then Eq. 2 for both subcircuits"}
    else:
        cc = circuits.grid_blocks(8, 10, 10, 0, 2, 2, 8, 25)
        ts = cutqc.simulate_tensors(cc, torch.float32, dev)
        problem = cutqc.Problem.from_cut(cc, ts)
        roles = dd.initial_roles(cc.n, 30)
        bins = torch.empty(2 ** 30, device=dev)
        ms = timed(lambda: cutqc.cutqc_reconstruct_dd(problem, roles, bins, 32, "auto"))
        extra = {"cc_only_ms": timed(lambda: cutqc.cutqc_reconstruct_dd(problem, roles, bins, 32, "cc"), "cc"),
                 "cc_only": "one recursion with the final contraction on the FP32 CUDA-core form"}
        # HBM roofline of one recursion: every tensor read once by the merges,
        # the merged tensors (rounded sum and compensation, 8 bytes a value)
        # written once and read once, the 2^30 bins written once
        merged = 0
        for sub in cc.subs:
            a_c = sum(1 for q in sub.out_qubit if roles[q] == 0)
            merged += (4 ** (sub.k_in + sub.k_out)) * (2 ** a_c) * 8
        b_alg = sum(t.numel() * 4 for t in ts) + 2 * merged + bins.numel() * 4
        pk, pk_src = peaks()
        extra["roofline"] = {"bound": "hbm", "achieved": b_alg / (ms / 1e3) / 1e9, "peak": pk["hbm_gbs"],
                             "unit": "GB/s", "frac": b_alg / (ms / 1e3) / 1e9 / pk["hbm_gbs"], "traffic": None,
                             "algorithmic_bytes": b_alg, "peak_file": pk_src,
                             "of": "one recursion: merges, contraction into the bins, top-32 and FP64 re-ranking"}
        if check:
            from oracle import reconstruct as rc
            top = cutqc.cutqc_reconstruct_dd(problem, roles, bins, 32, "auto")
            xs = product_bins(rng, cc, roles, 1024)
            slab = device_slab(torch, cc, ts, roles)
            t0 = time.perf_counter()
            cache = {}
            want_top = rc.dd_entries(cc.subs, slab, cc.n, cc.n_cuts, roles, top[0], cache)
            want = rc.dd_entries(cc.subs, slab, cc.n, cc.n_cuts, roles, xs, cache)
            dt = time.perf_counter() - t0
            err = error_stats(bins[torch.tensor(xs, device=dev)].double().cpu().numpy(), want,
                              f"{len(xs)} sampled bins of 2^30 vs the FP64 oracle's sum over merged tensors")
            err["top32_fp64_max_abs_err"] = float(np.abs(np.array(top[1]) - want_top).max())
            err["top1_matches_oracle"] = bool(top[0][int(np.argmax(want_top))] == top[0][0])
            extra.update({"error_vs_oracle": err,
                          "cpu_baseline": {"value": (len(xs) + len(top[0])) / dt, "unit": "bins/s", "cores": 1,
                                           "kind": "oracle", "sample_seconds": dt,
                                           "sample": "the recursion's top-32 and 1024 sampled bins by the plain FP64 "
                                                     "sum over merged tensors (merging read from the device)"}})
        del bins
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = dd.run(cc, ts, 30, 10, "bfs")
        torch.cuda.synchronize()
        extra.update({"ten_recursions_s": time.perf_counter() - t0, "recursions": len(st.recursions),
                      "ten_recursions": "Algorithm 1 driver, BFS, 10 recursions of 2^30 bins, host wall clock"})
        del st
        units, unit, dtype = 2 ** 30, "bins/s", "f32 bins, FP64 ranking"
        cfg = {"workload": "dd80_grid8x10_d10_30active_fp32", "n_qubits": cc.n, "n_cuts": cc.n_cuts,
               "subcircuits": [[s.d, s.k_in, s.k_out, s.n_eff] for s in cc.subs],
               "step": "one recursion: merge, contraction into 2^30 bins, top-32 with FP64 re-ranking"}
    line = {"metric": METRIC, "value": world * units / (ms / 1e3), "unit": unit, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "ms_best": stats["main"]["best"],
            "ms_mean": stats["main"]["mean"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": cfg}
    line.update(extra)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def launch_ranks(n):
    """--gpus N outside torchrun: start N ranks of this command on this node
    (one process per GPU, rendezvous on 127.0.0.1) and return their status."""
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def run_peaks(args):
    """Library peaks beside the driver's BF16 and copy figures: a plain
    torch.matmul of 8192^3 in TF32 (tensor cores), FP32 without TF32 (the
    library's CUDA-core GEMM) and FP64, best of `steps` after `warmup`, CUDA
    events; 2 N^3 flops each."""
    import torch
    torch.cuda.set_device(0)
    out = {}
    for name, dt, tf32 in (("tf32_tflops", torch.float32, True), ("fp32_tflops", torch.float32, False),
                           ("fp64_tflops", torch.float64, False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        n = 8192
        a = torch.randn(n, n, dtype=dt, device="cuda")
        b = torch.randn(n, n, dtype=dt, device="cuda")
        c = torch.empty(n, n, dtype=dt, device="cuda")
        for _ in range(max(args.warmup, 3)):
            torch.matmul(a, b, out=c)
        best = 1e30
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[name] = 2.0 * n ** 3 / (best / 1e3) / 1e12
        del a, b, c
    torch.backends.cuda.matmul.allow_tf32 = False
    # write-only HBM rate (context for kernels whose traffic is all stores):
    # torch's fill of 4 GiB, best of `steps`
    buf = torch.empty(1 << 30, dtype=torch.float32, device="cuda")
    best = 1e30
    for i in range(max(args.warmup, 3) + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        buf.fill_(float(i))
        e1.record()
        torch.cuda.synchronize()
        if i >= max(args.warmup, 3):
            best = min(best, e0.elapsed_time(e1))
    out["write_gbs"] = buf.numel() * 4 / (best / 1e3) / 1e9
    del buf
    print(json.dumps({"peaks": out, "how": "torch.matmul 8192^3 and torch fill of 4 GiB, best of %d, CUDA events"
                      % args.steps}), flush=True)


def main():
    args = parse()
    if args.workload == "peaks":
        run_peaks(args)
        return
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(launch_ranks(args.gpus))
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "supremacy_4x6":
        run_other(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
