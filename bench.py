#!/usr/bin/env python
"""Benchmark: forward + gradient of the IQP Monte-Carlo estimator.

Workload (default): m = 100000 random generators on k in {1,2,3} qubits,
n = 1000 qubits, l = 10000 observables (Bernoulli(0.05) bits), s = 10000
samples, theta ~ U(-0.05, 0.05). One step = one iqp_expval_value_and_grad
call for the linear loss sum_a w_a <Z_a> (parities once; one phase pass that
yields the cos / mean / standard-error partials and W; the gradient
contraction). The autograd form of the same step (iqp_expval_keep_phi, then
iqp_expval_grad_from_phi) is timed beside it (`other_step`).

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2501_04776_gb300 import inputs as I  # noqa: E402

METRIC = "fwd+grad ms, 10k observables x 10k samples x 1e5 gates"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="split_bf16", choices=["split_bf16", "fp32", "sparse_fp32", "loworder_fp32"])
    ap.add_argument("--workload", default="random", choices=["random", "mmd", "million"],
                    help="random: k in 1..3 random gates (sizes from --n --m --l --s); mmd: all 1- and 2-body "
                         "gates, p_sigma observables (--n --l --s); million: n=5000, 1e6 random 1-2-body gates")
    ap.add_argument("--n", type=int, default=1000)
    ap.add_argument("--m", type=int, default=100_000)
    ap.add_argument("--l", type=int, default=None)
    ap.add_argument("--s", type=int, default=None)
    ap.add_argument("--fp32-steps", type=int, default=2, help="timed steps of the plain FP32 form (0 = skip)")
    ap.add_argument("--step", default="fused", choices=["fused", "two-call"],
                    help="fused: iqp_expval_value_and_grad (one phase pass); two-call: the estimates, then the "
                         "gradient, as autograd runs them (Phi kept between the calls where the precision allows, "
                         "else recomputed); the other form is timed too")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-rows", action="store_true", help="skip the bitflip and MMD per-call timings")
    ap.add_argument("--cpu-sample-l", type=int, default=512)
    ap.add_argument("--cpu-sample-s", type=int, default=10_000)
    ap.add_argument("--ref-sample-l", type=int, default=64,
                    help="observables per timed step of the reference arm (the FP64 oracle)")
    return ap.parse_args()


def workload(args):
    if args.workload == "mmd":
        return I.mmd_training(n=args.n, l=args.l or 2000, s=args.s or 5000)
    if args.workload == "million":
        return I.million_gates(l=args.l or 4096, s=args.s or 16384)
    return I.random_gates(n=args.n, m=args.m, l=args.l or 10_000, s=args.s or 10_000)


def workload_name(args, p):
    if args.workload == "mmd":
        desc = f"all 1- and 2-body gates n={p.n} m={p.m}, l={p.l} observables ~ Bernoulli(p_sigma), s={p.s}"
    elif args.workload == "million":
        desc = f"random 1-2-body gates n={p.n} m={p.m}, l={p.l} (Bernoulli 0.01), s={p.s}"
    else:
        desc = f"random-gates n={p.n} m={p.m} (k in 1..3) l={p.l} (Bernoulli 0.05) s={p.s}"
    return desc + ", fwd+grad of sum_a w_a <Z_a>"


# ------------------------------------------------------------- CPU baseline

def cpu_baseline(p, args, gpu_ev=None, gpu_se=None, gpu_grad_fn=None):
    """Time the FP64 oracle on a bounded sample and extrapolate to the full
    step with its cost model T = 2 t_row (l + s) + c_phase l s: each oracle call
    forms both parity matrices (linear in rows) and then loops over
    (observable, sample) pairs. Also measures the GPU error on sampled
    observables against the oracle on identical samples."""
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    oracle.set_threads(cores)
    th = p.theta.astype(np.float64)
    ls, ss = min(args.cpu_sample_l, p.l), min(args.cpu_sample_s, p.s)
    A1, Z1 = p.A[:ls], p.Z[:ss]
    t0 = time.perf_counter()
    oracle.parity(p.n, Z1, p.G)
    t_par = time.perf_counter() - t0
    t_row = t_par / ss
    w = I.Rng(99).normal(p.l, 1)
    t0 = time.perf_counter()
    oracle.expval(p.n, p.G, A1, Z1, th)
    oracle.expval_grad(p.n, p.G, A1, Z1, th, -w[:ls] / ss, None)
    t_step = time.perf_counter() - t0
    c_phase = max(t_step - 2 * t_row * (ls + ss), 0.0) / (ls * ss)
    full_s = 2 * t_row * (p.l + p.s) + c_phase * p.l * p.s
    out = {
        "value": full_s * 1e3, "unit": "ms", "cores": cores, "kind": "oracle",
        "sample": (f"oracle expval+expval_grad on {ls} observables x {ss} samples x all {p.m} gates "
                   f"({t_step:.2f} s) plus parity of {ss} sample rows ({t_par:.2f} s); extrapolated to "
                   f"{p.l} x {p.s} with T = 2*t_row*(l+s) + c*l*s"),
        "measured_s": round(t_step + t_par, 3),
    }
    if gpu_ev is not None:
        idx = np.unique(np.sort(I.Rng(77).integers(8, p.l, 1)))
        ev, se, _, _ = oracle.expval(p.n, p.G, p.A[idx], p.Z, th)
        err = {"observables_checked": int(idx.size),
               "max_abs_err_expval": float(np.max(np.abs(gpu_ev[idx] - ev))),
               "max_abs_err_std_err": float(np.max(np.abs(gpu_se[idx] - se)))}
        if gpu_grad_fn is not None:
            alpha = np.zeros(p.l)
            alpha[idx] = -w[idx] / p.s
            g = gpu_grad_fn(alpha)
            want = oracle.expval_grad(p.n, p.G, p.A[idx], p.Z, th, alpha[idx], None)
            err["grad_rel_l2"] = float(np.linalg.norm(g - want) / np.linalg.norm(want))
        out["error_vs_fp64"] = err
    return out


def run_reference(args, rank, world):
    """The FP64 oracle on the machine's host cores, on the same workload, metric and unit as the GPU arm. A full
    step (10^4 observables x 10^4 samples x 10^5 gates) takes minutes of CPU time, so each timed step is a
    bounded sample: --ref-sample-l observables with all samples and gates (expval, then the gradient of
    sum_a w_a <Z_a>). The line's value is that sample extrapolated to all observables (the oracle's cost is
    the sample parities, formed once per call, plus a part linear in the observables) and says so
    ("extrapolated": true). The n=8 and n=300 configurations are also timed in full, once each."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    oracle.set_threads(cores)
    p = workload(args)
    th = p.theta.astype(np.float64)
    w = I.Rng(99).normal(p.l, 1)
    ls = min(args.ref_sample_l, p.l)
    A1 = p.A[:ls]
    t0 = time.perf_counter()
    oracle.parity(p.n, p.Z, p.G)  # the sample parities: the part of a call that does not scale with l
    t_zpar = time.perf_counter() - t0
    step_s = []
    for _ in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.expval(p.n, p.G, A1, p.Z, th)
        oracle.expval_grad(p.n, p.G, A1, p.Z, th, -w[:ls] / p.s, None)
        step_s.append(time.perf_counter() - t0)
    t_sample = statistics.mean(step_s[args.warmup:])
    per_obs = max(t_sample - 2 * t_zpar, 0.0) / ls
    ms = (2 * t_zpar + per_obs * p.l) * 1e3
    full = {}
    for q in (I.tiny_local(), I.local300()):
        wq = I.Rng(99).normal(q.l, 1)
        t0 = time.perf_counter()
        oracle.expval(q.n, q.G, q.A, q.Z, q.theta.astype(np.float64))
        oracle.expval_grad(q.n, q.G, q.A, q.Z, q.theta.astype(np.float64), -wq / q.s, None)
        full[q.name] = {"n": q.n, "m": q.m, "l": q.l, "s": q.s, "ms": round((time.perf_counter() - t0) * 1e3, 1),
                        "extrapolated": False}
    sample = (f"each step: oracle expval + expval_grad on {ls} of {p.l} observables x all {p.s} samples x all {p.m} "
              f"gates, {t_sample:.2f} s mean over {args.steps} timed steps; value = 2 t_par + (t_step - 2 t_par) "
              f"l / {ls} with t_par = {t_zpar:.2f} s (the sample parities, formed once per call)")
    base = {"value": ms, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample, "extrapolated": True,
            "sampled_fraction": round(ls / p.l, 5), "measured_step_s": round(t_sample, 3)}
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded splitmix64)",
        "config": {"workload": workload_name(args, p), "n": p.n, "m": p.m, "l": p.l, "s": p.s,
                   "precision": "fp64 CPU oracle"},
        "extrapolated": True, "sampled_fraction": round(ls / p.l, 5),
        "cpu_baseline": base, "full_runs": full,
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ traffic

def tensor_source_sha():
    """First 16 hex digits of sha256 over the tensor-core kernel sources (tc.cu, common.cuh): a committed ncu
    record applies only while the sources still hash to the value it was captured with."""
    import hashlib
    h = hashlib.sha256()
    for f in ("tc.cu", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2501_04776_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, sizes):
    """DRAM bytes per contraction of `kernel` (summed over its launches), from the committed one-pass ncu
    capture of the same workload (profiles/dram_traffic.json), or None if the kernel sources changed since the
    capture or the workload differs."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
        if tensor_source_sha() != rec["source_sha"]:
            return None
        if tuple(sizes) != tuple(rec["full_size"]):
            return None
        return rec["kernels"][kernel]["traffic_bytes_full"]
    except Exception:
        return None


def tensor_pipe_record(kernel):
    """Tensor-pipe activity of `kernel` from the committed ncu capture (profiles/tensor_pipe.json: metric
    sm__pipe_tensor_cycles_active, small case), with its source; None once the kernel sources changed."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "tensor_pipe.json")))
        if tensor_source_sha() != rec["source_sha"]:
            return None
        k = rec["kernels"][kernel]
        return {"pct_of_elapsed": k["pct_of_peak_sustained_elapsed"], "pct_of_active": k["pct_of_peak_sustained_active"],
                "metric": rec["metric"], "case": rec["case"], "source": "profiles/tensor_pipe.json, "
                + rec["summary"]}
    except Exception:
        return None


# --------------------------------------------------------------- replicas

def max_over_ranks(x: float, device=None) -> float:
    """The slowest replica's value (all ranks get it); x itself when no
    process group is running or it has one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------- rooflines and the other hot-path rows

def split_bf16_roofline(kt, dom, l, s, m, steps, peaks, step_ms=None, contractions=2):
    """Roofline of the dominant tensor-core kernel on the method's work: the contraction of eq. Emat is
    2 l s m flops (useful); the split-BF16 form runs two BF16 products (hi, lo) of it on the tensor pipe
    (executed, 4 l s m), reported beside it. One contraction per launch group (the phase kernel's whole
    tiles and split last round are timed together). The whole step's useful rate counts `contractions`
    contractions (fused step: phase and gradient; two-call with recompute: three)."""
    useful = 2.0 * l * s * m
    peak = peaks.get("bf16_tflops_sustained") or 1700.0
    per = kt[dom]["total_ms"] / max(1, steps)
    ach = useful / (per * 1e-3) / 1e12
    roof = {"bound": "tensor", "kernel": dom, "achieved": round(ach, 1), "peak": peak, "unit": "TFLOP/s",
            "frac": round(ach / peak, 4),
            "work": "useful: 2 l s m flops per contraction (eq. Emat); the split's second BF16 product is not counted",
            "flops_per_contraction": useful, "ms_per_contraction": round(per, 4),
            "launches_per_contraction": round(kt[dom]["launches"] / max(1, steps), 2),
            "executed": {"tflops": round(2 * ach, 1), "frac": round(2 * ach / peak, 4),
                         "flops_per_contraction": 2 * useful,
                         "note": "two BF16 products (hi and lo parts of 2 theta, or of W) per contraction on the "
                                 "tensor pipe"},
            "tensor_pipe": tensor_pipe_record(dom),
            "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"
            if "bf16_tflops_sustained" in peaks else "fallback 1.7 PFLOP/s sustained (of fallback)"}
    if step_ms:
        st = contractions * useful / (step_ms * 1e-3) / 1e12
        roof["step_useful"] = {"tflops": round(st, 1), "frac": round(st / peak, 4), "contractions": contractions}
    return roof

def tensor_algorithmic_bytes(kernel, l, s, m):
    """Bytes a tensor-core contraction must move at least once, each operand read once and each result
    written once. Phase pass of the fused step: P_A and P_Z bits (rows of ceil(m / 256) * 4 words), W hi and
    lo written (BF16, l x s each), the (sum cos, M2) partials (16 bytes per 64 samples). Gradient: W hi and lo
    read, P_Z^T and P_A^T bits, the FP64 partial rows (two per 256 observables)."""
    ldp = -(-m // 256) * 4
    if kernel == "grad_tc":
        return 4.0 * l * s + 32.0 * m * (-(-s // 256) + -(-l // 256)) + 16.0 * -(-l // 256) * m
    return 8.0 * ldp * (l + s) + 4.0 * l * s + 16.0 * l * -(-s // 64)


def generator_pairs(n, G):
    """Number of distinct qubit pairs that carry a weight-2 generator
    (host-side count from the packed rows)."""
    G = np.ascontiguousarray(G, dtype=np.uint64)
    wt = np.bitwise_count(G).sum(axis=1)
    rows = G[wt == 2]
    if rows.shape[0] == 0:
        return 0
    lo = np.full(rows.shape[0], -1, dtype=np.int64)
    hi = np.full(rows.shape[0], -1, dtype=np.int64)
    for w in range(rows.shape[1]):
        x = rows[:, w]
        nz = x != 0
        low = (x & (~x + np.uint64(1)))
        lbit = np.where(nz, np.log2(np.where(nz, low, 1).astype(np.float64)).astype(np.int64), -1) + 64 * w
        hbit = np.where(nz, np.floor(np.log2(np.where(nz, x, 1).astype(np.float64))).astype(np.int64), -1) + 64 * w
        lo = np.where((lo < 0) & nz, lbit, lo)
        hi = np.where(nz, hbit, hi)
    return int(np.unique(lo * n + hi).size)


def nnz_parities(api, n, A, G):
    """nnz(P_A) (computed on the GPU): the row-sparse form does nnz * s signed
    additions per pass."""
    x = api.parity(n, A, G).view(-1)
    x = x - ((x >> 1) & 0x5555555555555555)
    x = (x & 0x3333333333333333) + ((x >> 2) & 0x3333333333333333)
    x = (x + (x >> 4)) & 0x0F0F0F0F0F0F0F0F
    return int(((x * 0x0101010101010101) >> 56).sum().item())


def parity_roofline(kt, peaks, n, m, l, s, steps, calls=2, loworder=False):
    """The parity gathers of one step (`calls` library calls, each forming
    P_A, P_A^T and P_Z, P_Z^T from A and Z): algorithmic bytes = the bit
    matrices written (each l m / 8 or s m / 8 bytes, twice) plus the rows of
    A and Z read, against the measured HBM copy bandwidth. The low-order form
    forms no parity matrices: per call it lists the generators' supports (G
    read, 16 bytes per gate written) and transposes Z (bits read and
    written); the gradient transposes A once per step."""
    if "parity" not in kt:
        return None
    words = lambda bits: -(-bits // 64)
    if loworder:
        wn = words(n) + (words(n) & 1)
        nbytes = calls * (m * wn * 8 + m * 16 + 2 * s * wn * 8) + 2 * l * wn * 8
    else:
        nbytes = calls * 8 * (2 * l * words(m) + 2 * s * words(m) + (l + s) * words(n))
    ms = kt["parity"]["total_ms"] / max(1, steps)
    hbm = peaks.get("hbm_gbs") or 6800.0
    gbs = nbytes / (ms * 1e-3) / 1e9
    names = "k_support_list + k_bit_transpose" if loworder else "k_parity_prep + k_gather_transpose"
    return {"bound": "hbm", "kernels": names, "bytes_per_step": nbytes,
            "ms_per_step": round(ms, 4), "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(gbs / hbm, 4), "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}


def loworder_roofline(kt, clocks, n, G, s, peaks=None):
    """The low-order form's pair contractions (M = C S and H = (s V) S^T),
    one launch each. On the tensor cores (the default): dense n x n x s
    contractions in split BF16, 2 * 2 n^2 s executed flops per launch, against
    the measured sustained BF16 peak. As sign-flip additions (IQP_LO_TC=0):
    2 p s FP32 additions per launch, p = qubit pairs with a generator, against
    one add per lane per clock. Either way the useful work is 2 p s."""
    useful = 2.0 * generator_pairs(n, G) * s
    avg_ms = kt["loworder_gemm"]["avg_ms"]
    if os.environ.get("IQP_LO_TC", "1") != "0" and n >= 256:
        peaks = peaks or {}
        executed = 4.0 * n * n * s
        peak = peaks.get("bf16_tflops_sustained") or 1700.0
        ach = executed / (avg_ms * 1e-3) / 1e12
        return {"bound": "tensor", "kernel": "loworder_gemm (pair contractions, tcgen05 split BF16)",
                "achieved": round(ach, 1), "peak": peak, "unit": "TFLOP/s", "frac": round(ach / peak, 4),
                "flops_per_launch": executed, "useful_adds_per_launch": useful,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"
                if "bf16_tflops_sustained" in peaks else "fallback 1.7 PFLOP/s sustained (of fallback)"}
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = 152 * 128 * mhz * 1e6 / 1e12
    ach = useful / (avg_ms * 1e-3) / 1e12
    return {"bound": "alu", "kernel": "loworder_gemm (pair contractions)", "achieved": round(ach, 2),
            "peak": round(peak, 1), "unit": "Tadd/s", "frac": round(ach / peak, 4), "adds_per_launch": useful,
            "peak_source": "FP32 add: 152 SMs x 128 lanes x max SM clock"}


def _kernel_times(lib):
    from paper_2501_04776_gb300 import _lib
    kt = {}
    for k, name in enumerate(_lib.KERNELS):
        tot, cnt = ctypes.c_double(0), ctypes.c_uint64(0)
        lib.iqp_profile_query(k, ctypes.byref(tot), ctypes.byref(cnt))
        if cnt.value:
            kt[name] = {"launches": int(cnt.value), "total_ms": round(tot.value, 4),
                        "avg_ms": round(tot.value / cnt.value, 4)}
    return kt


def other_rows(args, lib, dev, st, timed, peaks, clocks, G, A, theta, w, n, m, l):
    """Per-call timings of the paths beside the headline step, each on its
    own workload: the bitflip circuit on the headline's G, A, theta, and one
    MMD^2 loss + gradient call of the MMD training workload."""
    import torch
    from paper_2501_04776_gb300 import _lib, api
    P = ctypes.c_void_p
    hbm = peaks.get("hbm_gbs") or 6800.0
    out = {}

    # Stochastic bitflip circuit: exact products and their gradient (FP64).
    ws = torch.empty(lib.iqp_workspace_bytes(_lib.OP_BITFLIP, n, m, l, 1, 0, _lib.FP32), dtype=torch.uint8,
                     device=dev)
    ev = torch.empty(l, dtype=torch.float64, device=dev)
    gr = torch.empty(m, dtype=torch.float64, device=dev)
    wd = torch.from_numpy(np.ascontiguousarray(w, dtype=np.float64)).to(dev)

    def bitflip():
        _lib.check(lib.iqp_bitflip_expval(n, P(G.data_ptr()), m, G.shape[1], P(A.data_ptr()), l, A.shape[1],
                                          P(theta.data_ptr()), P(ev.data_ptr()), P(ws.data_ptr()), ws.numel(), st),
                   "iqp_bitflip_expval")
        _lib.check(lib.iqp_bitflip_grad(n, P(G.data_ptr()), m, G.shape[1], P(A.data_ptr()), l, A.shape[1],
                                        P(theta.data_ptr()), P(wd.data_ptr()), P(gr.data_ptr()), P(ws.data_ptr()),
                                        ws.numel(), st), "iqp_bitflip_grad")

    lib.iqp_profile_reset()
    ms, _ = timed(None, args.steps, args.warmup, profile=True, fn=bitflip)
    kt = _kernel_times(lib)
    ldp, ldlt = -(-m // 256) * 4, -(-l // 256) * 4
    # The product / gradient-sum kernels read P_A (l x ldp words) or P_A^T
    # (m x ldlt words) once, a small fraction of HBM time; their work is one
    # FP64 multiply (product over a row's set bits, run by both calls) or add
    # (gradient sum over a column's set bits) per set bit: 3 nnz(P_A) FP64
    # operations per call pair, against the FP64 pipe's sustained rate of one
    # operation per SM per clock (the rate ncu's pipe_fp64 percentages imply
    # for these DMULs).
    nbytes = 8.0 * (l * ldp + m * ldlt)
    nnz = nnz_parities(api, n, A, G)
    fp64_ops = 3.0 * nnz
    bf_ms = kt.get("bitflip", {}).get("total_ms", 0.0) / max(1, args.steps)
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    fp64_peak = 152 * 1 * mhz * 1e6 / 1e12  # TFLOP/s, one DMUL / DADD per SM per clock
    ach = fp64_ops / (bf_ms * 1e-3) / 1e12 if bf_ms else None
    out["bitflip_fwd_grad"] = {
        "workload": f"bitflip circuit, n={n} m={m} l={l} (the headline's G, A, theta), FP64",
        "ms_per_call_pair": round(statistics.mean(ms), 3), "kernels": kt,
        "roofline": {"bound": "alu", "kernel": "bitflip (FP64 product and gradient sums)",
                     "achieved": round(ach, 4) if ach else None, "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
                     "frac": round(ach / fp64_peak, 4) if ach else None, "fp64_ops_per_call_pair": fp64_ops,
                     "nnz_PA": nnz, "bytes_per_call_pair": nbytes,
                     "hbm_frac": round(nbytes / (bf_ms * 1e-3) / 1e9 / hbm, 4) if bf_ms else None,
                     "peak_source": "FP64 pipe: 152 SMs x 1 operation per clock x max SM clock (from ncu's "
                                    "sm__inst_executed_pipe_fp64 percentage of peak for k_bitflip_rows)"}}
    del ws

    # MMD^2 loss and gradient, one training step's call (unbiased form), in
    # the tensor-core form and in the row-sparse form.
    p = I.mmd_training()
    Gm, Am, Zm, Xm = (torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).to(dev)
                      for x in (p.G, p.A, p.Z, p.X))
    thm = torch.from_numpy(p.theta).to(dev)
    mm, lm, sm, Nm = p.G.shape[0], p.A.shape[0], p.Z.shape[0], p.X.shape[0]
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    gm = torch.empty(mm, dtype=torch.float64, device=dev)
    nnz = nnz_parities(api, p.n, Am, Gm)
    for prec, tag in ((_lib.SPLIT_BF16, "split_bf16"), (_lib.SPARSE_FP32, "sparse_fp32"),
                      (_lib.LOWORDER_FP32, "loworder_fp32")):
        ws = torch.empty(lib.iqp_workspace_bytes(_lib.OP_MMD_LOSS_GRAD, p.n, mm, lm, sm, Nm, prec),
                         dtype=torch.uint8, device=dev)

        def mmd(sp=st):
            _lib.check(lib.iqp_mmd_loss_grad(p.n, P(Gm.data_ptr()), mm, Gm.shape[1], P(Am.data_ptr()), lm,
                                             Am.shape[1], P(Zm.data_ptr()), sm, Zm.shape[1], P(Xm.data_ptr()), Nm,
                                             Xm.shape[1], P(thm.data_ptr()), prec, 1, P(loss.data_ptr()),
                                             P(gm.data_ptr()), P(ws.data_ptr()), ws.numel(), sp),
                       "iqp_mmd_loss_grad")

        lib.iqp_profile_reset()
        ms, _ = timed(None, args.steps, args.warmup, profile=True, fn=mmd)
        kt = _kernel_times(lib)
        if prec == _lib.SPLIT_BF16:
            dom = max(("phase_tc", "recompute_tc", "grad_tc"), key=lambda k: kt.get(k, {}).get("total_ms", 0.0))
            roof = split_bf16_roofline(kt, dom, lm, sm, mm, args.steps, peaks, statistics.mean(ms), 2)
        elif prec == _lib.LOWORDER_FP32:
            roof = loworder_roofline(kt, clocks, p.n, p.G, sm, peaks)
        else:
            # Forward kernel: nnz * s FP32 signed additions; peak = one FP32
            # add per lane per clock: 152 SMs x 128 lanes x max SM clock.
            mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
            peak = 152 * 128 * mhz * 1e6 / 1e12
            ach = nnz * sm / (kt["phase_sparse"]["avg_ms"] * 1e-3) / 1e12
            roof = {"bound": "alu", "kernel": "phase_sparse", "achieved": round(ach, 2), "peak": round(peak, 1),
                    "unit": "Tadd/s", "frac": round(ach / peak, 4), "adds_per_launch": nnz * sm,
                    "nnz_PA": nnz, "density_PA": round(nnz / (lm * mm), 5),
                    "peak_source": "FP32 add: 152 SMs x 128 lanes x max SM clock"}
        out["mmd_loss_grad_" + tag] = {
            "workload": f"MMD^2 loss + grad, n={p.n} m={mm} (all 1- and 2-body) l={lm} s={sm} N={Nm}, {tag}",
            "ms_per_call": round(statistics.mean(ms), 3), "kernels": kt, "roofline": roof}
        if prec == _lib.LOWORDER_FP32:
            # The same call captured once in a CUDA graph and replayed (its
            # ~26 short launches then cost no host-side launch overhead).
            side = torch.cuda.Stream(dev)
            side.wait_stream(torch.cuda.current_stream(dev))
            with torch.cuda.stream(side):
                for _ in range(2):
                    mmd(P(side.cuda_stream))
            torch.cuda.current_stream(dev).wait_stream(side)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                mmd(P(torch.cuda.current_stream(dev).cuda_stream))
            ms_g, _ = timed(None, args.steps, args.warmup, profile=False, fn=graph.replay)
            out["mmd_loss_grad_" + tag]["ms_per_call_cuda_graph"] = round(statistics.mean(ms_g), 3)
            del graph
        del ws
    return out


# ------------------------------------------------ the other workload shapes

PREC_CODE = {"split_bf16": 1, "fp32": 0, "sparse_fp32": 2, "loworder_fp32": 3}


def alu_peak(clocks, per_lane_per_clock=1):
    """FP32 SIMT peak: 152 SMs x 128 lanes x max SM clock (x 2 for an FMA counted as two flops)."""
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    return 152 * 128 * per_lane_per_clock * mhz * 1e6 / 1e12


def row_roofline(prec, kt, p, steps, peaks, clocks, api, dev_A, dev_G, step_ms, contractions, fused):
    """Roofline of a row's dominant kernel, by form: split BF16 on the tensor pipe (useful 2 l s m per
    contraction), FP32 on the FMA pipe (2 l s m per launch), row-sparse on FP32 adds (nnz(P_A) s per pass,
    twice in the fused one-pass kernel), low-order on its pair contractions."""
    l, s, m = p.A.shape[0], p.Z.shape[0], p.G.shape[0]
    if prec == "split_bf16":
        dom = max(("phase_tc", "recompute_tc", "grad_tc"), key=lambda k: kt.get(k, {}).get("total_ms", 0.0))
        return split_bf16_roofline(kt, dom, l, s, m, steps, peaks, step_ms, contractions)
    if prec == "fp32":
        dom = max(("phase_fp32", "recompute_fp32", "grad_fp32"), key=lambda k: kt.get(k, {}).get("total_ms", 0.0))
        ach = 2.0 * l * s * m / (kt[dom]["avg_ms"] * 1e-3) / 1e12
        peak = alu_peak(clocks, 2)
        return {"bound": "alu", "kernel": dom, "achieved": round(ach, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
                "frac": round(ach / peak, 4), "flops_per_launch": 2.0 * l * s * m,
                "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 x max SM clock"}
    if prec == "sparse_fp32":
        nnz = nnz_parities(api, p.n, dev_A, dev_G)
        adds = (2 if fused else 1) * nnz * s
        ach = adds / (kt["phase_sparse"]["avg_ms"] * 1e-3) / 1e12
        peak = alu_peak(clocks)
        return {"bound": "alu", "kernel": "phase_sparse", "achieved": round(ach, 2), "peak": round(peak, 1),
                "unit": "Tadd/s", "frac": round(ach / peak, 4), "adds_per_launch": adds, "nnz_PA": nnz,
                "density_PA": round(nnz / (l * m), 5), "peak_source": "FP32 add: 152 SMs x 128 lanes x max SM clock"}
    return loworder_roofline(kt, clocks, p.n, p.G, s, peaks)


def sampled_oracle_errors(p, idx, ev, se, grad_fn):
    """Error of a GPU result against the FP64 oracle on the sampled observables idx, with the oracle
    restricted to the gates that anticommute with at least one of them (every other gate adds exactly zero
    to their phases and has an exactly zero gradient entry for a loss on them), on all samples."""
    import oracle
    A = p.A[idx]
    J = np.nonzero(oracle.parity(p.n, A, p.G).any(axis=0))[0]
    G, th = p.G[J], p.theta.astype(np.float64)[J]
    S1, S2 = np.zeros(idx.size), np.zeros(idx.size)
    for i0 in range(0, p.Z.shape[0], 4096):
        _, _, s1, s2 = oracle.expval(p.n, G, A, p.Z[i0:i0 + 4096], th)
        S1 += s1
        S2 += s2
    s = p.Z.shape[0]
    want_ev = S1 / s
    want_se = np.sqrt(np.maximum(S2 / s - want_ev ** 2, 0.0) / s)
    alpha = np.zeros(p.A.shape[0])
    alpha[idx] = I.Rng(7).normal(idx.size, 1) / s
    want_g = np.zeros(p.G.shape[0])
    for i0 in range(0, s, 4096):
        want_g[J] += oracle.expval_grad(p.n, G, A, p.Z[i0:i0 + 4096], th, alpha[idx], None)
    g = grad_fn(alpha)
    return {"observables_checked": int(idx.size), "gates_relevant": int(J.size),
            "max_abs_err_expval": float(np.max(np.abs(ev[idx] - want_ev))),
            "max_abs_err_std_err": float(np.max(np.abs(se[idx] - want_se))),
            "grad_rel_l2": float(np.linalg.norm(g - want_g) / np.linalg.norm(want_g))}


def workload_rows(args, lib, dev, st, timed, peaks, clocks):
    """The paper's other benchmark configurations (Sec. 4.1, 4.2), each timed through the C ABI on its own
    synthetic workload: the n=300 one- and two-body circuit (estimates, then the gradient of sum_a w_a <Z_a>
    as autograd runs them), the 1e5-gate random circuit at n=100 and n=5000 (one fused call), the
    million-gate circuit in all three forms that apply (one fused call), and 50 Adam steps of the MMD
    training workload. FP64 errors on sampled observables come from the CPU oracle (skipped with
    --no-cpu-baseline)."""
    import torch
    from paper_2501_04776_gb300 import _lib, api, train
    P = ctypes.c_void_p
    specs = [
        ("local300", lambda: I.local300(), [("split_bf16", 3, 2), ("fp32", 2, 1)], False, 8),
        ("random_gates_n100", lambda: I.random_gates(n=100), [("split_bf16", 3, 2), ("fp32", 1, 1)], True, 8),
        ("random_gates_n5000", lambda: I.random_gates(n=5000), [("split_bf16", 3, 2), ("fp32", 1, 1)], True, 8),
        ("million_gates", lambda: I.million_gates(),
         [("split_bf16", 2, 1), ("sparse_fp32", 2, 1), ("loworder_fp32", 5, 2)], True, 6),
    ]
    rows = {}
    for name, make, forms, fused, nsample in specs:
        try:
            p = make()
            n, m, l, s = p.n, p.G.shape[0], p.A.shape[0], p.Z.shape[0]
            G, A, Z = (api.to_device_bits(x, dev) for x in (p.G, p.A, p.Z))
            th = torch.from_numpy(p.theta).to(dev)
            w = I.Rng(99).normal(l, 1)
            al = torch.from_numpy(-w / s).to(dev)
            ev = torch.empty(l, dtype=torch.float64, device=dev)
            se = torch.empty_like(ev)
            g = torch.empty(m, dtype=torch.float64, device=dev)
            row = {"workload": p.name, "n": n, "m": m, "l": l, "s": s,
                   "step": "one iqp_expval_value_and_grad call" if fused else
                   "iqp_expval(_keep_phi), then iqp_expval_grad(_from_phi) (the autograd pair; Phi kept where the "
                   "form allows)", "forms": {}}
            for prec, steps, warm in forms:
                code = PREC_CODE[prec]
                nb = max(lib.iqp_workspace_bytes(_lib.OP_EXPVAL, n, m, l, s, 0, code),
                         lib.iqp_workspace_bytes(_lib.OP_EXPVAL_GRAD, n, m, l, s, 0, code))
                ws = torch.zeros(nb, dtype=torch.uint8, device=dev)
                keep = code in api.KEEP_PHI and not fused
                phi = torch.empty((l, api.phi_ld(s)) if keep else (1, 64), dtype=torch.float32, device=dev)
                args_bits = (n, P(G.data_ptr()), m, G.shape[1], P(A.data_ptr()), l, A.shape[1], P(Z.data_ptr()), s,
                             Z.shape[1], P(th.data_ptr()))

                def call(args_bits=args_bits, code=code, ws=ws, phi=phi, keep=keep):
                    if fused:
                        _lib.check(lib.iqp_expval_value_and_grad(*args_bits, P(al.data_ptr()), None, code,
                                                                 P(ev.data_ptr()), P(se.data_ptr()), P(g.data_ptr()),
                                                                 P(ws.data_ptr()), ws.numel(), st), "value_and_grad")
                    elif keep:
                        _lib.check(lib.iqp_expval_keep_phi(*args_bits, code, P(ev.data_ptr()), P(se.data_ptr()),
                                                           P(phi.data_ptr()), phi.shape[1], P(ws.data_ptr()),
                                                           ws.numel(), st), "keep_phi")
                        _lib.check(lib.iqp_expval_grad_from_phi(*args_bits, P(al.data_ptr()), None, code,
                                                                P(phi.data_ptr()), phi.shape[1], P(g.data_ptr()),
                                                                P(ws.data_ptr()), ws.numel(), st), "grad_from_phi")
                    else:
                        _lib.check(lib.iqp_expval(*args_bits, code, P(ev.data_ptr()), P(se.data_ptr()),
                                                  P(ws.data_ptr()), ws.numel(), st), "expval")
                        _lib.check(lib.iqp_expval_grad(*args_bits, P(al.data_ptr()), None, code, P(g.data_ptr()),
                                                       P(ws.data_ptr()), ws.numel(), st), "expval_grad")

                ms, launches = timed(None, steps, warm, profile=True, fn=call)
                kt = _kernel_times(lib)
                status = lib.iqp_read_status(P(ws.data_ptr()), ws.numel(), st)
                mean_ms = statistics.mean(ms)
                contractions = 2 if (fused or keep) else 3
                f = {"ms_per_call": round(mean_ms, 3), "calls_timed": steps, "gpu_launches_per_call":
                     round(launches / steps, 1), "device_status": int(status), "kernels": kt,
                     "roofline": row_roofline(prec, kt, p, steps, peaks, clocks, api, A, G, mean_ms, contractions,
                                              fused)}
                if not args.no_cpu_baseline:
                    call()
                    torch.cuda.synchronize()
                    evh, seh = ev.cpu().numpy(), se.cpu().numpy()

                    def grad_fn(alpha_np, args_bits=args_bits, code=code, ws=ws):
                        a2 = torch.from_numpy(alpha_np).to(dev)
                        g2 = torch.empty(m, dtype=torch.float64, device=dev)
                        _lib.check(lib.iqp_expval_grad(*args_bits, P(a2.data_ptr()), None, code, P(g2.data_ptr()),
                                                       P(ws.data_ptr()), ws.numel(), st), "expval_grad")
                        return g2.cpu().numpy()
                    idx = np.unique(np.sort(I.Rng(77).integers(nsample, l, 1)))
                    f["error_vs_fp64"] = sampled_oracle_errors(p, idx, evh, seh, grad_fn)
                row["forms"][prec] = f
                del ws, phi
                torch.cuda.empty_cache()
            rows[name] = row
            del G, A, Z
            torch.cuda.empty_cache()
        except Exception as e:  # a failed row is reported, the headline line still prints
            rows[name] = {"error": repr(e)[:400]}

    # 50 Adam steps of the MMD^2 loss (training workload: fresh observables and samples drawn on the device
    # every step), in the low-order form and in split BF16.
    p = I.mmd_training()
    adam = {"workload": p.name + ", 50 Adam steps, lr 1e-3, device-drawn observables and samples", "forms": {}}
    for prec in ("loworder_fp32", "split_bf16"):
        try:
            train.adam_mmd(p, steps=2, lr=1e-3, precision=prec, device_rng=True)  # warm-up (and the build)
            torch.cuda.synchronize()
            lib.iqp_profile_reset()
            lib.iqp_profile_enable(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, losses = train.adam_mmd(p, steps=50, lr=1e-3, precision=prec, device_rng=True)
            e1.record()
            torch.cuda.synchronize()
            lib.iqp_profile_enable(0)
            kt = _kernel_times(lib)
            ms = e0.elapsed_time(e1) / 50
            if prec == "split_bf16":
                dom = max(("phase_tc", "recompute_tc", "grad_tc"), key=lambda k: kt.get(k, {}).get("total_ms", 0.0))
                roof = split_bf16_roofline(kt, dom, p.A.shape[0], p.Z.shape[0], p.G.shape[0], 50, peaks, ms, 2)
            else:
                roof = loworder_roofline(kt, clocks, p.n, p.G, p.Z.shape[0], peaks)
            adam["forms"][prec] = {"ms_per_step": round(ms, 3), "loss_first": losses[0], "loss_last": losses[-1],
                                   "kernels": kt, "roofline": roof}
        except Exception as e:
            adam["forms"][prec] = {"error": repr(e)[:400]}
    rows["mmd_training_adam"] = adam
    return rows


# ---------------------------------------------------------------- GPU arm

def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_2501_04776_gb300 import _lib, api, build

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    lib = _lib.load()
    prec = {"split_bf16": _lib.SPLIT_BF16, "fp32": _lib.FP32, "sparse_fp32": _lib.SPARSE_FP32,
            "loworder_fp32": _lib.LOWORDER_FP32}[args.precision]
    if prec == _lib.SPLIT_BF16 and not lib.iqp_tensor_path_available():
        raise SystemExit("the split-BF16 tensor path needs an sm_103 GPU")

    p = workload(args)
    n, m, l, s = p.n, p.m, p.l, p.s
    w = I.Rng(99).normal(l, 1)
    dev = torch.device("cuda", local)
    G, A, Z = (api.to_device_bits(x, dev) for x in (p.G, p.A, p.Z))
    theta = torch.from_numpy(p.theta).to(dev)
    alpha = torch.from_numpy(-w / s).to(dev)
    ev = torch.empty(l, dtype=torch.float64, device=dev)
    se = torch.empty(l, dtype=torch.float64, device=dev)
    grad = torch.empty(m, dtype=torch.float64, device=dev)
    nbytes = max(lib.iqp_workspace_bytes(_lib.OP_EXPVAL, n, m, l, s, 0, prec),
                 lib.iqp_workspace_bytes(_lib.OP_EXPVAL_GRAD, n, m, l, s, 0, prec))
    ws = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    P = ctypes.c_void_p
    st = P(stream.cuda_stream)

    keep = prec in api.KEEP_PHI
    phi = torch.empty((l, api.phi_ld(s)) if keep else (1, 64), dtype=torch.float32, device=dev)

    def two_call_step(precision, Gd=G, Ad=A, Zd=Z, th=theta, al=alpha, evd=ev, sed=se, gd=grad):
        # what autograd runs: the estimates, then the gradient from a second
        # call; Phi kept between them where the precision supports it
        # (iqp_expval_keep_phi + iqp_expval_grad_from_phi), else recomputed
        # (iqp_expval + iqp_expval_grad)
        if keep and precision in api.KEEP_PHI:
            _lib.check(lib.iqp_expval_keep_phi(n, P(Gd.data_ptr()), m, Gd.shape[1], P(Ad.data_ptr()), l, Ad.shape[1],
                                               P(Zd.data_ptr()), s, Zd.shape[1], P(th.data_ptr()), precision,
                                               P(evd.data_ptr()), P(sed.data_ptr()), P(phi.data_ptr()), phi.shape[1],
                                               P(ws.data_ptr()), ws.numel(), st), "iqp_expval_keep_phi")
            _lib.check(lib.iqp_expval_grad_from_phi(n, P(Gd.data_ptr()), m, Gd.shape[1], P(Ad.data_ptr()), l,
                                                    Ad.shape[1], P(Zd.data_ptr()), s, Zd.shape[1], P(th.data_ptr()),
                                                    P(al.data_ptr()), None, precision, P(phi.data_ptr()),
                                                    phi.shape[1], P(gd.data_ptr()), P(ws.data_ptr()), ws.numel(),
                                                    st), "iqp_expval_grad_from_phi")
            return
        _lib.check(lib.iqp_expval(n, P(Gd.data_ptr()), m, Gd.shape[1], P(Ad.data_ptr()), l, Ad.shape[1],
                                  P(Zd.data_ptr()), s, Zd.shape[1], P(th.data_ptr()), precision, P(evd.data_ptr()),
                                  P(sed.data_ptr()), P(ws.data_ptr()), ws.numel(), st), "iqp_expval")
        _lib.check(lib.iqp_expval_grad(n, P(Gd.data_ptr()), m, Gd.shape[1], P(Ad.data_ptr()), l, Ad.shape[1],
                                       P(Zd.data_ptr()), s, Zd.shape[1], P(th.data_ptr()), P(al.data_ptr()), None,
                                       precision, P(gd.data_ptr()), P(ws.data_ptr()), ws.numel(), st),
                   "iqp_expval_grad")

    def fused_step(precision, Gd=G, Ad=A, Zd=Z, th=theta, al=alpha, evd=ev, sed=se, gd=grad):
        # one call: parities once, one phase pass for the statistics and W, the gradient contraction
        _lib.check(lib.iqp_expval_value_and_grad(n, P(Gd.data_ptr()), m, Gd.shape[1], P(Ad.data_ptr()), l,
                                                 Ad.shape[1], P(Zd.data_ptr()), s, Zd.shape[1], P(th.data_ptr()),
                                                 P(al.data_ptr()), None, precision, P(evd.data_ptr()),
                                                 P(sed.data_ptr()), P(gd.data_ptr()), P(ws.data_ptr()), ws.numel(),
                                                 st), "iqp_expval_value_and_grad")

    step = fused_step if args.step == "fused" else two_call_step

    def timed(precision, k, warm, profile=False, fn=None):
        fn = fn or (lambda: step(precision))
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if profile:
            lib.iqp_profile_reset()
            lib.iqp_profile_enable(1)
        launches0 = lib.iqp_launch_count()
        evs = []
        for _ in range(k):
            flush.zero_()  # L2 flush between steps, outside the step's events
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        launches = lib.iqp_launch_count() - launches0
        if profile:
            lib.iqp_profile_enable(0)
        ms = [a.elapsed_time(b) for a, b in evs]
        return ms, launches

    vis = [x for x in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if x.strip()]
    sampler = ClockSampler(vis[local].strip() if local < len(vis) else str(local))
    sampler.start()
    ms_list, launches = timed(prec, args.steps, args.warmup, profile=True)
    clocks = sampler.stop()
    status = lib.iqp_read_status(P(ws.data_ptr()), ws.numel(), st)
    if status != 0:
        raise SystemExit(f"device status {status}: {_lib.status_string(status)}")
    ms = max_over_ranks(statistics.mean(ms_list), dev)

    # Per-kernel live timings of the timed region (events on the launch stream).
    kt = {}
    for k, name in enumerate(_lib.KERNELS):
        tot, cnt = ctypes.c_double(0), ctypes.c_uint64(0)
        lib.iqp_profile_query(k, ctypes.byref(tot), ctypes.byref(cnt))
        if cnt.value:
            kt[name] = {"launches": int(cnt.value), "total_ms": round(tot.value, 4),
                        "avg_ms": round(tot.value / cnt.value, 4)}
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    if prec == _lib.SPLIT_BF16:
        dom = max(("phase_tc", "recompute_tc", "grad_tc"), key=lambda k: kt.get(k, {}).get("total_ms", 0.0))
        roof = split_bf16_roofline(kt, dom, l, s, m, args.steps, peaks, ms,
                                   contractions=2 if args.step == "fused" else 3)
        roof["traffic"] = measured_traffic(dom, (n, m, l, s))
        alg = tensor_algorithmic_bytes(dom, l, s, m)
        roof["algorithmic_bytes"] = alg
        roof["traffic_ratio"] = None if roof["traffic"] is None else round(roof["traffic"] / alg, 3)
    elif prec == _lib.LOWORDER_FP32:
        roof = loworder_roofline(kt, clocks, n, p.G, s, peaks)
        roof["traffic"] = None
    elif prec == _lib.SPARSE_FP32:
        nnz = nnz_parities(api, p.n, A, G)
        mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
        peak = 152 * 128 * mhz * 1e6 / 1e12
        # the fused step's one-pass kernel (k_sparse<2>) does both the phase's
        # nnz * s signed additions and the gradient's nnz * s signed terms
        adds = (2 if args.step == "fused" else 1) * nnz * s
        achieved = adds / (kt["phase_sparse"]["avg_ms"] * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "phase_sparse", "achieved": round(achieved, 2), "peak": round(peak, 1),
                "unit": "Tadd/s", "frac": round(achieved / peak, 4), "traffic": None, "adds_per_launch": adds,
                "nnz_PA": nnz, "density_PA": round(nnz / (l * m), 5),
                "peak_source": "FP32 add: 152 SMs x 128 lanes x max SM clock"}
    else:
        dom = max(("phase_fp32", "recompute_fp32", "grad_fp32"), key=lambda k: kt.get(k, {}).get("total_ms", 0.0))
        flops = 2.0 * l * s * m
        achieved = flops / (kt[dom]["avg_ms"] * 1e-3) / 1e12
        peak = 152 * 128 * 2 * (clocks or {}).get("sm_mhz", 1425.0) * 1e6 / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": round(achieved, 2), "peak": round(peak, 1),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                "flops_per_launch": flops, "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 x median SM clock"}

    # The other step form on the same workload (same timing rules).
    other_fn = (lambda: two_call_step(prec)) if args.step == "fused" else (lambda: fused_step(prec))
    lib.iqp_profile_reset()
    ms_other, _ = timed(prec, max(2, args.steps // 2), 2, profile=True, fn=other_fn)
    other = {"step": "two-call" if args.step == "fused" else "fused",
             "ms_per_step": round(max_over_ranks(statistics.mean(ms_other), dev), 3),
             "kernels": {k: v["avg_ms"] for k, v in _kernel_times(lib).items()}}

    # Plain FP32 form on the same GPU, same workload.
    fp32 = None
    if prec == _lib.SPLIT_BF16 and args.fp32_steps > 0:
        ms32, _ = timed(_lib.FP32, args.fp32_steps, 1, fn=lambda: step(_lib.FP32))
        fp32 = {"ms_per_step": round(statistics.mean(ms32), 3), "steps": args.fp32_steps}

    # End to end: host (pinned) inputs -> device, both calls, results -> host.
    hG, hA, hZ = (x.cpu().pin_memory() for x in (G, A, Z))
    hth, hal = theta.cpu().pin_memory(), alpha.cpu().pin_memory()
    hev, hse, hgr = (torch.empty(x.shape, dtype=x.dtype).pin_memory() for x in (ev, se, grad))
    dG, dA, dZ = (torch.empty_like(x) for x in (G, A, Z))
    dth, dal = torch.empty_like(theta), torch.empty_like(alpha)
    h2d = sum(x.numel() * x.element_size() for x in (hG, hA, hZ, hth, hal))
    d2h = sum(x.numel() * x.element_size() for x in (hev, hse, hgr))
    e2e_ms = []
    for it in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for d, h in ((dG, hG), (dA, hA), (dZ, hZ), (dth, hth), (dal, hal)):
            d.copy_(h, non_blocking=True)
        step(prec, dG, dA, dZ, dth, dal)  # through the same public call as the timed step
        for h, d in ((hev, ev), (hse, se), (hgr, grad)):
            h.copy_(d, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if it >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e = {"value": round(statistics.mean(e2e_ms), 3), "unit": "ms", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h)}

    line = {
        "metric": METRIC, "value": round(ms, 3), "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if prec == _lib.SPLIT_BF16 else "f32",
        "data": "synthetic (seeded splitmix64), shaped like the paper's op_expval benchmark",
        "config": {"workload": workload_name(args, p), "n": n, "m": m, "l": l, "s": s,
                   "precision": args.precision + (" (2 theta = hi + lo BF16, FP32 accumulate in TMEM, FP64 "
                                                  "reductions)" if prec == _lib.SPLIT_BF16 else ""),
                   "l2": "flushed between steps (256 MiB write, outside the step events)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "step": ("one iqp_expval_value_and_grad call (parities once, one phase pass for the statistics and W, the "
                 "gradient contraction)" if args.step == "fused" else
                 "iqp_expval then iqp_expval_grad (as autograd runs them; Phi recomputed in the second)"),
        "other_step": other,
        "roofline": roof, "parity_roofline": parity_roofline(kt, peaks, n, m, l, s, args.steps,
                                                              1 if args.step == "fused" else 2,
                                                              loworder=prec == _lib.LOWORDER_FP32),
        "kernels": kt, "gpu_launches": int(launches), "clocks": clocks, "e2e": e2e,
        "ms_steps": [round(x, 3) for x in ms_list],
    }
    if fp32 is not None:
        line["fp32_form"] = fp32
    if not args.no_rows and prec == _lib.SPLIT_BF16:
        line["rows"] = other_rows(args, lib, dev, st, timed, peaks, clocks, G, A, theta, w, n, m, l)
        line["rows"].update(workload_rows(args, lib, dev, st, timed, peaks, clocks))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        def gpu_grad_fn(alpha_np):
            al = torch.from_numpy(alpha_np).to(dev)
            g2 = torch.empty(m, dtype=torch.float64, device=dev)
            _lib.check(lib.iqp_expval_grad(n, P(G.data_ptr()), m, G.shape[1], P(A.data_ptr()), l, A.shape[1],
                                           P(Z.data_ptr()), s, Z.shape[1], P(theta.data_ptr()), P(al.data_ptr()),
                                           None, prec, P(g2.data_ptr()), P(ws.data_ptr()), ws.numel(), st),
                       "iqp_expval_grad")
            return g2.cpu().numpy()
        step(prec)
        torch.cuda.synchronize()
        line["cpu_baseline"] = cpu_baseline(p, args, ev.cpu().numpy(), se.cpu().numpy(), gpu_grad_fn)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
