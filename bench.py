"""Benchmark of the element-integration hot path on GB300.

A step is one pass of the whole hot path (geometry, Jacobians, point
operators, contraction, load vectors, stores) over one batch of synthetic
prisms already resident in HBM.  Default workload: p = 4, 100 000 jittered
prisms (the single-degree configuration), precision = the fastest path that
meets 1e-6 relative error.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload p4]
                    [--precision tc_f16x3|fp32|fp64] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun every rank integrates its own
copy of the workload (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1310_1194_gb300 import inputs  # noqa: E402

WORKLOAD_TEXT = {
    "pr1": "PR1: 4096 prisms (16x16x8 grid, 2 prisms per hex, jitter 10% h), p=1",
    "p4": "single degree: 100000 prisms (50x50x20 grid, jitter 10% h), p=4, N_sh=75, N_q=125",
    "mixed": "mixed degree: 200000 prisms (50x50x40 grid), p in 1..7 with probabilities .25/.2/.15/.15/.1/.1/.05",
    "diff": "differentiation: 20000 prisms (25x20x20), p=5, per-point coefficient fields",
    "p7": "high order: 32768 prisms (32x32x16 grid, jitter 25% h, det J > 0 certified), p=7",
    "p1m": "PR1 recipe at 1 000 000 prisms (100x100x50 grid, jitter 10% h), p=1 (supplementary, store-bound)",
    "p4sym": "symmetric single degree: the p=4 100000-prism batch with b=0, A_e stored as upper triangles",
}


def nsh(p):
    return (p + 1) * (p + 1) * (p + 2) // 2


def nq(p):
    return (p + 1) ** 3


def flops_per_element(p):
    """Algorithmic flops per element: 8 N_sh^2 N_q (contraction with the 4x4
    point operator) + 2 N_sh N_q (load vector) + 220 N_q (geometry, the
    paper's constant per point, Table 3)."""
    s, q = nsh(p), nq(p)
    return 8 * s * s * q + 2 * s * q + 220 * q


def tc_hw_flops(p, precision="tc_f16x3"):
    """Tensor-core flops issued per element by the split contraction: 3
    products x 2 x (N_sh rows, stacked in 128-row tiles) x N_pad x 4 N_q
    (N_q padded to the kernel's points per chunk: 128-byte operand rows of
    fp16 or TF32 values, 64-byte rows at p = 7)."""
    s, q = nsh(p), nq(p)
    npad = 224 if p == 6 else (s + 15) // 16 * 16
    row_values = (64 if p == 7 else 128) // (4 if precision == "tc_3xtf32" else 2)
    ppc = row_values // 4
    kpad = ((q + ppc - 1) // ppc) * ppc * 4
    return 3 * 2 * s * npad * kpad


def sf_flops_per_element(p):
    """Flops per element of the sum-factorised kernel (M = p+1 nodes per
    direction, T = (p+1)(p+2)/2 triangle functions, 21 pairs of gradient
    terms, 4 pairs of zeta factors): per pair the u sum M^3 (M + 2 M^2) and
    the v sum T^2 M (1 + 2 M), the zeta sum 4 T^2 M (M + 2 M^2), the load
    vector 2 (M^4 + M^2 T + N_sh M) and the geometry 220 N_q."""
    M, T = p + 1, (p + 1) * (p + 2) // 2
    TT = T * T
    pairs = 21 * (M ** 3 * (M + 2 * M * M) + TT * M * (1 + 2 * M))
    return pairs + 4 * TT * M * (M + 2 * M * M) + 2 * (M ** 4 + M * M * T + nsh(p) * M) + 220 * nq(p)


def kernel_flops(counts, precision):
    """Flops one step's kernels do for the per-degree counts: the sum-
    factorised kernel's own count at p >= 3 under sf_fp32, the dense
    contraction's count otherwise."""
    return sum(int(counts[d]) * (sf_flops_per_element(d) if (precision == "sf_fp32" and d >= 3)
                                 else flops_per_element(d)) for d in range(1, 8))


def fp64_pipe_ops_per_element(p):
    """FP64-pipe instructions per element of the FP32 path at p <= 2: the 21
    element-vector components (3 adds, a multiply, a conversion each), per
    vertical node 36 (the columns c1, c2: 6; n3: 6; n3.C, n3.D1, n3.D2: 9;
    the w_z products: 3; three FP32-pair splits: 12) and the 14 coefficient
    conversions."""
    return 21 * 5 + 36 * (p + 1) + 14


def bwd_flops_per_element(p):
    """Algorithmic flops of the adjoint per element: W = gA G^T (8 N_sh^2
    N_q), dL/dDt = G_q W_q (32 N_sh N_q), the load-vector adjoint (2 N_sh
    N_q) and the per-point chain to the coefficients and vertices (about
    600 flops per point)."""
    s, q = nsh(p), nq(p)
    return 8 * s * s * q + 34 * s * q + 600 * q


def adj_tc_hw_flops(p):
    """Issued tensor flops of the tensor-core adjoint per element: three
    products of M = 128-row tiles of (q, b) (ceil(4 N_q / 128) of them),
    N = N_sh padded to 16 and K = N_sh padded to 32."""
    s, q = nsh(p), nq(p)
    return 3 * 2 * ((4 * q + 127) // 128) * 128 * ((s + 15) // 16 * 16) * ((s + 31) // 32 * 32)


def quad_bwd_flops_per_element(p):
    """Algorithmic flops of the quadratic-loss adjoint per element: v_q =
    G_q u (8 N_sh N_q), the outer products (16 N_q) and the per-point chain
    (about 600 flops per point)."""
    s, q = nsh(p), nq(p)
    return 8 * s * q + 616 * q


def bytes_per_element(p, out_bytes, per_qp=False, upper=False):
    """Algorithmic HBM bytes: geometry 144 B + coefficients 112 B (per
    element) or 112 N_q B (per point) + outputs (N_sh^2 + N_sh) * s, with
    N_sh (N_sh + 1) / 2 values of A_e in the upper-triangle layout."""
    s = nsh(p)
    coef = 112 * (nq(p) if per_qp else 1)
    return 144 + coef + ((s * (s + 1) // 2 if upper else s * s) + s) * out_bytes


def measured_traffic(kernel_key, p, n_elem):
    """DRAM bytes of one launch of the dominant kernel from the committed ncu
    capture (profiles/traffic.json, per element, scaled by the elements of
    this launch), or None when the capture is of another kernel source or
    another degree."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    rec = d.get(kernel_key)
    if not rec or str(p) not in rec:
        return None
    with open(os.path.join(ROOT, rec["source"]), "rb") as fh:
        if hashlib.sha256(fh.read()).hexdigest() != rec["sha256"]:
            return None
    return rec[str(p)]["bytes_per_element"] * n_elem


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.25)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines):
        """Median SM clock, the largest max clock, and every throttle reason
        seen Active, from nvidia-smi lines in the order of FIELDS."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def cpu_sample_size(w, per_qp, target_s):
    """Elements the oracle integrates in about target_s seconds on all host
    cores (calibrated on a small prefix)."""
    n0 = 64 if (w["p"] or 7) >= 6 else 256
    rate, _, _, _, _ = cpu_oracle_run(w, n0, per_qp)
    return int(max(min(n0, len(w["geom"])), min(len(w["geom"]), rate * target_s)))


def cpu_oracle_run(w, n_sample, per_qp):
    """Oracle (FP64 C, all host cores) on the first n_sample elements:
    (elements/s, cores, elements, seconds, (A, b, status, offsets))."""
    import oracle
    n = min(n_sample, len(w["geom"]))
    sl = slice(0, n)
    degree = None if w["p"] is not None else w["degree"][:n]
    p = w["p"]
    if per_qp:
        q = nq(p)
        K, b, c, f = w["K"][: n * q], w["b"][: n * q], w["c"][: n * q], w["f"][: n * q]
    else:
        K, b, c, f = w["K"][sl], w["b"][sl], w["c"][sl], w["f"][sl]
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    out = oracle.integrate(w["geom"][sl], K, b, c, f, p=p, degree=degree, per_qp=per_qp, nthreads=cores)
    dt = time.perf_counter() - t0
    return n / dt, cores, n, dt, out


def errors_vs_oracle(A, bv, st, ref, n_s, upper_p=None):
    """Per-element relative Frobenius error of A_e (2-norm of b_e) of the
    first n_s elements of a device result against the oracle's, which uses
    the same prefix layout.  Returns max, p99 and mean of A's errors, the
    max of b's, and whether the statuses agree.  upper_p: the device result
    holds each A_e of this uniform degree as its upper triangle (mirrored
    back to the full matrix for the comparison)."""
    Ao, bo, so, (oA, ob, _) = ref
    if upper_p is not None:
        s = nsh(upper_p)
        su = s * (s + 1) // 2
        iu = np.triu_indices(s)
        rows = []
        for e0 in range(0, n_s, 2048):
            e1 = min(n_s, e0 + 2048)
            pk = A[e0 * su:e1 * su].double().cpu().numpy().reshape(-1, su)
            full = np.zeros((e1 - e0, s, s))
            full[:, iu[0], iu[1]] = pk
            full[:, iu[1], iu[0]] = pk
            rows.append(full.reshape(-1))
        A = torch_from(np.concatenate(rows))
    offs = np.asarray(oA[: n_s + 1], dtype=np.int64)
    boffs = np.asarray(ob[: n_s + 1], dtype=np.int64)
    ea = np.empty(n_s)
    eb = np.empty(n_s)
    # element chunks of about 32 M values, compared on the host in FP64
    e0 = 0
    while e0 < n_s:
        e1 = int(np.searchsorted(offs, offs[e0] + (1 << 25), side="right")) - 1
        e1 = min(max(e1, e0 + 1), n_s)
        a = A[int(offs[e0]):int(offs[e1])].double().cpu().numpy()
        r = Ao[int(offs[e0]):int(offs[e1])]
        seg = offs[e0:e1] - offs[e0]
        num = np.add.reduceat((a - r) ** 2, seg)
        den = np.add.reduceat(r * r, seg)
        ea[e0:e1] = np.sqrt(num / np.maximum(den, 1e-300))
        e0 = e1
    bg = bv[: int(boffs[n_s])].double().cpu().numpy()
    segb = boffs[:n_s]
    num = np.add.reduceat((bg - bo[: int(boffs[n_s])]) ** 2, segb)
    den = np.add.reduceat(bo[: int(boffs[n_s])] ** 2, segb)
    eb[:] = np.sqrt(num / np.maximum(den, 1e-300))
    so = np.asarray(so[:n_s])
    ok = so == 0
    return {"elements": int(n_s), "max": float(ea[ok].max()) if ok.any() else None,
            "p99": float(np.percentile(ea[ok], 99)) if ok.any() else None,
            "mean": float(ea[ok].mean()) if ok.any() else None,
            "b_max": float(eb[ok].max()) if ok.any() else None,
            "status_equal": bool(np.array_equal(st[:n_s].cpu().numpy(), so))}


def torch_from(x):
    import torch
    return torch.from_numpy(x)


def shard_workload(w, rank, world, mode):
    """The part of the job that this rank integrates.  strong: the workload
    is the whole job, split by shard.partition (contiguous ranges balanced
    by F(p)).  weak: the job is `world` copies of the workload, each copy's
    mesh translated by its index along x, split the same way, so a rank
    holds about one workload's worth of work (exactly one copy for a
    uniform degree)."""
    from paper_1310_1194_gb300 import shard
    if world == 1:
        return w
    if mode == "strong":
        return shard.shard(w, rank, world)
    n = len(w["geom"])
    deg1 = w["degree"] if w.get("degree") is not None else np.full(n, w["p"], dtype=np.int32)
    lo, hi = shard.partition(np.tile(deg1, world), world)[rank]
    idx = np.arange(lo, hi)
    copy, e = idx // n, idx % n
    out = dict(w)
    geom = w["geom"][e].copy()
    geom[:, :, 0] += copy[:, None].astype(np.float64)
    out["geom"] = np.ascontiguousarray(geom)
    out["degree"] = np.ascontiguousarray(deg1[e])
    if w.get("per_qp"):
        q = (np.asarray(deg1, dtype=np.int64) + 1) ** 3
        qo = np.concatenate([[0], np.cumsum(q)])
        rows = np.concatenate([np.arange(qo[k], qo[k + 1]) for k in e]) if len(e) else np.zeros(0, np.int64)
    else:
        rows = e
    for k in ("K", "b", "c", "f"):
        out[k] = np.ascontiguousarray(w[k][rows])
    out["start"], out["end"] = lo, hi
    return out


def roofline_of(dom, counts, precision, peaks, peak_src, live, Bts, ms_all, p, n, per_qp):
    """The roofline object of the dominant kernel `dom` (its algorithmic
    flops over its own duration, against the pipe that bounds it)."""
    F, ms = dom["F"], dom["ms"]
    counts = dom["counts"]
    precision = dom["precision"]
    hw = None
    low_p = p is not None and p <= 2 and dom["kernel"] == "forward"
    f64_peak = live.get("fp64_fma_tflops") if live else None
    f32_peak = live.get("fp32_fma_tflops") if live else None
    f64_note = "FP64 FMA, measured (csrc_peaks, best of 5)" if f64_peak else "FP64 FMA derived: 152 x 2 x 2 x clock"
    f32_note = "FP32 FMA, measured (csrc_peaks, best of 5)" if f32_peak else "FP32 FMA derived: 152 x 128 x 2 x clock"
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    if not f64_peak:
        f64_peak = 152 * 2 * 2 * sm_max * 1e6 / 1e12
    if not f32_peak:
        f32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
    if low_p and precision == "fp64":
        # the FP64 path at p <= 2: every flop in FP64
        bound, peak, unit, achieved = "alu", f64_peak, "TFLOP/s", F / (ms * 1e-3) / 1e12
        peak_note = f64_note
        hw = {"hbm_gbs": Bts / (ms * 1e-3) / 1e9, "hbm_frac": Bts / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
              "hbm_peak_gbs": peaks["hbm_gbs"]}
    elif low_p:
        # p <= 2 on the FP32 path: a few kflops per element against 0.4-0.6 KB
        # of traffic, but reading the FP64 inputs needs FP64 work, and at
        # GB300's FP64 rate (1/64 of FP32) that, not HBM, binds.  The work is
        # counted in FP64-pipe instructions per element (the element vectors:
        # 21 x (3 adds, a multiply, a conversion); per vertical node the
        # columns, n3 and its three dot products, w_z and the FP32-pair
        # splits: 36; the 14 coefficient conversions) against the measured
        # FP64 FMA instruction rate (half the FP64 flop peak)
        ops = sum(int(counts[d]) * fp64_pipe_ops_per_element(d) for d in range(1, 3))
        bound, peak, unit, achieved = "alu", f64_peak / 2, "Tinst/s", ops / (ms * 1e-3) / 1e12
        peak_note = f64_note + " / 2: FP64 pipe instructions (the FP64 input work binds before HBM)"
        hw = {"hbm_gbs": Bts / (ms * 1e-3) / 1e9, "hbm_frac": Bts / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
              "hbm_peak_gbs": peaks["hbm_gbs"], "fp64_pipe_ops_per_element": {
                  str(d): fp64_pipe_ops_per_element(d) for d in range(1, 3) if counts[d]}}
    elif precision in ("tc_f16x3", "tc_3xtf32"):
        # every algorithmic multiply-add is three tensor products (hi*hi,
        # hi*lo, lo*hi), so the peak for algorithmic flops is a third of the
        # dense peak of the operand type: fp16 (= bf16, the driver's
        # measurement) or TF32 (measured here with a library GEMM, else the
        # bf16 figure times the nominal ratio 1.1 / 2.25)
        if precision == "tc_f16x3":
            tpeak, tnote = peaks["bf16_tflops"], f"bf16/fp16 dense peak ({peak_src})"
        elif live and live.get("tf32_tensor_tflops"):
            tpeak, tnote = live["tf32_tensor_tflops"], "TF32 dense peak (measured: torch.matmul, TF32 allowed)"
        else:
            tpeak, tnote = peaks["bf16_tflops"] * 1.1 / 2.25, f"TF32: bf16 peak ({peak_src}) x nominal 1.1/2.25"
        bound, peak, unit, achieved = "tensor", tpeak / 3, "TFLOP/s", F / (ms * 1e-3) / 1e12
        peak_note = tnote + " / 3"
        if dom["kernel"].startswith("adjoint"):
            hwF = sum(int(counts[d]) * adj_tc_hw_flops(d) for d in range(3, 6))
            hw_note = ("issued tcgen05 flops of W^T: 3 products x 2 x 128-row tiles of (q, b) x N_sh pad 16 x "
                       "N_sh pad 32; the time includes the FP32 chain kernel")
        else:
            hwF = sum(int(counts[d]) * tc_hw_flops(d, precision) for d in range(3, 8))
            hw_note = "issued tcgen05 flops: 3 products x 2 x 128-row tiles x N_pad x 4 N_q"
        hw = {"tensor_tflops": hwF / (ms * 1e-3) / 1e12,
              "frac_of_tensor_peak": hwF / (ms * 1e-3) / 1e12 / tpeak,
              "note": hw_note}
    elif precision == "sf_fp32":
        # the sum-factorised kernel does its own, smaller flop count on the
        # FP32 FMA pipe; the dense contraction's count over the same time is
        # reported beside it as the equivalent rate
        Fk = kernel_flops(counts, precision)
        bound, peak, unit, achieved = "alu", f32_peak, "TFLOP/s", Fk / (ms * 1e-3) / 1e12
        peak_note = f32_note + " (sum-factorised flop count)"
        hw = {"dense_equivalent_tflops": F / (ms * 1e-3) / 1e12,
              "note": "dense contraction flops (8 N_sh^2 N_q + ...) over the same time"}
    elif precision == "fp32":
        bound, peak, unit, achieved = "alu", f32_peak, "TFLOP/s", F / (ms * 1e-3) / 1e12
        peak_note = f32_note
    else:
        bound, peak, unit, achieved = "alu", f64_peak, "TFLOP/s", F / (ms * 1e-3) / 1e12
        peak_note = f64_note
    traffic = None
    if dom["kernel"] == "forward" and p is not None and p >= 3 and precision in ("tc_f16x3", "sf_fp32"):
        traffic = measured_traffic("tc_forward_kernel" if precision == "tc_f16x3" else "sf_forward_kernel", p, n)
    r = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
         "traffic": traffic, "peak_source": peak_note, "kernel": dom["kernel"], "kernel_ms": ms,
         "step_hbm_gbs": Bts / (ms_all * 1e-3) / 1e9, "step_hbm_frac": Bts / (ms_all * 1e-3) / 1e9 / peaks["hbm_gbs"],
         "hardware": hw}
    if "fwd_ms" in dom:
        r["forward_ms"] = dom["fwd_ms"]
    if "fp32_adjoint_ms" in dom:
        r["fp32_cuda_core_adjoint_ms"] = dom["fp32_adjoint_ms"]
    if "adjoint_ms" in dom:
        r["adjoint_ms"] = dom["adjoint_ms"]
        r["adjoint"] = "quadratic loss (gA never formed)"
    return r


def run_workload(name, args, ctx, headline):
    """One workload: the timed steps of the fastest path that meets 1e-6,
    its dominant kernel's roofline, the plain FP64 GPU path on the same
    batch, and errors against the FP64 oracle on the prefix the oracle
    integrates.  The headline adds the FP32 CUDA-core path, end to end
    through the host-memory entry, and the CPU baseline."""
    import torch
    from paper_1310_1194_gb300 import api, _lib
    world, rank, dev, stream, flush, peaks, peak_src, live = (ctx[k] for k in (
        "world", "rank", "dev", "stream", "flush", "peaks", "peak_src", "live"))
    steps = args.steps if headline else max(2, min(args.steps, args.per_workload_steps))
    w0 = inputs.workload(name, n_max=(args.elements or None) if headline else None)
    upper = name == "p4sym"  # a symmetric weak form: A_e as upper triangles
    w = shard_workload(w0, rank, world, args.scaling)
    per_qp = bool(w["per_qp"])
    p = w["p"]
    n = len(w["geom"])
    # the whole job's elements (every rank's share)
    n_job = n if world == 1 else len(w0["geom"]) * (world if args.scaling == "weak" else 1)
    g = {k: torch.from_numpy(np.ascontiguousarray(w[k])).to(dev) for k in ("geom", "K", "b", "c", "f")}
    deg = None if p is not None else torch.from_numpy(np.ascontiguousarray(w["degree"])).to(dev)

    # the oracle on a prefix of this rank's batch (N = 1 only): the CPU
    # baseline, and the reference every path's error is measured against
    ref = None
    n_s = 0
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        secs = args.cpu_seconds if headline else args.per_workload_cpu_seconds
        n_s = args.cpu_sample if (args.cpu_sample and headline) else cpu_sample_size(w, per_qp, secs)
        rate, cores, n_s, dt, ref = cpu_oracle_run(w, n_s, per_qp)
        cpu = {"value": rate, "unit": "elements/s", "cores": cores, "kind": "oracle",
               "sample": f"first {n_s} elements of the workload ({dt:.1f} s on the host cores)"}

    precision = args.precision if headline else None
    if precision is None:
        # the fastest path within 1e-6 of the oracle: the FP32 kernels at
        # p <= 2, the split tensor-core kernel at p = 3, 4, the sum-factorised
        # kernel at p = 5..7, and per degree the tuner's pick for a mixed batch
        precision = "auto" if p is None else "fp32" if p <= 2 else "tc_f16x3" if p <= 4 else "sf_fp32"
    layout = api.fei_plan_offsets(deg, upper) if deg is not None else api.uniform_layout(n, p, upper)
    refs = [api.fei_reference_create(d) for d in ([p] if p is not None else range(1, 8))]
    out_dtype = torch.float64 if precision == "fp64" else torch.float32
    A = torch.empty(layout.A_total, dtype=out_dtype, device=dev)
    bv = torch.empty(layout.b_total, dtype=out_dtype, device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)

    # mixed degree: a plan (bucketing + one kernel per degree in one CUDA
    # graph), its per-degree kernel shapes tuned once before timing
    plan = None
    plan_choices = None
    if deg is not None:
        plan = api.Plan(degrees=range(1, 8), max_elem=n, precision=precision)
        plan.tune(g["geom"], g["K"], g["b"], g["c"], g["f"], degree=deg, per_qp=per_qp, layout=layout,
                  out=(A, bv, st))
        plan_choices = {f"p{d}": dict(zip(("variant", "grid_cap", "tuned_ms"), plan.choice(d)))
                        for d in range(1, 8) if (w["degree"] == d).any()}

    # differentiation: the step is the forward and the adjoint of
    # L = sum_e u_e^T A_e u_e - u_e^T b_e (gA_e = u_e u_e^T, gb_e = -u_e)
    grads = None
    if name == "diff":
        u = torch.from_numpy(inputs.loss_weights(layout.b_total, 4)).to(dev)
        if args.adjoint == "general" and headline:
            s_ = nsh(p)
            uu = u.view(n, s_)
            grads = ((uu[:, :, None] * uu[:, None, :]).reshape(-1).to(torch.float32), (-u).to(torch.float32))
        else:
            grads = (u,)
    # the general adjoint: W = gA G^T on the tensor cores (split fp16) at a
    # uniform degree 3..5, else the FP32 CUDA-core adjoint
    bwd_prec = "tc_f16x3" if (grads is not None and len(grads) == 2 and deg is None and p in (3, 4, 5)) else "fp32"

    def step(prec=precision, outs=(A, bv, st), mid=None, bprec=None):
        if plan is not None and prec == precision:
            plan.execute(g["geom"], g["K"], g["b"], g["c"], g["f"], degree=deg, per_qp=per_qp, layout=layout,
                         out=outs)
        else:
            api.fei_integrate(g["geom"], g["K"], g["b"], g["c"], g["f"], p=p, degree=deg, per_qp=per_qp,
                              precision=prec, refs=refs, layout=layout, out=outs, upper=upper)
        if grads is not None and prec == precision:
            if mid is not None:
                mid.record(stream)
            if len(grads) == 2:
                api.fei_integrate_backward(g["geom"], g["K"], g["b"], g["c"], g["f"], grads[0], grads[1], p=p,
                                           degree=deg, per_qp=per_qp, precision=bprec or bwd_prec, refs=refs,
                                           layout=layout)
            else:
                api.fei_integrate_backward_quadratic(g["geom"], g["K"], g["b"], g["c"], g["f"], grads[0], p=p,
                                                     degree=deg, per_qp=per_qp, precision="fp32", refs=refs,
                                                     layout=layout)

    # kernels of one step: bucketing + one per degree (a plan), or one
    launches_per_step = (1 + len(refs)) if deg is not None else 1
    if grads is not None:
        launches_per_step += 1
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(ctx["local"])
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    mids = [torch.cuda.Event(enable_timing=True) for _ in range(steps)] if grads is not None else None
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.nvtx.range_push(f"timed steps {name}")
    for k in range(steps):
        flush.fill_(float(k))  # evict L2 between steps (outside the events)
        evs[k][0].record(stream)
        step(mid=mids[k] if mids else None)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = sum(step_ms) / len(step_ms)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = n_job / (ms * 1e-3)

    # errors of the timed path's outputs (the last step) against the oracle
    err = errors_vs_oracle(A, bv, st, ref, n_s, p if upper else None) if ref is not None else None

    # algorithmic flops / bytes of one step
    degs = np.full(n, p) if p is not None else np.asarray(w["degree"])
    counts = np.bincount(degs, minlength=8)
    out_b = 8 if precision == "fp64" else 4
    F = sum(int(counts[d]) * flops_per_element(d) for d in range(1, 8))
    Bts = sum(int(counts[d]) * bytes_per_element(d, out_b, per_qp, upper) for d in range(1, 8))
    # the dominant kernel and its own duration (CUDA events on its stream):
    # the one kernel of a uniform forward step; the slowest degree of a
    # plan (timed per degree by the plan's tuner above); the adjoint kernel
    # of a differentiation step (events around it)
    dom = {"kernel": "forward", "ms": ms, "F": F, "precision": precision, "counts": counts}
    plan_buckets = None
    if plan is not None:
        per_deg = {d: plan.choice(d)[2] for d in range(1, 8) if counts[d]}
        d_star = max(per_deg, key=per_deg.get)
        c1 = np.zeros(8, dtype=np.int64)
        c1[d_star] = counts[d_star]
        kernel_prec = {"cuda_core": "fp64" if precision == "fp64" else "fp32",
                       "tensor_core": "tc_3xtf32" if precision == "tc_3xtf32" else "tc_f16x3",
                       "sum_factorised": "sf_fp32"}
        prec_of = {d: kernel_prec[plan.kernel(d)] for d in per_deg}
        dom = {"kernel": f"forward, p={d_star} bucket", "ms": per_deg[d_star],
               "F": int(counts[d_star]) * flops_per_element(d_star), "precision": prec_of[d_star], "counts": c1}
        # every bucket against its own roofline (its tuned time, CUDA events)
        plan_buckets = {}
        for d, tms in per_deg.items():
            cd = np.zeros(8, dtype=np.int64)
            cd[d] = counts[d]
            prec_d = prec_of[d]
            dd = {"kernel": "forward", "ms": tms, "F": int(counts[d]) * flops_per_element(d), "precision": prec_d,
                  "counts": cd}
            Bd = int(counts[d]) * bytes_per_element(d, out_b, per_qp, upper)
            rd = roofline_of(dd, cd, prec_d, peaks, peak_src, live, Bd, tms, d, int(counts[d]), per_qp)
            plan_buckets[f"p{d}"] = {"elements": int(counts[d]), "ms": tms, "kernel": plan.kernel(d),
                                     "precision": prec_d, "bound": rd["bound"], "achieved": rd["achieved"],
                                     "peak": rd["peak"], "frac": rd["frac"]}
    elif grads is not None:
        bwd_ms = statistics.median([mids[k].elapsed_time(evs[k][1]) for k in range(steps)])
        fwd_ms = statistics.median([evs[k][0].elapsed_time(mids[k]) for k in range(steps)])
        if len(grads) == 2:
            kname = ("adjoint (tensor-core W^T = G gA^T in split fp16, FP32 chain)" if bwd_prec == "tc_f16x3"
                     else "adjoint (FP32 CUDA-core contraction, FP32 chain)")
            dom = {"kernel": kname, "ms": bwd_ms, "F": n * bwd_flops_per_element(p), "precision": bwd_prec,
                   "counts": counts, "fwd_ms": fwd_ms}
            if bwd_prec == "tc_f16x3" and rank == 0:
                # the FP32 CUDA-core adjoint on the same cotangents, for comparison
                tb = []
                for k in range(min(steps, 3)):
                    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                    flush.fill_(float(k))
                    e0.record(stream)
                    step(mid=e1, bprec="fp32")
                    e2.record(stream)
                    torch.cuda.synchronize()
                    tb.append(e1.elapsed_time(e2))
                dom["fp32_adjoint_ms"] = statistics.median(tb)
        elif bwd_ms > fwd_ms:
            dom = {"kernel": "quadratic-loss adjoint (fp32 G u, fp64 chain)", "ms": bwd_ms,
                   "F": n * quad_bwd_flops_per_element(p), "precision": "fp32", "counts": counts, "fwd_ms": fwd_ms}
        else:
            dom = {"kernel": "forward", "ms": fwd_ms, "F": F, "precision": precision, "counts": counts,
                   "adjoint_ms": bwd_ms}
    roofline = roofline_of(dom, dom["counts"], dom["precision"], peaks, peak_src, live, Bts, ms, p, n, per_qp)
    if plan is not None:
        step_flops = sum(int(counts[d]) * (sf_flops_per_element(d) if prec_of[d] == "sf_fp32" else
                                           flops_per_element(d)) for d in range(1, 8) if counts[d])
    else:
        step_flops = kernel_flops(counts, precision)

    # the plain FP64 GPU path on the same batch (the comparison the metric
    # asks for), its error against the oracle, and for the headline the
    # FP32 CUDA-core path
    fp64 = None
    fp32_path = None
    if precision != "fp64" and rank == 0:
        A64 = torch.empty(layout.A_total, dtype=torch.float64, device=dev)
        b64 = torch.empty(layout.b_total, dtype=torch.float64, device=dev)
        st64 = torch.empty(n, dtype=torch.int32, device=dev)
        step("fp64", (A64, b64, st64))
        torch.cuda.synchronize()
        t64 = []
        for _ in range(args.fp64_steps if headline else 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(1.0)
            e0.record(stream)
            step("fp64", (A64, b64, st64))
            e1.record(stream)
            torch.cuda.synchronize()
            t64.append(e0.elapsed_time(e1))
        fp64 = {"elements_per_s": n / (statistics.median(t64) * 1e-3), "ms_per_step": statistics.median(t64),
                "steps": len(t64), "forward_only": grads is not None}
        if ref is not None:
            fp64["rel_err_vs_oracle"] = errors_vs_oracle(A64, b64, st64, ref, n_s, p if upper else None)
        del A64, b64, st64
        if precision in ("tc_f16x3", "tc_3xtf32") and headline:
            A32 = torch.empty(layout.A_total, dtype=torch.float32, device=dev)
            b32 = torch.empty(layout.b_total, dtype=torch.float32, device=dev)
            st32 = torch.empty(n, dtype=torch.int32, device=dev)
            step("fp32", (A32, b32, st32))
            torch.cuda.synchronize()
            t32 = []
            for _ in range(max(1, args.fp64_steps)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                flush.fill_(2.0)
                e0.record(stream)
                step("fp32", (A32, b32, st32))
                e1.record(stream)
                torch.cuda.synchronize()
                t32.append(e0.elapsed_time(e1))
            fp32_path = {"elements_per_s": n / (statistics.median(t32) * 1e-3),
                         "ms_per_step": statistics.median(t32)}
            if ref is not None:
                fp32_path["rel_err_vs_oracle"] = errors_vs_oracle(A32, b32, st32, ref, n_s, p if upper else None)
            del A32, b32, st32

    # the other paths on the same batch (time, roofline and error): the
    # other split of the tensor-core contraction for the headline (fp16 or
    # TF32 operands), and both splits for the p = 7 workload, where the
    # sum-factorised kernel is the timed path
    alts = []
    if rank == 0 and p is not None and p >= 3 and grads is None:
        if headline and precision in ("tc_f16x3", "tc_3xtf32"):
            alts = ["tc_3xtf32" if precision == "tc_f16x3" else "tc_f16x3"]
        elif name == "p7":
            alts = [x for x in ("tc_f16x3", "tc_3xtf32", "sf_fp32") if x != precision]
    other = {}
    for alt in alts:
        Aa = torch.empty(layout.A_total, dtype=torch.float32, device=dev)
        ba = torch.empty(layout.b_total, dtype=torch.float32, device=dev)
        sa = torch.empty(n, dtype=torch.int32, device=dev)
        step(alt, (Aa, ba, sa))
        torch.cuda.synchronize()
        ta = []
        for _ in range(max(2, min(steps, 5))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(3.0)
            e0.record(stream)
            step(alt, (Aa, ba, sa))
            e1.record(stream)
            torch.cuda.synchronize()
            ta.append(e0.elapsed_time(e1))
        ma = statistics.median(ta)
        da = {"kernel": "forward", "ms": ma, "F": F, "precision": alt, "counts": counts}
        other[alt] = {"precision": alt, "elements_per_s": n / (ma * 1e-3), "ms_per_step": ma,
                      "roofline": roofline_of(da, counts, alt, peaks, peak_src, live, Bts, ma, p, n, per_qp)}
        if ref is not None:
            other[alt]["rel_err_vs_oracle"] = errors_vs_oracle(Aa, ba, sa, ref, n_s, p if upper else None)
        del Aa, ba, sa
    alt_tc = other.get("tc_3xtf32" if precision == "tc_f16x3" else "tc_f16x3") if headline else None

    # end to end through the public API with host buffers
    e2e = None
    if (headline or upper) and not args.no_e2e:
        e2e = end_to_end(args, ctx, w, g, deg, p, per_qp, layout, refs, precision, out_dtype, grads, step, A, bv,
                         n_job, upper)

    assembly = None
    if headline and args.assemble and rank == 0 and world == 1:
        assembly = assembly_measure(api, w, [g[k] for k in ("geom", "K", "b", "c", "f")], deg, refs, precision,
                                    flush, max(3, min(steps, 10)))
        assembly["assemble_hbm_frac"] = assembly["assemble_gbs"] / peaks["hbm_gbs"]

    res = {"workload": WORKLOAD_TEXT[name], "elements": n_job, "elements_per_s": value, "ms_per_step": ms,
           "steps": steps, "precision": precision,
           # flops the timed kernels do: the dense contraction's count, or
           # for the sum-factorised degrees that kernel's own (smaller)
           # count; the dense count over the same time beside it
           "gflops_algorithmic": step_flops / (ms * 1e-3) / 1e9 * (n_job / n),
           "gflops_dense_equivalent": F / (ms * 1e-3) / 1e9 * (n_job / n),
           "roofline": roofline, "rel_err_vs_oracle": err, "fp64_path": fp64, "clocks": clk,
           "launches_per_step": launches_per_step}
    if fp64 is not None:
        res["speedup_vs_fp64_path"] = fp64["ms_per_step"] / ms if not fp64["forward_only"] else None
    if fp32_path is not None:
        res["fp32_path"] = fp32_path
    if alt_tc is not None:
        res["other_tc_split"] = alt_tc
    if other and not headline:
        res["other_paths"] = other
    if plan_choices is not None:
        res["plan"] = plan_choices
        res["plan_buckets"] = plan_buckets
    if cpu is not None:
        res["cpu_baseline"] = cpu
    if e2e is not None:
        res["e2e"] = e2e
    if assembly is not None:
        res["assembly"] = assembly
    del A, bv, st, g, plan
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return res


def end_to_end(args, ctx, w, g, deg, p, per_qp, layout, refs, precision, out_dtype, grads, step, A, bv, n_job,
               upper=False):
    """The same workload through the library's public entry with host
    buffers: pinned inputs, the uploads and downloads inside the timed
    region (fei_integrate_host for a forward batch; copy in, forward +
    adjoint, copy back for the differentiation step)."""
    import torch
    from paper_1310_1194_gb300 import api
    n = len(w["geom"])
    hin = {k: torch.from_numpy(np.ascontiguousarray(w[k])).pin_memory() for k in ("geom", "K", "b", "c", "f")}
    hA = torch.empty(layout.A_total, dtype=out_dtype).pin_memory()
    hb = torch.empty(layout.b_total, dtype=out_dtype).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in hin.values())
    d2h = hA.numel() * hA.element_size() + hb.numel() * hb.element_size()
    e2e_steps = max(2, min(args.steps, 5))
    pipe = None
    hdeg = None
    hst = None
    if grads is None:
        pipe = api.Pipeline(precision=precision, refs=refs)
        hdeg = (torch.from_numpy(np.ascontiguousarray(w["degree"])).to(torch.int32).pin_memory()
                if deg is not None else None)
        hst = torch.empty(n, dtype=torch.int32).pin_memory()
        d2h += hst.numel() * 4
        if hdeg is not None:
            h2d += hdeg.numel() * 4

    def e2e_step():
        if pipe is not None:
            pipe.integrate_host(hin["geom"], hin["K"], hin["b"], hin["c"], hin["f"], p=p, degree=hdeg,
                                per_qp=per_qp, out=(hA, hb, hst), upper=upper)
            return
        for k in hin:
            g[k].copy_(hin[k], non_blocking=True)
        step()
        hA.copy_(A, non_blocking=True)
        hb.copy_(bv, non_blocking=True)

    e2e_step()  # untimed: first-use allocations
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("end-to-end steps")
    e2e_ms = []
    for _ in range(e2e_steps):
        if ctx["world"] > 1:
            torch.distributed.barrier()
        t1 = time.perf_counter()
        e2e_step()
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t1) * 1e3)
    torch.cuda.nvtx.range_pop()
    # the median step: the host link is shared with the machine's other
    # tenants, and a burst of their traffic can slow single steps
    dt = statistics.median(e2e_ms) * 1e-3
    if ctx["world"] > 1:
        t = torch.tensor([dt], device=ctx["dev"])
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        dt = float(t.item())
    return {"value": n_job / dt, "unit": "elements/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": dt * 1e3, "step_ms": [round(x, 3) for x in e2e_ms],
            "pipeline": (f"fei_integrate_host: {pipe.n_chunks} chunks of <= {pipe.slot_bytes >> 20} MiB of A_e "
                         "through two device slots, downloads overlapped with integration")
            if pipe is not None else "copy in, forward + adjoint, copy back"}


def run_reference(args, world, rank):
    """Reference arm: the FP64 oracle on the host cores, on a bounded sample
    of the same workload per step."""
    if rank != 0:
        return
    w = inputs.workload(args.workload)
    per_qp = bool(w["per_qp"])
    n_sample = args.cpu_sample or cpu_sample_size(w, per_qp, max(1.0, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_oracle_run(w, max(64, n_sample // 8), per_qp)
    rates, times = [], []
    cores = None
    for _ in range(args.steps):
        r, cores, n, dt, _ = cpu_oracle_run(w, n_sample, per_qp)
        rates.append(r)
        times.append(dt)
    value = statistics.median(rates)
    line = {
        "impl": "reference", "metric": metric_name(args), "value": value, "unit": "elements/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": True, "scaling": args.scaling,
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload], "precision": "fp64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": "elements/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {n_sample} elements of the workload per step"},
        "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


METRIC = "elements/s & GFLOP/s per degree p vs plain FP64 GPU path at rel err ≤1e-6"


def metric_name(args):
    # the workload is named in config.workload; GFLOP/s is in
    # config.gflops_algorithmic and the FP64 GPU path in fp64_path
    return METRIC


def assembly_measure(api, w, g, deg, refs, precision, flush, steps):
    """Assembly of the workload into CSR with the vertex-sharing DOF map:
    host build time, the fused integrate-and-assemble step, and the
    assembly of precomputed element matrices with its algorithmic bytes."""
    import torch
    t0 = time.perf_counter()
    l2g, nd = inputs.dof_map(w)
    t1 = time.perf_counter()
    asm = api.Assembly(l2g, nd, p=w["p"], degree=w["degree"] if w["p"] is None else None)
    t2 = time.perf_counter()
    per_qp = bool(w["per_qp"])
    vt = torch.float64 if precision == "fp64" else torch.float32
    vsize = 8 if precision == "fp64" else 4
    values = torch.empty(asm.nnz, dtype=vt, device="cuda")
    rhs = torch.empty(asm.n_dof, dtype=vt, device="cuda")
    st = torch.empty(len(w["degree"]), dtype=torch.int32, device="cuda")
    A, bv, st3, layout = api.fei_integrate(*g, p=w["p"], degree=deg, per_qp=per_qp, precision=precision,
                                           refs=refs)
    values2 = torch.empty_like(values)
    rhs2 = torch.empty_like(rhs)

    def fused():
        asm.integrate_assemble(*g, precision=precision, per_qp=per_qp, degree=deg, refs=refs, out=(values, rhs, st))

    def standalone():
        asm.assemble(A, bv, precision=precision, out=(values2, rhs2))

    def integrate():
        api.fei_integrate(*g, p=w["p"], degree=deg, per_qp=per_qp, precision=precision, refs=refs, layout=layout,
                          out=(A, bv, st3))

    def timed(fn):
        for _ in range(2):
            fn()
        ts = []
        for k in range(steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    fused_ms = timed(fused)
    integrate_ms = timed(integrate)
    asm_ms = timed(standalone)
    torch.cuda.synchronize()
    # algorithmic bytes of the standalone assembly: what any assembly must
    # move, the element matrices and vectors read once and the CSR values and
    # right-hand side written once
    bytes_asm = (int(A.numel()) + int(bv.numel()) + asm.nnz + asm.n_dof) * vsize
    return {
        "dof_map": "vertex-sharing: 6 local functions on the prism's mesh vertices, the rest private (synthetic)",
        "n_dof": asm.n_dof, "nnz": asm.nnz, "colours": asm.n_colours, "chunks": asm.n_chunks,
        "host_build_s": round(t2 - t1, 3), "dof_map_s": round(t1 - t0, 3),
        "fused_ms": fused_ms, "fused_elements_per_s": len(w["degree"]) / (fused_ms * 1e-3),
        "integrate_ms": integrate_ms, "assemble_ms": asm_ms, "unfused_ms": integrate_ms + asm_ms,
        "assemble_bytes": bytes_asm, "assemble_gbs": bytes_asm / (asm_ms * 1e-3) / 1e9,
        "fused_equals_unfused": bool(torch.equal(values, values2) and torch.equal(rhs, rhs2)),
    }


PER_WORKLOAD_ORDER = ("pr1", "p1m", "p4", "p4sym", "mixed", "diff", "p7")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="p4", choices=sorted(WORKLOAD_TEXT))
    ap.add_argument("--precision", default=None)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="N > 1: weak = N translated copies of the workload, strong = the workload itself; either "
                         "way the job is split into contiguous element ranges balanced by F(p) (shard.partition)")
    ap.add_argument("--cpu-sample", type=int, default=0, help="elements; 0 = about --cpu-seconds of work")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-per-workload", action="store_true",
                    help="skip the other workloads (by default every workload is measured after the headline, "
                         "at N = 1)")
    ap.add_argument("--per-workload-steps", type=int, default=5)
    ap.add_argument("--per-workload-cpu-seconds", type=float, default=4.0)
    ap.add_argument("--adjoint", default="quadratic", choices=["quadratic", "general"],
                    help="differentiation workload: the adjoint of the quadratic loss (gA never formed) or the "
                         "general adjoint given gA = u u^T, gb = -u")
    ap.add_argument("--assemble", action="store_true",
                    help="also measure colour-by-colour assembly into CSR (vertex-sharing DOF map): the fused "
                         "integrate-and-assemble step and the assembly of given element matrices")
    ap.add_argument("--elements", type=int, default=0,
                    help="integrate only the first N elements of the workload (small profiling cases); "
                         "0 = the whole workload")
    args = ap.parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
        return

    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    from paper_1310_1194_gb300 import peaks as peak_probe

    dev = torch.device("cuda", local)
    # a non-default stream for everything (a plan captures its launches into
    # a CUDA graph, which the legacy default stream does not allow)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    peaks, peak_src = load_peaks()
    try:
        live = peak_probe.measure()
    except Exception as exc:  # the probe is a measurement aid: report, derive instead
        live = {"error": str(exc)}
    # 1 GiB > 8 x L2: written between steps, it evicts the L2 and keeps the
    # device busy while the host enqueues the next step, so that the events
    # around a step time its kernels, not the host's launch path
    flush = torch.empty(1024 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ctx = {"world": world, "rank": rank, "local": local, "dev": dev, "stream": stream, "flush": flush,
           "peaks": peaks, "peak_src": peak_src, "live": live if "error" not in live else None}

    head = run_workload(args.workload, args, ctx, headline=True)
    per = None
    if rank == 0 and world == 1 and not args.no_per_workload and not args.elements:
        per = {}
        for name in PER_WORKLOAD_ORDER:
            if name == args.workload:
                continue
            try:
                per[name] = run_workload(name, args, ctx, headline=False)
            except Exception as exc:  # one workload's failure must not hide the headline
                per[name] = {"error": f"{type(exc).__name__}: {exc}"}
                torch.cuda.synchronize()
                torch.cuda.empty_cache()

    if rank == 0:
        precision = head["precision"]
        err = head["rel_err_vs_oracle"]
        line = {
            "metric": metric_name(args), "value": head["elements_per_s"], "unit": "elements/s", "n_gpus": world,
            "steps": head["steps"], "warmup": max(3, args.warmup), "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": args.scaling, "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "tc_f16x3": "f16x3->f32", "tc_3xtf32": "tf32x3->f32",
                      "sf_fp32": "f32", "auto": "f32 (per degree: f32, f16x3->f32 or sum-factorised f32)"}[precision],
            "data": "synthetic",
            "config": {"workload": head["workload"], "precision": precision, "elements": head["elements"],
                       "l2": "1 GiB buffer written between timed steps (outside the events); "
                             "each step also writes its outputs (> L2)",
                       "gflops_algorithmic": head["gflops_algorithmic"],
                       "rel_err_vs_oracle_max": err["max"] if err else None,
                       "rel_err_vs_oracle_elements": err["elements"] if err else None,
                       "sharding": (f"{args.scaling}: contiguous element ranges balanced by F(p) "
                                    "(shard.partition), no data-path collective") if world > 1 else None},
            "roofline": head["roofline"], "cpu_baseline": head.get("cpu_baseline"), "e2e": head.get("e2e"),
            "gpu_launches": head["launches_per_step"] * head["steps"], "clocks": head["clocks"],
            "rel_err_vs_oracle": err,
            "fp64_path": head["fp64_path"], "fp32_path": head.get("fp32_path"),
            "other_tc_split": head.get("other_tc_split"),
            "speedup_vs_fp64_path": head.get("speedup_vs_fp64_path"),
            "plan": head.get("plan"), "plan_buckets": head.get("plan_buckets"),
            "peaks_measured": live,
        }
        if "assembly" in head:
            line["assembly"] = head["assembly"]
        if per is not None:
            line["per_workload"] = per
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
