#!/usr/bin/env python
"""Throughput of one forward + gradient evaluation (fwd+grad slice-steps/s) on a GB300.

Workload (default): transmon (4 levels) x cavity (10 levels), d = 40, N = 2000 slices, dt = 1 ns,
two transmon drives, |g,0> -> |g,1> state transfer with a forbidden-level penalty at every slice,
FP32 products, sqrt(N) checkpointing.  A "step" is one full evaluation: norm bound and (p, n),
all slice exponentials, the forward propagation with per-slice costs, the backward costate
sweep with recomputation from checkpoints, the exact adjoint of every truncated exponential
and the gradient reduction.  Metric: N x trajectories / seconds per evaluation.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank evaluates its own replica (the path has no data exchange); the
value is the sum over ranks of slice-steps divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+grad slice-steps/s"
UNIT = "slice-steps/s"
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, averaged over the launches
# of one evaluation) measured by ncu, keyed by (workload, precision, kernel, wave slices)
MEASURED_TRAFFIC = {
    # DRAM bytes per slice of the dominant kernel, keyed (workload, precision, kernel, Taylor scheme):
    # the Paterson-Stockmeyer split exponential (k_expm_fwd_ps), one full ncu capture of a 1125-slice
    # launch, 163,072 bytes read + 83,686,144 written; reported per launch as bytes per slice times
    # the launch's average slices
    ("transmon_cavity_d40", "fp32", "expm_fwd", 1): (163072.0 + 83686144.0) / 1125,
}
# executed side of the same kernel from that capture: FMA pipe and issue activity, % of peak over
# active cycles
MEASURED_PIPES = {
    ("transmon_cavity_d40", "fp32", "expm_fwd", 1): {"fma_pipe_pct": 52.0, "issue_active_pct": 69.5},
}
# FP32 FMA peak from unit counts (context only; the roofline uses the measured peak):
# SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (the maximum SM clock)
def derived_fp32_peak_tflops(sms):
    return sms * 128 * 2 * 2.07e9 / 1e12


L2_FLUSH_BYTES = 256 << 20


def measured_peaks(device):
    """Denominators of the roofline fractions: FP32 and FP64 FMA throughput measured on this
    device by the library's FMA-chain kernel (qoc_measure_fma_peak), the SM count read from the
    device, and the BF16 tensor and HBM peaks of MEASURED_PEAKS.json (copy and cuBLAS GEMM
    measured on the GB300s) when that file is present."""
    from paper_1612_04929_gb300 import qoc_measure_fma_peak
    fp32, sms = qoc_measure_fma_peak(device, fp64=False)
    fp64, _ = qoc_measure_fma_peak(device, fp64=True)
    peaks = {"fp32_tflops": fp32, "fp64_tflops": fp64, "sms": sms,
             "fp32_derived_tflops": derived_fp32_peak_tflops(sms),
             "fp_source": "measured: qoc_measure_fma_peak (independent FMA chains on every SM, best of 3 "
                          "CUDA-event timings)"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            mp = json.load(open(path))
            peaks.update({"bf16_tflops": mp.get("bf16_tflops"), "bf16_tflops_sustained": mp.get("bf16_tflops_sustained"),
                          "hbm_gbs": mp.get("hbm_gbs"), "tensor_source": "MEASURED_PEAKS.json (measured)"})
        except (OSError, ValueError):
            pass
    if peaks.get("bf16_tflops") is None:
        peaks.update({"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0,
                      "tensor_source": "fallback (no MEASURED_PEAKS.json)"})
    return peaks


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="transmon_cavity")
    ap.add_argument("--precision", default=None)
    ap.add_argument("--ckpt-stride", type=int, default=0)
    ap.add_argument("--N", type=int, default=0, help="override the slice count (profiling runs)")
    ap.add_argument("--count", type=int, default=128, help="problems of the batched sweep (--workload batch)")
    ap.add_argument("--ensemble", type=int, default=32, help="members per problem (--workload batch)")
    ap.add_argument("--profile-batch", action="store_true", help="per-kernel event times (--workload batch)")
    ap.add_argument("--cpu-sample", type=int, default=0, help="slices in the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true", help="skip timing the plain FP64 GPU form")
    ap.add_argument("--no-per-config", action="store_true",
                    help="skip the per-config lines (the other four configurations, a few seconds each)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="take the planner's choices instead of timing the candidates (qoc_options.autotune) "
                         "during the warm-up")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every kernel of each evaluation instead of replaying the evaluation from a "
                         "captured CUDA graph (per-slice path; the batched path always launches directly)")
    ap.add_argument("--propagation", choices=["unitary", "state"], default="unitary",
                    help="form U_j (unitary) or apply the series to the propagated columns (state mode)")
    ap.add_argument("--exponential", choices=["taylor", "chebyshev"], default="taylor",
                    help="slice exponential: Taylor with scaling and squaring, or Chebyshev (state mode)")
    ap.add_argument("--members", type=int, default=1, help="detuning-ensemble members (cat_state workload)")
    ap.add_argument("--taylor-scheme", choices=["auto", "horner"], default="auto",
                    help="evaluation of the Taylor polynomial (auto: Paterson-Stockmeyer where built)")
    ap.add_argument("--gradient", choices=["exact", "first_order"], default="exact",
                    help="exact derivative of the truncated series, or the paper's first-order Eq. 11")
    args = ap.parse_args()
    args.graph = not args.no_graph
    return args


def make_problem(name, N=0, members=1):
    import synthetic as sy
    kw = {"N": N} if N else {}
    if members > 1:
        kw["ensemble"] = members
    return sy.WORKLOADS[name](**kw)


def config_of(prob, precision, stride, extra=None):
    cfg = {"workload": prob.name, "d": prob.d, "N": prob.N, "M": prob.M, "S": prob.S, "E": prob.E,
           "precision": precision, "ckpt_stride": stride,
           "l2": "flushed before every timed step (256 MiB write outside the step's events)"}
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = sorted(float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit())
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------ oracle (CPU) timing
def oracle_sample_time(workload, nslices, repeats=1, ref_slices=0, exact=True, maker=None, min_seconds=0.0,
                       threads=1):
    """Times the CPU FP64 oracle on the first `nslices` slices of the workload in a child
    process with `threads` BLAS threads (0: the library's default, all host cores): at least
    `repeats` evaluations, and more until `min_seconds` of timed work.  With ref_slices > 0 the
    child also evaluates the oracle once on the first ref_slices slices (untimed) and returns its
    cost and gradient, the reference for the GPU result's error.  `maker` is an expression in n
    that builds the problem (default: the named workload with N = n).  Returns (seconds per
    evaluation, slices, reference, evaluations, threads that gained CPU time while timing)."""
    code = f"""
import json, os, sys, time
sys.path.insert(0, {ROOT!r})
import synthetic as sy
from oracle import qoc_oracle as orc
def ticks():
    out = {{}}
    try:
        for tid in os.listdir("/proc/self/task"):
            with open("/proc/self/task/%s/stat" % tid) as f:
                fl = f.read().rsplit(")", 1)[1].split()
            out[tid] = int(fl[11]) + int(fl[12])
    except (OSError, ValueError, IndexError):
        return None
    return out
make = (lambda n: {maker}) if {maker!r} else (lambda n: sy.WORKLOADS[{workload!r}](N=n))
p = make({nslices})
orc.cost_and_grad(p, p.u)
ts = []
t0k = ticks()
while len(ts) < {repeats} or (sum(ts) < {min_seconds} and len(ts) < 1000):
    t0 = time.perf_counter(); orc.cost_and_grad(p, p.u); ts.append(time.perf_counter() - t0)
t1k = ticks()
busy = None if t0k is None or t1k is None else sum(1 for k, v in t1k.items() if v > t0k.get(k, 0))
ref = None
if {ref_slices} > 0:
    q = make({ref_slices})
    c, g, _ = orc.cost_and_grad(q, q.u, exact={exact!r})
    ref = {{"N": {ref_slices}, "cost": float(c), "grad": [float(x) for x in g.ravel()]}}
print(json.dumps({{"t": sum(ts) / len(ts), "n": len(ts), "ref": ref, "busy": busy}}))
"""
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if threads > 0:
            env[var] = str(threads)
        else:
            env.pop(var, None)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr)
    res = json.loads(r.stdout.strip().splitlines()[-1])
    return float(res["t"]), nslices, res["ref"], int(res["n"]), res.get("busy")


def thread_cpu_ticks():
    """{thread id: utime + stime clock ticks} of this process's threads (Linux /proc), or None."""
    try:
        out = {}
        for tid in os.listdir("/proc/self/task"):
            with open(f"/proc/self/task/{tid}/stat") as f:
                fields = f.read().rsplit(")", 1)[1].split()
            out[tid] = int(fields[11]) + int(fields[12])   # utime, stime (stat fields 14, 15)
        return out
    except (OSError, ValueError, IndexError):
        return None


def busy_threads(before, after):
    """Threads that accumulated CPU time between two thread_cpu_ticks() snapshots."""
    if before is None or after is None:
        return None
    return sum(1 for tid, t in after.items() if t > before.get(tid, 0))


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    prob = make_problem(args.workload)
    nsl = args.cpu_sample or max(20, prob.N // 20)
    import synthetic as sy
    from oracle import qoc_oracle as orc
    sample = sy.WORKLOADS[args.workload](N=nsl)
    for _ in range(args.warmup):
        orc.cost_and_grad(sample, sample.u)
    ts = []
    ticks0 = thread_cpu_ticks()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        orc.cost_and_grad(sample, sample.u)
        ts.append(time.perf_counter() - t0)
    used = busy_threads(ticks0, thread_cpu_ticks())
    t = sum(ts) / len(ts)
    value = nsl * sample.E / t
    desc = (f"CPU FP64 oracle (eigendecomposition exponentials, explicit adjoint) on the first {nsl} of "
            f"{prob.N} slices, steps={args.steps}, numpy BLAS default threads; cores = threads of this "
            f"process that gained CPU time in the timed steps ({os.cpu_count()} host cores)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(prob, "fp64-oracle", 0, {"sample_slices": nsl,
                                                          "l2": "not applicable (host CPU timing)"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def ps_top(p):
    """Top block of the Paterson-Stockmeyer form (blocks of three Taylor terms)."""
    return p // 3 - 1 if (p % 3 == 0 and p >= 3) else p // 3


def expm_products(p, n, scheme=0):
    """Complex d x d products of one slice exponential: Horner p - 1 steps (scheme 0), or
    Paterson-Stockmeyer X^2, X^3 and one chain product per block below the top (scheme 1); then
    n squarings."""
    if scheme == 1:
        return (p >= 2) + (p >= 3) + ps_top(p) + n
    return p - 1 + n


def expm_flops_per_slice(d, p, n, scheme=0):
    """Algorithmic flops of one slice exponential at 8 d^3 real flops per complex product."""
    return expm_products(p, n, scheme) * 8.0 * d ** 3


def adj_flops_per_slice(form, d, p, n, S, scheme=0):
    """Algorithmic flops of one slice's adjoint.  Horner (scheme 0): reverse mode 2 products per
    forward product plus Ubar = G Psi^dag; block recursion 3; low-rank reverse mode (cotangent as
    d x r factors, r = 2^n S): 2 d x d by d x r products per squaring level (r doubling from S), 3
    per Horner step and one final rank-r update.  Paterson-Stockmeyer (scheme 1): reverse mode
    2 per squaring and chain product plus the four power products (two when p = 2); low-rank:
    the same squaring levels, 3 d x d by d x r per chain product, the rank-r updates of the top
    block and of the X and X^2 cotangents, and the dense power products."""
    r = S << n
    if scheme == 1 and form in (0, 3):
        powers = 2 * (p >= 3) + 2 * (p >= 2)
        qt = ps_top(p)
        if form == 0:
            return 8.0 * d ** 3 * (2 * n + 2 * qt + powers) + 8.0 * d * d * S
        updates = 2 + (1 if (p % 3 == 0 and p >= 3) else 0)
        return 8.0 * d * d * (2 * S * ((1 << n) - 1) + 3 * qt * r + updates * r) + 8.0 * d ** 3 * powers
    if form == 3:
        return 8.0 * d * d * (2 * S * ((1 << n) - 1) + 3 * (p - 1) * r + r)
    k = 2 if form == 0 else 3
    return k * expm_flops_per_slice(d, p, n) + 8.0 * d * d * S


def slowest_rank_ms(ms, world, device):
    """The job's time per step: the largest of the ranks' times (every rank must call this)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    tt = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(units_per_rank, world, t_max_ms):
    """Whole-job throughput of `world` replicas (weak scaling): every rank's units over the slowest
    rank's time."""
    return units_per_rank * world / (t_max_ms / 1e3)


def roofline_of(prob, precision, info, prof, K, peaks, traffic_key=None):
    """The dominant exponential kernel of one evaluation: its algorithmic flops (8 d^3 per
    complex product) over its summed event time, against the measured peak of the arithmetic
    it runs on (FP32 or FP64 FMA lanes; BF16 tensor cores for the exact-accumulation tensor-core
    products, whose executed MMA flops are reported beside)."""
    d, p, n = prob.d, info["p"], info["n"]
    if info["kernel_path"] == 2:
        return state_roofline(prob, precision, info, prof, K, peaks)
    scheme = info.get("taylor_scheme", 0)
    per_slice = {"expm_fwd": expm_flops_per_slice(d, p, n, scheme),
                 "expm_fwd (recompute)": expm_flops_per_slice(d, p, n, scheme),
                 "expm_adj": adj_flops_per_slice(info.get("adjoint_form", 1), d, p, n, prob.S, scheme)}
    if info.get("adjoint_form") == 2:   # first-order gradient: no adjoint exponential
        per_slice.pop("expm_adj")
    cands = {k: v for k, v in prof.items() if k in per_slice}
    if not cands:
        return None
    top_name, (top_launches, top_ms) = max(cands.items(), key=lambda kv: kv[1][1])
    N_w = info["wave_slices"]
    last = prob.N - (info["n_waves"] - 1) * N_w
    slices = prob.N if top_name != "expm_fwd (recompute)" else prob.N - last
    flops = per_slice[top_name] * slices * prob.E * K
    achieved = flops / (top_ms / 1e3) / 1e12
    tensor = precision == "bf16" and top_name == "expm_adj" and info["kernel_path"] == 1
    if tensor:
        peak, bound, src = peaks["bf16_tflops"], "tensor", peaks["tensor_source"] + ", BF16 burst"
    elif precision == "fp64":
        peak, bound, src = peaks["fp64_tflops"], "alu", peaks["fp_source"] + ", FP64"
    else:
        peak, bound, src = peaks["fp32_tflops"], "alu", peaks["fp_source"] + ", FP32"
    # the counters belong to one kernel of one configuration: reported only when that kernel dominates
    per_slice_bytes = MEASURED_TRAFFIC.get(traffic_key) if traffic_key and traffic_key[2] == top_name else None
    traffic = per_slice_bytes * slices * prob.E * K / top_launches if per_slice_bytes else None
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": top_name, "launches": top_launches, "avg_launch_ms": top_ms / top_launches,
            "peak_source": src + " (of measured)",
            "traffic_source": ("dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of this kernel at "
                               "this workload, per slice, times this run's average slices per launch") if traffic else None}
    if tensor:
        roof["executed_mma_tflops"] = achieved * OZ_MMA_PER_COMPLEX_PRODUCT / 4.0
        roof["note"] = ("algorithmic flops count 8 d^3 per complex product; the exact-accumulation tensor-core "
                        "products issue %d real BF16 GEMMs of d^3 per complex product" % OZ_MMA_PER_COMPLEX_PRODUCT)
    elif precision != "fp64" and top_name.startswith("expm_fwd") and info["kernel_path"] == 0:
        roof["note"] = ("algorithmic flops (8 d^3 per complex product); the FP32 form's grid-split products "
                        "execute 12 FMAs per complex multiply-add (3.25 per algorithmic one), so the split "
                        "exponential's fraction is bounded near 0.3 by construction")
    return roof


def state_matvecs_per_slice(info):
    """Matrix-vector products per slice application in state mode: p 2^n (Taylor, Horner) or the
    Chebyshev degree K (reported as p with n = 0)."""
    return info["p"] * (1 << info["n"])


def state_roofline(prob, precision, info, prof, K, peaks):
    """State mode: the dominant kernel is one of the serial chains (forward or costate), one CTA per
    (panel, member); its algorithmic flops are 8 d^2 S per matrix-vector product (complex), one
    product per Horner step or Chebyshev term.  The peak is the FP32 (FP64) FMA peak of the whole
    GPU although the chain runs on one SM per (panel, member): the fraction shows how far a single
    trajectory is from the GPU's throughput."""
    cands = {k: v for k, v in prof.items() if k.startswith("state_chain")}
    if not cands:
        return None
    top_name, (top_launches, top_ms) = max(cands.items(), key=lambda kv: kv[1][1])
    flops = prob.N * prob.E * state_matvecs_per_slice(info) * 8.0 * prob.d ** 2 * prob.S * K
    achieved = flops / (top_ms / 1e3) / 1e12
    peak = peaks["fp64_tflops"] if precision == "fp64" else peaks["fp32_tflops"]
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": top_name, "launches": top_launches, "avg_launch_ms": top_ms / top_launches,
            "peak_source": peaks["fp_source"] + " (of measured)",
            "note": "serial chain: one CTA per (column panel, member), so at most E * panels SMs are busy"}


# real BF16 GEMMs of d^3 per complex product in the exact-accumulation tensor-core form: 10 slice
# pairs x 4 real products
OZ_MMA_PER_COMPLEX_PRODUCT = 40


def time_device_evals(ctx, u, grad, out, K, warmup, flush, stream):
    """K evaluations after `warmup`, each bracketed by CUDA events on the evaluation's stream
    with the L2 flushed before it (outside the events); returns the mean ms."""
    import torch
    for _ in range(max(warmup, 1)):
        ctx.evaluate_device(u.data_ptr(), grad.data_ptr(), out.data_ptr())
    ctx.sync()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    torch.cuda.synchronize()
    for k in range(K):
        flush.zero_()
        starts[k].record(stream)
        ctx.evaluate_device(u.data_ptr(), grad.data_ptr(), out.data_ptr())
        ends[k].record(stream)
    torch.cuda.synchronize()
    ctx.sync()
    return sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / K


def truncated(prob, n):
    """The same system, targets and controls restricted to the first n slices."""
    import dataclasses
    path = None if prob.psiT_path is None else prob.psiT_path[:n]
    return dataclasses.replace(prob, N=n, u=prob.u[:, :n].copy(), psiT_path=path)


def oracle_reference(q, threads=0):
    """Cost and gradient of problem q by the CPU FP64 oracle, in a child process with `threads`
    BLAS threads (0: the library default)."""
    import pickle
    import tempfile
    with tempfile.NamedTemporaryFile(suffix=".pkl", delete=False) as f:
        pickle.dump(q, f)
        path = f.name
    code = f"""
import json, pickle, sys
sys.path.insert(0, {ROOT!r})
from oracle import qoc_oracle as orc
q = pickle.load(open({path!r}, "rb"))
c, g, _ = orc.cost_and_grad(q, q.u)
print(json.dumps({{"cost": float(c), "grad": [float(x) for x in g.ravel()]}}))
"""
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if threads > 0:
            env[var] = str(threads)
        else:
            env.pop(var, None)
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
        if r.returncode != 0:
            raise RuntimeError(r.stderr[-500:])
        return json.loads(r.stdout.strip().splitlines()[-1])
    finally:
        os.unlink(path)


def gpu_error_vs_oracle(prob, precision, stream, ref_slices, threads=0, form=None):
    """Relative cost and gradient error of the GPU form against the CPU FP64 oracle on the first
    ref_slices slices of the problem (the whole problem when ref_slices >= N)."""
    import numpy as np
    from paper_1612_04929_gb300 import Context
    q = prob if ref_slices >= prob.N else truncated(prob, ref_slices)
    ref = oracle_reference(q, threads)
    with Context(precision, device=0, stream=stream.cuda_stream, **(form or {})) as cq:
        cq.set_problem(q)
        c_gpu, g_gpu, _ = cq.evaluate(q.u)
    g_ref = np.asarray(ref["grad"])
    return {"precision": precision, "slices": q.N, "cost_rel": abs(c_gpu - ref["cost"]) / abs(ref["cost"]),
            "grad_rel": float(np.linalg.norm(np.ravel(g_gpu) - g_ref) / np.linalg.norm(g_ref))}


def measure_config(name, precision, peaks, stream, flush, K, warmup, fp64_N=0, err_slices=0, fp64_cache=None,
                   form=None, members=1, N=0):
    """One per-config line: device time per evaluation, slice-steps/s, its own roofline, the
    plain FP64 GPU form's time on the same workload (on its first fp64_N slices, scaled by N,
    when fp64_N > 0; fp64_N < 0: not timed), and the error against the oracle on the first
    err_slices slices.  form: Context options (propagation, exponential)."""
    import torch
    from paper_1612_04929_gb300 import Context
    form = form or {}
    prob = make_problem(name, N, members)
    u = torch.tensor(prob.u, dtype=torch.float64, device="cuda")
    grad = torch.empty_like(u)
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    # timed without per-kernel events, replayed from a captured graph where the path allows it (the
    # per-slice path); the per-kernel times of the roofline from a second, event-bracketed context
    with Context(precision, device=0, stream=stream.cuda_stream, graph=True, **form) as ctx:
        ctx.set_problem(prob)
        ms = time_device_evals(ctx, u, grad, out, K, warmup, flush, stream)
        info = ctx.info()
    with Context(precision, device=0, stream=stream.cuda_stream, profile=True, **form) as cp:
        cp.set_problem(prob)
        time_device_evals(cp, u, grad, out, 1, 0, flush, stream)
        cp.reset_profile()
        ms_p = time_device_evals(cp, u, grad, out, K, 0, flush, stream)   # per-kernel events
        prof = cp.profile()
    units = prob.N * prob.E
    row = {"workload": prob.name, "precision": precision, "d": prob.d, "N": prob.N, "M": prob.M, "S": prob.S,
           "E": prob.E, "p": info["p"], "n": info["n"], "kernel_path": info["kernel_path"],
           "taylor_scheme": ["horner", "paterson-stockmeyer"][info.get("taylor_scheme", 0)],
           "ms_per_step": ms, "value": units / (ms / 1e3), "unit": UNIT, "steps": K,
           "graph": info["kernel_path"] == 0,
           "roofline": roofline_of(prob, precision, info, prof, K, peaks), **form}
    row["roofline_events_ms_per_step"] = ms_p
    if precision != "fp64" and fp64_N >= 0:
        key = (name, fp64_N)
        if fp64_cache is not None and key in fp64_cache:
            row["fp64_form"] = fp64_cache[key]
        else:
            q = prob if not fp64_N else truncated(prob, fp64_N)
            uq = torch.tensor(q.u, dtype=torch.float64, device="cuda")
            gq = torch.empty_like(uq)
            with Context("fp64", device=0, stream=stream.cuda_stream) as c64:
                c64.set_problem(q)
                ms64 = time_device_evals(c64, uq, gq, out, 1 if fp64_N else 2, 1, flush, stream)
            scale = prob.N / q.N
            row["fp64_form"] = {"ms_per_step": ms64 * scale, "value": units / (ms64 * scale / 1e3),
                                "measured_slices": q.N,
                                "how": "timed on the whole workload" if q is prob else
                                       f"timed on the first {q.N} slices and scaled by N (time is linear in N)"}
            if fp64_cache is not None:
                fp64_cache[key] = row["fp64_form"]
        row["speedup_vs_fp64_form"] = row["fp64_form"]["ms_per_step"] / ms
    if err_slices:
        try:
            row["error_vs_oracle"] = gpu_error_vs_oracle(prob, precision, stream, err_slices, form=form)
        except Exception as exc:
            row["error_vs_oracle"] = {"failed": str(exc)[:200]}
    return row


def measure_batch(count, ensemble, K, warmup, stream, flush, one_by_one=True, profile=False, err_problems=()):
    """The batched sweep: `count` problems of uneven d, N, M with `ensemble`-member detuning
    ensembles, FP32 form, one launch of the batch captured into a CUDA graph per step (the
    timed value; without per-kernel profiling), beside one qoc_evaluate_batch call per step
    (streams fanned out from the host) and, optionally, the same contexts evaluated one after
    another; checked against the oracle on the first 40 slices of the listed problems."""
    import torch
    import synthetic as sy
    from paper_1612_04929_gb300 import Batch, Context, qoc_evaluate_batch
    probs = sy.batch_problems(count, ensemble=ensemble)
    ctxs = []
    for p in probs:
        c = Context("fp32", profile=profile)
        c.set_problem(p)
        ctxs.append(c)
    us = [torch.tensor(p.u, dtype=torch.float64, device="cuda") for p in probs]
    gs = [torch.empty_like(u) for u in us]
    outs = [torch.empty(6, dtype=torch.float64, device="cuda") for _ in probs]
    ptr = lambda ts: [t.data_ptr() for t in ts]

    def batch():
        qoc_evaluate_batch(ctxs, ptr(us), ptr(gs), ptr(outs), stream.cuda_stream)

    def seq():
        for c, u, g, o in zip(ctxs, us, gs, outs):
            c.evaluate_device(u.data_ptr(), g.data_ptr(), o.data_ptr())
            c.sync()

    def timed(step):
        ts = []
        for _ in range(K):
            flush.zero_()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            e.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(e))
        return sum(ts) / len(ts)

    for _ in range(max(warmup, 1)):
        batch()
    torch.cuda.synchronize()
    ms_fanout = timed(batch)
    ms_graph = None
    graph = None
    if not profile:   # the captured batch: one graph launch per step
        graph = Batch(ctxs, ptr(us), ptr(gs), ptr(outs), stream.cuda_stream)
        for _ in range(max(warmup, 1)):
            graph.launch(stream.cuda_stream)
        graph.sync()
        ms_graph = timed(lambda: graph.launch(stream.cuda_stream))
        graph.sync()
        graph.close()
    ms = ms_graph if ms_graph is not None else ms_fanout
    by_d = {}
    if profile:     # per-kernel event time summed over the contexts (overlapping)
        for c, p in zip(ctxs, probs):
            for k, (n_l, t) in c.profile().items():
                key = f"d{p.d}:{k}"
                by_d[key] = by_d.get(key, 0.0) + t / K
    ms_seq = None
    if one_by_one:
        seq()
        t0 = time.perf_counter()
        reps = max(1, min(K, 2))
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            seq()
        ms_seq = (time.perf_counter() - t0) * 1e3 / reps
    infos = [c.info() for c in ctxs]
    for c in ctxs:
        c.close()
    units = sum(p.N * p.E for p in probs)
    flops = 0.0
    for p, inf in zip(probs, infos):
        flops += p.N * p.E * (expm_flops_per_slice(p.d, inf["p"], inf["n"]) +
                              adj_flops_per_slice(inf.get("adjoint_form", 1), p.d, inf["p"], inf["n"], p.S))
    row = {"workload": f"batch{count}_E{ensemble}", "problems": count, "members": ensemble, "precision": "fp32",
           "slice_steps_per_step": units, "ms_per_step": ms, "value": units / (ms / 1e3), "unit": UNIT, "steps": K,
           "launch": "one CUDA-graph launch of the captured batch" if ms_graph is not None else "qoc_evaluate_batch",
           "fanout_ms_per_step": ms_fanout,
           "d_counts": {str(d): sum(1 for p in probs if p.d == d) for d in sorted({p.d for p in probs})},
           "one_by_one_ms_per_step": ms_seq, "batch_speedup_vs_one_by_one": (ms_seq / ms) if ms_seq else None,
           "graph_speedup_vs_fanout": (ms_fanout / ms_graph) if ms_graph else None,
           "step_algorithmic_tflops": flops / (ms / 1e3) / 1e12,
           "note": "step_algorithmic_tflops: the exponentials' and adjoints' algorithmic flops (8 d^3 per complex "
                   "product) of every problem over the batch's time (no single dominant kernel)"}
    if by_d:
        row["kernel_ms_by_d"] = {k: round(v, 3) for k, v in sorted(by_d.items(), key=lambda kv: -kv[1])[:16]}
    if err_problems:
        errs = []
        for i in err_problems:
            try:
                e = gpu_error_vs_oracle(probs[i], "fp32", stream, 40)
                e["problem"] = probs[i].name
            except Exception as exc:
                e = {"problem": probs[i].name, "failed": str(exc)[:200]}
            errs.append(e)
        row["error_vs_oracle"] = errs
    return row


def per_config_lines(args, peaks, stream, flush):
    """The other configurations, each bounded to a few seconds of GPU time: the gate (d = 4,
    FP64), the 81-level and 256-level systems in the FP32 and BF16_SPLIT forms, and the batched
    sweep with 1 and 32 ensemble members (32 members on the first 16 problems, 512 trajectories)."""
    rows = {}
    fp64_cache = {}
    plan = [("c1_cnot2q_fp64", "cnot2q", "fp64", 5, 0, 200),
            ("c3_transmon4_fp32", "transmon4", "fp32", 3, 0, 1000),
            ("c3_transmon4_bf16", "transmon4", "bf16", 3, 0, 1000),
            ("c4_gue256_fp32", "gue256", "fp32", 2, 200, 40),
            ("c4_gue256_bf16", "gue256", "bf16", 2, 200, 40)]
    state = {"propagation": "state"}
    cheb = {"propagation": "state", "exponential": "chebyshev"}
    # the cat-state system (d = 154, N = 8000): unitary form and state mode; and a 16-member
    # robust-control ensemble on its first 1000 slices, where state mode runs the members at once
    plan += [("f1_cat_state_unitary_fp32", "cat_state", "fp32", 2, -1, 200, {}, 1, 0),
             ("f1_cat_state_chebyshev_fp32", "cat_state", "fp32", 1, -1, 200, cheb, 1, 0),
             ("f1_cat_state_E16_N1000_unitary_fp32", "cat_state", "fp32", 2, -1, 0, {}, 16, 1000),
             ("f1_cat_state_E16_N1000_taylor_fp32", "cat_state", "fp32", 2, -1, 0, state, 16, 1000),
             ("f1_cat_state_E16_N1000_chebyshev_fp32", "cat_state", "fp32", 2, -1, 40, cheb, 16, 1000)]
    for entry in plan:
        key, name, prec, K, fp64_N, err = entry[:6]
        form, members, nsl = (entry[6:] + ({}, 1, 0))[:3] if len(entry) > 6 else ({}, 1, 0)
        try:
            rows[key] = measure_config(name, prec, peaks, stream, flush, K, 1, fp64_N=fp64_N, err_slices=err,
                                       fp64_cache=fp64_cache, form=form, members=members, N=nsl)
        except Exception as exc:
            rows[key] = {"failed": str(exc)[:300]}
        print(f"# per_config {key}: {json.dumps(rows[key])[:300]}", file=sys.stderr, flush=True)
    # error samples: problems 2 (d = 81), 7 (d = 40) and 15 (d = 128) of the sweep
    for key, count, ens, K, seq, errs in (("c5_batch128_E1", 128, 1, 2, True, (2, 7, 15)),
                                          ("c5_batch16_E32", 16, 32, 1, False, (15,))):
        try:
            rows[key] = measure_batch(count, ens, K, 1, stream, flush, one_by_one=seq, err_problems=errs)
        except Exception as exc:
            rows[key] = {"failed": str(exc)[:300]}
        print(f"# per_config {key}: {json.dumps(rows[key])[:300]}", file=sys.stderr, flush=True)
    return rows


def ours_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1612_04929_gb300 import Context, build as qbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    if rank == 0:
        qbuild.build()
    if world > 1:
        dist.barrier()
    peaks = measured_peaks(local)
    prob = make_problem(args.workload, args.N, args.members)
    precision = args.precision or prob.precision
    stream = torch.cuda.Stream()          # every kernel of the step and every event on one stream
    torch.cuda.set_stream(stream)
    form = dict(propagation=args.propagation, exponential=args.exponential)
    if args.taylor_scheme != "auto":
        form["taylor_scheme"] = args.taylor_scheme
    if not args.no_autotune:   # timed during the warm-up; the other contexts below take the cached choice
        form["autotune"] = True
    ctx = Context(precision, device=local, stream=stream.cuda_stream, ckpt_stride=args.ckpt_stride,
                  gradient=args.gradient, graph=args.graph, **form)
    ctx.set_problem(prob)
    u = torch.tensor(prob.u, dtype=torch.float64, device="cuda")
    grad = torch.empty_like(u)
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def step():
        ctx.evaluate_device(u.data_ptr(), grad.data_ptr(), out.data_ptr())

    for _ in range(max(args.warmup, 3)):
        step()
    ctx.sync()
    info = ctx.info()
    K = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(K):
            flush.zero_()
            starts[k].record(stream)
            step()
            ends[k].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / K
    ctx.sync()
    t_max = slowest_rank_ms(ms, world, "cuda")
    units = prob.N * prob.E
    value = job_value(units, world, t_max)

    # The per-kernel times come from a second timed pass of the same K steps with every kernel
    # bracketed by CUDA events on the context stream (the headline above runs without them).
    # The dominant kernel's roofline: algorithmic flops / its summed event time.
    cp = Context(precision, device=local, stream=stream.cuda_stream, ckpt_stride=args.ckpt_stride,
                 profile=True, gradient=args.gradient, **form)
    cp.set_problem(prob)
    gp = torch.empty_like(u)
    op = torch.empty(6, dtype=torch.float64, device="cuda")
    ms_prof = time_device_evals(cp, u, gp, op, K, max(args.warmup, 3), flush, stream)
    cp.reset_profile()
    time_device_evals(cp, u, gp, op, K, 0, flush, stream)
    prof = cp.profile()
    cp.close()
    roof = roofline_of(prob, precision, info, prof, K, peaks,
                       traffic_key=(prob.name, precision, "expm_fwd", info.get("taylor_scheme", 0)))
    if roof is not None:
        pipes = MEASURED_PIPES.get((prob.name, precision, roof["kernel"], info.get("taylor_scheme", 0)))
        if pipes:
            roof["executed"] = dict(pipes, source="ncu --set full, one launch of this kernel at this workload "
                                                  "(sm__pipe_fma_cycles_active, smsp__issue_active)")
        roof["events_pass_ms_per_step"] = ms_prof
    kernels = {k: {"launches": v[0], "ms_per_step": v[1] / K} for k, v in prof.items()}

    # end to end through the host API with pinned buffers
    uh = torch.tensor(prob.u, dtype=torch.float64).pin_memory()
    gh = torch.empty_like(uh).pin_memory()
    ctx.evaluate_host_ptr(uh.data_ptr(), gh.data_ptr())
    e2e_t = []
    for k in range(max(1, min(K, 5))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.evaluate_host_ptr(uh.data_ptr(), gh.data_ptr())
        e2e_t.append(time.perf_counter() - t0)
    e2e_value = units * world / (sum(e2e_t) / len(e2e_t))
    mn_bytes = prob.M * prob.N * 8

    # the other launch mode on the per-slice path: plain launches when the headline replays a
    # captured graph, the graph replay when it launches directly
    graph_replay = plain_launches = None
    graphed = args.graph and info["kernel_path"] == 0
    if info["kernel_path"] == 0:
        cg = Context(precision, device=local, stream=stream.cuda_stream, ckpt_stride=args.ckpt_stride,
                     gradient=args.gradient, graph=not args.graph, **form)
        cg.set_problem(prob)
        gg = torch.empty_like(u)
        og = torch.empty(6, dtype=torch.float64, device="cuda")
        msg = time_device_evals(cg, u, gg, og, K, 3, flush, stream)
        same = bool(torch.equal(gg, grad) and torch.equal(og, out))
        if args.graph:
            plain_launches = {"value": units / (msg / 1e3), "unit": UNIT, "ms_per_step": msg, "steps": K,
                              "identical_to_graph_replay": same}
        else:
            graph_replay = {"value": units / (msg / 1e3), "unit": UNIT, "ms_per_step": msg, "steps": K,
                            "identical_to_plain_launches": same}
        cg.close()

    # the plain FP64 GPU form on the same workload (the metric's second part: speedup of the
    # mixed form over it, at the error stated below)
    fp64_form = None
    if precision != "fp64" and not args.no_fp64_form:
        c64 = Context("fp64", device=local, stream=stream.cuda_stream, ckpt_stride=args.ckpt_stride,
                      gradient=args.gradient)
        c64.set_problem(prob)
        g64 = torch.empty_like(u)
        o64 = torch.empty(6, dtype=torch.float64, device="cuda")
        K64 = max(1, min(K, 5))
        ms64 = time_device_evals(c64, u, g64, o64, K64, 3, flush, stream)
        i64 = c64.info()
        fp64_form = {"value": units / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64, "steps": K64,
                     "p": i64["p"], "n": i64["n"]}
        c64.close()

    cpu = None
    error = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nsl = args.cpu_sample or max(20, prob.N // 10)
        # the error reference: the whole workload where the oracle takes seconds, else the sample
        ref_n = prob.N if prob.d <= 81 else nsl
        try:
            mk = f"sy.WORKLOADS[{args.workload!r}](N=n, ensemble={args.members})" if args.members > 1 else None
            t, nsl, ref, nev, busy = oracle_sample_time(args.workload, nsl, ref_slices=ref_n, maker=mk,
                                                        exact=args.gradient == "exact", min_seconds=10.0,
                                                        threads=0)
            t1, _, _, nev1, _ = oracle_sample_time(args.workload, nsl, min_seconds=5.0, threads=1, maker=mk)
            cpu = {"value": nsl * prob.E / t, "unit": UNIT, "cores": busy, "kind": "oracle",
                   "sample": f"first {nsl} of {prob.N} slices of the same workload, FP64 oracle, BLAS default "
                             f"threads on {os.cpu_count()} host cores ({busy} threads gained CPU time), "
                             f"{nev} evaluations in {t * nev:.1f} s ({t:.2f} s each)",
                   "host_cores": os.cpu_count(),
                   "one_thread": {"value": nsl * prob.E / t1, "unit": UNIT, "cores": 1,
                                  "sample": f"the same sample with 1 BLAS thread, {nev1} evaluations in "
                                            f"{t1 * nev1:.1f} s"}}
            if ref is not None:
                if ref_n == prob.N:
                    c_gpu, g_gpu = float(out[0].item()), grad.cpu().numpy()
                else:   # evaluate the same form on the sample problem
                    q = make_problem(args.workload, ref_n, args.members)
                    with Context(precision, device=local, stream=stream.cuda_stream, gradient=args.gradient,
                                 **form) as cq:
                        cq.set_problem(q)
                        c_gpu, g_gpu, _ = cq.evaluate(q.u)
                g_ref = np.asarray(ref["grad"])
                error = {"precision": precision, "slices": ref_n,
                         "cost_rel": abs(c_gpu - ref["cost"]) / abs(ref["cost"]),
                         "grad_rel": float(np.linalg.norm(np.ravel(g_gpu) - g_ref) / np.linalg.norm(g_ref)),
                         "against": "CPU FP64 oracle (eigendecomposition exponentials, explicit adjoint)"}
        except Exception as exc:   # keep the GPU line even if the CPU leg fails
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {exc}"}

    per_config = None
    if rank == 0 and world == 1 and not args.no_per_config:
        per_config = per_config_lines(args, peaks, stream, flush)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": max(args.warmup, 3), "ms_per_step": t_max, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "fp32": "f32", "tf32": "tf32x3", "bf16": "bf16x3"}[precision],
                "data": f"synthetic (seeded {prob.name} system, random controls)",
                "config": config_of(prob, precision, info["ckpt_stride"],
                                    {"p": p_of(info), "n": info["n"], "wave_slices": info["wave_slices"],
                                     "autotune": (None if args.no_autotune else
                                                  {"candidates_timed": info.get("autotune_candidates")}),
                                     "n_waves": info["n_waves"], "gradient": args.gradient, "graph": graphed,
                                     "propagation": args.propagation, "exponential": args.exponential,
                                     "taylor_scheme": ["horner", "paterson-stockmeyer"][info.get("taylor_scheme", 0)],
                                     "adjoint": {0: "reverse mode", 1: "block recursion", 2: "none (first-order)",
                                                 3: "low-rank reverse mode", 4: "state-mode reverse pass"}.get(
                                         info.get("adjoint_form"), "?")}),
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": mn_bytes,
                        "d2h_bytes_per_step": mn_bytes + 6 * 8 + 32},
                "gpu_launches": info["launches_per_eval"] * K,
                "clocks": clk.summary(), "kernels": kernels,
                "peaks": peaks,
                "graph_replay": graph_replay,
                "plain_launches": plain_launches,
                "fp64_form": fp64_form,
                "speedup_vs_fp64_form": (value / fp64_form["value"]) if fp64_form else None,
                "error_vs_oracle": error,
                "per_config": per_config,
                "cost": float(out[0].item())}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def p_of(info):
    return info["p"]


def batch_arm(args):
    """The batched sweep alone (--workload batch): `count` problems of uneven d in
    {4, 8, 16, 40, 81, 128}, N in [200, 4000], M in [2, 8], each with an `ensemble`-member
    detuning ensemble, FP32 form, evaluated by one qoc_evaluate_batch call per step; compared
    with evaluating the same contexts one after another.  Metric: sum_i N_i E_i / seconds per
    step."""
    import torch
    from paper_1612_04929_gb300 import build as qbuild
    qbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        row = measure_batch(args.count, args.ensemble, args.steps, args.warmup, stream, flush,
                            profile=args.profile_batch)
    line = {"metric": METRIC, "value": row["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": row["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded batched sweep)",
            "config": {"workload": row["workload"], "problems": args.count, "members": args.ensemble,
                       "slice_steps_per_step": row["slice_steps_per_step"], "d_counts": row["d_counts"],
                       "launch": row["launch"]},
            "fanout_ms_per_step": row["fanout_ms_per_step"], "graph_speedup_vs_fanout": row["graph_speedup_vs_fanout"],
            "one_by_one_ms_per_step": row["one_by_one_ms_per_step"],
            "batch_speedup_vs_one_by_one": row["batch_speedup_vs_one_by_one"],
            "kernel_ms_by_d": row.get("kernel_ms_by_d"), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def dsweep_arm(args):
    """The per-d sweep: for d = 2 .. 256 (log2(d) qubits, GUE drift, Pauli controls, Haar target,
    full unitary, FP32 form), the fwd+grad slice-steps/s, the plain FP64 GPU form's and the
    speedup over it, and the relative error against the oracle (whole evolution for d <= 64, the
    first 100 slices above).  Each point is timed over `steps` evaluations after `warmup`, with
    the L2 flushed before each."""
    import numpy as np
    import torch
    import synthetic as sy
    from paper_1612_04929_gb300 import Context, build as qbuild
    qbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def timed(ctx, u, steps):
        g = torch.empty_like(u)
        o = torch.empty(6, dtype=torch.float64, device="cuda")
        for _ in range(max(args.warmup, 3)):
            ctx.evaluate_device(u.data_ptr(), g.data_ptr(), o.data_ptr())
        ctx.sync()
        ts = []
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.evaluate_device(u.data_ptr(), g.data_ptr(), o.data_ptr())
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return sum(ts) / len(ts), g, o

    per_d = {}
    tot_units = tot_ms = 0.0
    with ClockSampler(0) as clk:
        for d in sy.DSWEEP_D:
            N = 2000 if d <= 64 else 500
            prob = sy.dsweep_problem(d, N=N)
            u = torch.tensor(prob.u, dtype=torch.float64, device="cuda")
            # tuned during the warm-up and, on the per-slice path, replayed from a captured graph (as
            # the headline; --no-autotune / --no-graph take the planner's choices / plain launches)
            with Context("fp32", stream=stream.cuda_stream, graph=args.graph, autotune=not args.no_autotune) as c:
                c.set_problem(prob)
                ms, g, o = timed(c, u, args.steps)
                info = c.info()
                g32, c32 = g.cpu().numpy(), float(o[0].item())
            with Context("fp64", stream=stream.cuda_stream) as c:
                c.set_problem(prob)
                ms64, _, _ = timed(c, u, max(1, min(args.steps, 3)))
            row = {"N": N, "ms_per_step": ms, "value": N / (ms / 1e3), "fp64_ms_per_step": ms64,
                   "speedup_vs_fp64_form": ms64 / ms, "p": info["p"], "n": info["n"],
                   "kernel_path": info["kernel_path"], "graph": bool(args.graph and info["kernel_path"] == 0),
                   "wave_slices": info["wave_slices"]}
            if not args.no_cpu_baseline:
                ref_n = N if d <= 64 else 100
                try:
                    t, _, ref, _, _ = oracle_sample_time("dsweep", min(N, 50), ref_slices=ref_n,
                                                   maker=f"sy.dsweep_problem({d}, N=n)")
                    if ref_n == N:
                        c_gpu, g_gpu = c32, g32
                    else:
                        q = sy.dsweep_problem(d, N=ref_n)
                        with Context("fp32", stream=stream.cuda_stream) as cq:
                            cq.set_problem(q)
                            c_gpu, g_gpu, _ = cq.evaluate(q.u)
                    g_ref = np.asarray(ref["grad"])
                    row["grad_rel"] = float(np.linalg.norm(np.ravel(g_gpu) - g_ref) / np.linalg.norm(g_ref))
                    row["cost_rel"] = abs(c_gpu - ref["cost"]) / abs(ref["cost"])
                    row["error_slices"] = ref_n
                    row["oracle_slice_steps_per_s"] = min(N, 50) / t
                except Exception as exc:
                    row["oracle"] = f"failed: {exc}"
            per_d[str(d)] = row
            tot_units += N
            tot_ms += ms
    line = {"metric": METRIC, "value": tot_units / (tot_ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": tot_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded GUE-drift qubit registers)",
            "config": {"workload": "dsweep", "d": list(sy.DSWEEP_D), "precision": "fp32",
                       "l2": "flushed before every timed evaluation", "autotune": not args.no_autotune},
            "per_d": per_d, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload.startswith("batch"):
        batch_arm(args)
    elif args.workload == "dsweep":
        dsweep_arm(args)
    else:
        ours_arm(args)


if __name__ == "__main__":
    main()
