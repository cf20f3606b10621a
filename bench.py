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
    # split exponential, waves of 1125 and 875 slices: 139,826,432 and 91,752,192 bytes
    ("transmon_cavity_d40", "fp32", "expm_fwd", 1125): 115789312.0,
}
# executed side of the same kernel from one full ncu capture (1125-slice launch): FMA pipe and
# issue activity, % of peak over active cycles
MEASURED_PIPES = {
    ("transmon_cavity_d40", "fp32", "expm_fwd", 1125): {"fma_pipe_pct": 47.2, "issue_active_pct": 68.7},
}
# FP32 FMA peak from unit counts: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (max SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
L2_FLUSH_BYTES = 256 << 20


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
    ap.add_argument("--graph", action="store_true", help="replay each evaluation from a captured CUDA graph")
    ap.add_argument("--gradient", choices=["exact", "first_order"], default="exact",
                    help="exact derivative of the truncated series, or the paper's first-order Eq. 11")
    return ap.parse_args()


def make_problem(name, N=0):
    import synthetic as sy
    return sy.WORKLOADS[name](N=N) if N else sy.WORKLOADS[name]()


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
def oracle_sample_time(workload, nslices, repeats=1, ref_slices=0, exact=True, maker=None, min_seconds=0.0):
    """Times the CPU FP64 oracle on the first `nslices` slices of the workload in a child
    process limited to one BLAS thread: at least `repeats` evaluations, and more until
    `min_seconds` of timed work.  With ref_slices > 0 the child also evaluates the oracle once on
    the first ref_slices slices (untimed) and returns its cost and gradient, the reference for
    the GPU result's error.  Returns (seconds per evaluation, slices, reference, evaluations)."""
    code = f"""
import json, os, sys, time
sys.path.insert(0, {ROOT!r})
import synthetic as sy
from oracle import qoc_oracle as orc
make = (lambda n: {maker}) if {maker!r} else (lambda n: sy.WORKLOADS[{workload!r}](N=n))
p = make({nslices})
orc.cost_and_grad(p, p.u)
ts = []
while len(ts) < {repeats} or (sum(ts) < {min_seconds} and len(ts) < 1000):
    t0 = time.perf_counter(); orc.cost_and_grad(p, p.u); ts.append(time.perf_counter() - t0)
ref = None
if {ref_slices} > 0:
    q = make({ref_slices})
    c, g, _ = orc.cost_and_grad(q, q.u, exact={exact!r})
    ref = {{"N": {ref_slices}, "cost": float(c), "grad": [float(x) for x in g.ravel()]}}
print(json.dumps({{"t": sum(ts) / len(ts), "n": len(ts), "ref": ref}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr)
    res = json.loads(r.stdout.strip().splitlines()[-1])
    return float(res["t"]), nslices, res["ref"], int(res["n"])


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
def expm_flops_per_slice(d, p, n):
    """Algorithmic flops of one slice exponential: p - 1 Horner and n squaring complex d x d
    products at 8 d^3 real flops each."""
    return (p - 1 + n) * 8.0 * d ** 3


def adj_flops_per_slice(form, d, p, n, S):
    """Algorithmic flops of one slice's adjoint: reverse mode 2 products per forward product plus
    Ubar = G Psi^dag; block recursion 3; low-rank reverse mode (cotangent as d x r factors,
    r = 2^n S): 2 d x d by d x r products per squaring level (r doubling from S), 3 per Horner step
    and one final rank-r update."""
    if form == 3:
        r = S << n
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
    prob = make_problem(args.workload, args.N)
    precision = args.precision or prob.precision
    stream = torch.cuda.Stream()          # every kernel of the step and every event on one stream
    torch.cuda.set_stream(stream)
    # per-kernel events (profile) need plain launches; with --graph the step is a graph replay
    ctx = Context(precision, device=local, stream=stream.cuda_stream, ckpt_stride=args.ckpt_stride,
                  profile=not args.graph, gradient=args.gradient, graph=args.graph)
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
    ctx.reset_profile()
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
    prof = ctx.profile()
    ctx.sync()
    t_max = slowest_rank_ms(ms, world, "cuda")
    units = prob.N * prob.E
    value = job_value(units, world, t_max)

    # dominant kernel and its roofline (algorithmic flops / measured launch time)
    d, p, n = prob.d, info["p"], info["n"]
    per_slice = {"expm_fwd": expm_flops_per_slice(d, p, n),
                 "expm_fwd (recompute)": expm_flops_per_slice(d, p, n),
                 "expm_adj": adj_flops_per_slice(info.get("adjoint_form", 1), d, p, n, prob.S)}
    # the roofline line covers the dominant kernel that has an algorithmic flop count (the
    # exponential kernels); the serial sweeps are latency-bound and reported in "kernels"
    if info.get("adjoint_form") == 2:   # first-order gradient: no adjoint exponential
        per_slice.pop("expm_adj")
    cands = {k: v for k, v in prof.items() if k in per_slice}
    roof = None
    if cands:
        top_name, (top_launches, top_ms) = max(cands.items(), key=lambda kv: kv[1][1])
        N_w = info["wave_slices"]
        last = prob.N - (info["n_waves"] - 1) * N_w
        slices = prob.N if top_name != "expm_fwd (recompute)" else prob.N - last
        flops = per_slice[top_name] * slices * prob.E * K
        achieved = flops / (top_ms / 1e3) / 1e12
        fp32 = precision != "fp64"
        # DRAM bytes per launch of the dominant kernel, from an ncu capture of the same kernel at
        # this workload (dram__bytes_read.sum + dram__bytes_write.sum); None where none was taken
        traffic = MEASURED_TRAFFIC.get((prob.name, precision, top_name, info["wave_slices"]))
        pipes = MEASURED_PIPES.get((prob.name, precision, top_name, info["wave_slices"]))
        roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS if fp32 else None,
                "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS if fp32 else None,
                "traffic": traffic, "kernel": top_name, "launches": top_launches,
                "avg_launch_ms": top_ms / top_launches,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz",
                "note": "algorithmic flops (8 d^3 per complex product); the FP32 form's grid-split "
                        "products execute 12 FMAs per complex multiply-add (3.25 per algorithmic one), "
                        "so the split exponential's fraction is bounded near 0.3 by construction",
                "traffic_source": ("dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of this "
                                   "kernel at this workload") if traffic else None}
        if pipes:
            roof["executed"] = dict(pipes, source="ncu --set full, one launch of this kernel at this workload "
                                                  "(sm__pipe_fma_cycles_active, smsp__issue_active)")
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

    # the same evaluation replayed from a captured CUDA graph (per-slice path only; the timed
    # region above uses plain launches so that every kernel carries its own events)
    graph_replay = None
    if not args.graph and info["kernel_path"] == 0:
        cg = Context(precision, device=local, stream=stream.cuda_stream, ckpt_stride=args.ckpt_stride,
                     gradient=args.gradient, graph=True)
        cg.set_problem(prob)
        gg = torch.empty_like(u)
        og = torch.empty(6, dtype=torch.float64, device="cuda")
        for _ in range(3):
            cg.evaluate_device(u.data_ptr(), gg.data_ptr(), og.data_ptr())
        cg.sync()
        sg = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        eg = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        torch.cuda.synchronize()
        for k in range(K):
            flush.zero_()
            sg[k].record(stream)
            cg.evaluate_device(u.data_ptr(), gg.data_ptr(), og.data_ptr())
            eg[k].record(stream)
        torch.cuda.synchronize()
        msg = sum(s.elapsed_time(e) for s, e in zip(sg, eg)) / K
        graph_replay = {"value": units / (msg / 1e3), "unit": UNIT, "ms_per_step": msg, "steps": K,
                        "identical_to_plain_launches": bool(torch.equal(gg, grad) and torch.equal(og, out))}
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
        for _ in range(3):
            c64.evaluate_device(u.data_ptr(), g64.data_ptr(), o64.data_ptr())
        c64.sync()
        K64 = max(1, min(K, 5))
        s64 = [torch.cuda.Event(enable_timing=True) for _ in range(K64)]
        e64 = [torch.cuda.Event(enable_timing=True) for _ in range(K64)]
        torch.cuda.synchronize()
        for k in range(K64):
            flush.zero_()
            s64[k].record(stream)
            c64.evaluate_device(u.data_ptr(), g64.data_ptr(), o64.data_ptr())
            e64[k].record(stream)
        torch.cuda.synchronize()
        ms64 = sum(s.elapsed_time(e) for s, e in zip(s64, e64)) / K64
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
            t, nsl, ref, nev = oracle_sample_time(args.workload, nsl, ref_slices=ref_n,
                                                  exact=args.gradient == "exact", min_seconds=10.0)
            cpu = {"value": nsl * prob.E / t, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"first {nsl} of {prob.N} slices of the same workload, FP64 oracle, 1 BLAS thread, "
                             f"{nev} evaluations in {t * nev:.1f} s ({t:.2f} s each)"}
            if ref is not None:
                if ref_n == prob.N:
                    c_gpu, g_gpu = float(out[0].item()), grad.cpu().numpy()
                else:   # evaluate the same form on the sample problem
                    q = make_problem(args.workload, ref_n)
                    with Context(precision, device=local, stream=stream.cuda_stream, gradient=args.gradient) as cq:
                        cq.set_problem(q)
                        c_gpu, g_gpu, _ = cq.evaluate(q.u)
                g_ref = np.asarray(ref["grad"])
                error = {"precision": precision, "slices": ref_n,
                         "cost_rel": abs(c_gpu - ref["cost"]) / abs(ref["cost"]),
                         "grad_rel": float(np.linalg.norm(np.ravel(g_gpu) - g_ref) / np.linalg.norm(g_ref)),
                         "against": "CPU FP64 oracle (eigendecomposition exponentials, explicit adjoint)"}
        except Exception as exc:   # keep the GPU line even if the CPU leg fails
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {exc}"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": max(args.warmup, 3), "ms_per_step": t_max, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "fp32": "f32", "tf32": "tf32x3", "bf16": "bf16x3"}[precision],
                "data": f"synthetic (seeded {prob.name} system, random controls)",
                "config": config_of(prob, precision, info["ckpt_stride"],
                                    {"p": p, "n": n, "wave_slices": info["wave_slices"], "n_waves": info["n_waves"],
                                     "gradient": args.gradient, "graph": args.graph,
                                     "adjoint": {0: "reverse mode", 1: "block recursion", 2: "none (first-order)",
                                                 3: "low-rank reverse mode"}.get(
                                         info.get("adjoint_form"), "?")}),
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": mn_bytes,
                        "d2h_bytes_per_step": mn_bytes + 6 * 8 + 32},
                "gpu_launches": info["launches_per_eval"] * K,
                "clocks": clk.summary(), "kernels": kernels,
                "graph_replay": graph_replay,
                "fp64_form": fp64_form,
                "speedup_vs_fp64_form": (value / fp64_form["value"]) if fp64_form else None,
                "error_vs_oracle": error,
                "cost": float(out[0].item())}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def batch_arm(args):
    """The batched sweep: `count` problems of uneven d in {4, 8, 16, 40, 81, 128}, N in
    [200, 4000], M in [2, 8], each with an `ensemble`-member detuning ensemble, FP32 form,
    evaluated by one qoc_evaluate_batch call per step; compared with evaluating the same
    contexts one after another.  Metric: sum_i N_i E_i / seconds per step."""
    import torch
    import synthetic as sy
    from paper_1612_04929_gb300 import Context, build as qbuild, qoc_evaluate_batch
    qbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    probs = sy.batch_problems(args.count, ensemble=args.ensemble)
    ctxs = []
    for p in probs:
        c = Context("fp32", profile=args.profile_batch)
        c.set_problem(p)
        ctxs.append(c)
    us = [torch.tensor(p.u, dtype=torch.float64, device="cuda") for p in probs]
    gs = [torch.empty_like(u) for u in us]
    outs = [torch.empty(6, dtype=torch.float64, device="cuda") for _ in probs]
    ptr = lambda ts: [t.data_ptr() for t in ts]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def batch():
        qoc_evaluate_batch(ctxs, ptr(us), ptr(gs), ptr(outs), stream.cuda_stream)

    def one_by_one():
        for c, u, g, o in zip(ctxs, us, gs, outs):
            c.evaluate_device(u.data_ptr(), g.data_ptr(), o.data_ptr())
            c.sync()

    for _ in range(max(args.warmup, 1)):
        batch()
    torch.cuda.synchronize()
    K = args.steps
    ts = []
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for _ in range(K):
            flush.zero_()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            batch()
            e.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(e))
    ms = sum(ts) / len(ts)
    by_d = {}
    if args.profile_batch:     # per-kernel event time summed over the contexts (overlapping)
        for c, p in zip(ctxs, probs):
            for k, (n_l, t) in c.profile().items():
                key = f"d{p.d}:{k}"
                by_d[key] = by_d.get(key, 0.0) + t / K
        for c in ctxs:
            c.reset_profile()
    one_by_one()
    t0 = time.perf_counter()
    for _ in range(max(1, min(K, 2))):
        flush.zero_()
        torch.cuda.synchronize()
        one_by_one()
    ms_seq = (time.perf_counter() - t0) * 1e3 / max(1, min(K, 2))
    units = sum(p.N * p.E for p in probs)
    line = {"metric": METRIC, "value": units / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded batched sweep)",
            "config": {"workload": f"batch{args.count}_E{args.ensemble}", "problems": args.count,
                       "members": args.ensemble, "slice_steps_per_step": units,
                       "d_counts": {str(d): sum(1 for p in probs if p.d == d) for d in sorted({p.d for p in probs})}},
            "one_by_one_ms_per_step": ms_seq, "batch_speedup_vs_one_by_one": ms_seq / ms,
            "kernel_ms_by_d": {k: round(v, 3) for k, v in sorted(by_d.items(), key=lambda kv: -kv[1])[:16]},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    for c in ctxs:
        c.close()


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
            with Context("fp32", stream=stream.cuda_stream) as c:
                c.set_problem(prob)
                ms, g, o = timed(c, u, args.steps)
                info = c.info()
                g32, c32 = g.cpu().numpy(), float(o[0].item())
            with Context("fp64", stream=stream.cuda_stream) as c:
                c.set_problem(prob)
                ms64, _, _ = timed(c, u, max(1, min(args.steps, 3)))
            row = {"N": N, "ms_per_step": ms, "value": N / (ms / 1e3), "fp64_ms_per_step": ms64,
                   "speedup_vs_fp64_form": ms64 / ms, "p": info["p"], "n": info["n"],
                   "kernel_path": info["kernel_path"]}
            if not args.no_cpu_baseline:
                ref_n = N if d <= 64 else 100
                try:
                    t, _, ref, _ = oracle_sample_time("dsweep", min(N, 50), ref_slices=ref_n,
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
                       "l2": "flushed before every timed evaluation"},
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
