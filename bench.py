#!/usr/bin/env python3
"""Benchmark: 3-D C2C FFT under OpenFFT's decomposition on one GB300.

Default workload (one step): 512 x 512 x 512 complex128 (2.1 GB), re/im
i.i.d. uniform[-1, 1) (seeded), for each P in {64, 256, 1024} logical ranks
one forward and one backward transform -> 6 transforms per step.  Plans are
built and auto-tuned before timing (the paper's initialisation phase,
excluded from timing).  Inputs stay resident in HBM; every array is larger
than L2, so no flush is needed between steps.

Metric: GFLOP/s in the 5 N log2 N convention, whole job (all ranks).
Reported beside it: the roofline of the dominant kernel (live CUDA-event
timing of every launch), end-to-end throughput through the host-buffer C
ABI call (copies included), the plain FP64 form of the same workload, the
FP64 oracle on the host cores, clocks, and the other forms (the 256^3
forward + backward step, FP32, the batched, mixed-radix, real and learned
forms).

``--impl reference`` times the FP64 oracle (plain C, host cores) on a
bounded sample of the same workload: per step, on every host thread the
memory allows, one forward transform of a 64 x 512 x 512 box of the input
(an eighth of the volume, the same 512-point lines), all threads at once.

Multi-GPU (torchrun): every rank runs its own replica of the workload (the
transform does not need another GPU); value = all ranks' flops / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3-D C2C FFT GFLOP/s (5N log2N) & % HBM roofline, plain FP64 vs tuned forms"
UNIT = "GFLOP/s"
N1D = 512
PS = (64, 256, 1024)
WORKLOAD = "512x512x512 complex128 uniform[-1,1), forward+backward at P=64,256,1024 (6 transforms/step)"
# the 256^3 configuration, reported among the forms
N256 = 256
PS256 = (16, 64, 256)
WORKLOAD256 = "256x256x256 complex128 standard-normal, forward+backward at P=16,64,256 (6 transforms/step)"
# the oracle's sample of the headline workload: a box of the first 64 a-planes
SAMPLE_SHAPE = (64, 512, 512)


def flops(N: int) -> float:
    return 5.0 * N * math.log2(N)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


STAGE_SOURCES = ("fft_warp.cuh", "fft_warp_tma.cuh", "fft_tile.cuh", "stage_io.cuh", "arith.cuh", "arith_pair.cuh",
                 "warp_plan.h", "fft_stage.h", "generic_stage.cuh", "fft_stage.cu", "fft_tile_df.cu", "fft_tma_256.cu",
                 "fft_tma_512.cu")


def source_code_only(text: str) -> str:
    """A C/CUDA source with its comments removed and every run of white space
    made one blank, so that editing a comment leaves the hash unchanged."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return re.sub(r"\s+", " ", text).strip()


def stage_source_hash() -> str:
    """Hash of the code of the stage-kernel sources (comments and white space
    aside): a committed DRAM-traffic figure is only reported while the kernel it
    was measured on is unchanged."""
    h = hashlib.sha256()
    for f in STAGE_SOURCES:
        with open(os.path.join(ROOT, "paper_1501_07350_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(source_code_only(fh.read()).encode("utf-8"))
    return h.hexdigest()[:16]


def profiled_traffic(kernel_hash: str, family: str, G: int, n: int = N1D, path: str = ""):
    """DRAM bytes per point of one stage launch of the double-float stage kernel
    of `family` with G lines per CTA over lines of n points, from the committed
    ncu summary, if it was taken on the current kernel sources."""
    path = path or os.path.join(ROOT, "profiles", "fft_%s_kernel_df_n%d.md" % (family, n))
    vals = {}
    try:
        with open(path) as fh:
            for line in fh:
                line = line.strip()
                for key in ("source_hash:", "dram_bytes_per_point G%d:" % G):
                    if line.startswith(key):
                        vals[key[:-1]] = line[len(key):].strip()
        if vals.get("source_hash") == kernel_hash:
            return float(vals["dram_bytes_per_point G%d" % G])
    except Exception:
        pass
    return None


def profiled_traffic_scaled(kernel_hash: str, family: str, G: int, n: int, N: int):
    """roofline.traffic: the profiled DRAM bytes per point times the points of
    one launch (traffic grows in proportion to the points; the capture is
    taken on a smaller array with the same line length)."""
    b = profiled_traffic(kernel_hash, family, G, n)
    return None if b is None else round(b * N)


def df_ops_per_point(n: int) -> float:
    """FP32 operations per point of one double-float stage over lines of n =
    2^k points, as the warp kernel's radix plan runs them: the remainder radix
    (2 or 4) first, then radix 8.  A double-float complex addition costs 16
    operations (TwoSum plus the lo sum, per real part), a twiddle product 32.
    Per point: radix 2 = 16, radix 4 = 32, radix 8 = 54 (24 additions and two
    multiplications by (1 - i)/sqrt 2 per 8 points), plus (R - 1)/R x 32 for
    the twiddles of every pass after the first."""
    per = {2: 16.0, 4: 32.0, 8: 54.0}
    radices, m = [], n
    while m % 8 == 0:
        m //= 8
        radices.append(8)
    if m > 1:
        radices.insert(0, m)
    ops = 0.0
    for i, r in enumerate(radices):
        ops += per[r] + (32.0 * (r - 1) / r if i > 0 else 0.0)
    return ops


def dominant_kernel(chosen: dict):
    """(family, G) that most of the timed plans use (ties: the first P)."""
    fam = {0: "warp", 1: "warp", 2: "tile", 3: "generic"}
    picks = [(fam[c["kernel"]], c["lines_per_cta"]) for c in chosen.values()]
    return max(picks, key=picks.count)


class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.device)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[2]) for r in rows if num(r[2]) is not None]
        mx = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        pw = [num(r[4]) for r in rows if num(r[4]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ------------------------------------------------------- multi-rank ----

def reduce_max(value: float, world: int, device) -> float:
    """Maximum of `value` over all ranks (the slowest rank sets the step time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(work_per_rank_step: float, world: int, ms_per_step: float) -> float:
    """Whole-job throughput (GFLOP/s): every rank's work over the slowest rank's time."""
    return world * work_per_rank_step / (ms_per_step * 1e-3) / 1e9


# ------------------------------------------------------------------ ours --

def time_step(of, torch, n, Ps, x, y, z, stream, args, world, sampler=None):
    """Plans for every P (auto-tuned unless --tune default), warm-up, then
    exactly args.steps timed steps of forward + backward at every P, with a
    barrier and a synchronize on both sides.  Returns the plans (left open)
    and the measurements of this rank."""
    import torch.distributed as dist
    plans = {}
    for P in Ps:
        h = of.openfft_plan(n, n, n, P, of.C2C_F64)
        of.openfft_set_stream(h, stream)
        if args.tune == "exhaustive":
            of.openfft_set_tuning(h, of.TUNE_EXHAUSTIVE)
        plans[P] = h
    chosen = {P: of.openfft_candidate(h, of.openfft_current_candidate(h)) for P, h in plans.items()}

    def step():
        for P in Ps:
            of.openfft_exec_c2c(plans[P], x, y, of.FORWARD)
            of.openfft_exec_c2c(plans[P], y, z, of.BACKWARD)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for h in plans.values():
        of.openfft_set_timing(h, True)
        of.openfft_get_timing(h)       # reset
    if sampler is not None:
        sampler.start()
        time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed_steps_n%d" % n)    # lets a profiler keep the timed launches only
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    clocks = None
    if sampler is not None:
        time.sleep(0.3)
        clocks = sampler.stop()
    phases = {}
    for h in plans.values():
        t = of.openfft_get_timing(h)
        of.openfft_set_timing(h, False)
        for k, v in t.items():
            phases.setdefault(k, {"ms": 0.0, "launches": 0})
            phases[k]["ms"] += v["ms"]
            phases[k]["launches"] += v["launches"]
    launches = sum(phases[k]["launches"] for k in ("fft", "buffer_comm", "communication"))
    return {"plans": plans, "chosen": chosen, "ms_total": e0.elapsed_time(e1), "phases": phases,
            "launches": launches, "clocks": clocks}


def stage_roofline(of, torch, dev, n, chosen, phases, clocks):
    """Roofline of the dominant kernel, the FFT stage kernel (with the fused
    transposes): per launch it reads and writes the array once, 2 x 16 x N
    bytes; its average duration comes from the library's per-launch CUDA
    events over the timed region."""
    N = n ** 3
    peak, peak_kind = load_peaks()
    fft_ms = phases["fft"]["ms"]
    fft_n = max(1, phases["fft"]["launches"])
    avg_s = fft_ms / fft_n * 1e-3
    alg_bytes = 2 * N * 16
    achieved = alg_bytes / avg_s / 1e9
    family, G_dom = dominant_kernel(chosen)
    traffic = profiled_traffic_scaled(stage_source_hash(), family, G_dom, n, N)
    arith_name = "ArDP" if all(c["arith"] == of.ARITH_DOUBLE_FLOAT for c in chosen.values()) else "ArF64"
    if family == "warp" and arith_name == "ArDP" and n in (256, 512):
        kname = "fft_warp_tma_kernel<%d, G=%d> (packed double-float, asynchronous output)" % (n, G_dom)
    else:
        kname = "fft_%s_kernel<%s, %d, G=%d>" % (family, arith_name, n, G_dom)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": kname + " (the tuned stage kernel of most plans; every stage launch of the step is "
                                  "one of the chosen stage kernels)",
                "peak_kind": peak_kind,
                "alg_bytes_per_launch": alg_bytes, "avg_launch_us": round(avg_s * 1e6, 2),
                "share_of_step": round(fft_ms / max(1e-9, phases["exec"]["ms"]), 4)}
    if arith_name == "ArDP":
        # the binding resource of the double-float kernel: the FP32 pipe
        ops = df_ops_per_point(n)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
        alu_peak = sms * 128 * mhz * 1e6 / 1e9
        alu_ach = ops * N / avg_s / 1e9
        roofline["alu"] = {"bound": "alu", "unit": "G FP32 ops/s", "ops_per_point": ops,
                           "achieved": round(alu_ach, 1), "peak": round(alu_peak, 1),
                           "frac": round(alu_ach / alu_peak, 4),
                           "peak_kind": "SMs x 128 FP32 lanes x max SM clock (%d MHz)" % mhz,
                           "ops": "double-float arithmetic of the radix passes only (no conversions, "
                                  "loads or index math); a packed FP32x2 instruction counts as two"}
    return roofline


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1501_07350_gb300 import _build
    from paper_1501_07350_gb300 import openfft as of
    from paper_1501_07350_gb300 import synth

    _build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    n = N1D
    N = n ** 3
    x_np = synth.complex_field((N,), seed=synth.config_seed(5))
    x_host = torch.from_numpy(x_np).pin_memory()
    x = x_host.to(dev)
    y = torch.empty_like(x)
    z = torch.empty_like(x)

    sampler = ClockSampler(local_rank)
    m = time_step(of, torch, n, PS, x, y, z, stream, args, world, sampler)
    plans, chosen, phases, clocks = m["plans"], m["chosen"], m["phases"], m["clocks"]
    t_max = reduce_max(m["ms_total"], world, dev)
    ms_per_step = t_max / args.steps
    work_per_step = 2 * len(PS) * flops(N)
    value = job_value(work_per_step, world, ms_per_step)
    # correctness of the timed outputs (round trip) on this rank
    rt_err = float(torch.linalg.vector_norm(z - x) / torch.linalg.vector_norm(x))
    roofline = stage_roofline(of, torch, dev, n, chosen, phases, clocks)

    # end to end through the host-buffer C ABI (copies inside the timed region).
    # The six transforms of a step are enqueued with the asynchronous call and
    # synchronised at the end, so one transform's host-to-device copy runs
    # beside another's device-to-host copy.  Each backward transform reads the
    # host output of its plan's forward transform: the library orders calls on
    # one plan (an upload waits for the plan's previous download).
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    for P in PS:                    # one upload and one download queue for the three plans
        of.openfft_set_copy_streams(plans[P], up, down)
    y_host = {P: torch.empty_like(x_host).pin_memory() for P in PS}
    z_host = {P: torch.empty_like(x_host).pin_memory() for P in PS}
    xh = x_host.numpy()
    yh = {P: t.numpy() for P, t in y_host.items()}
    zh = {P: t.numpy() for P, t in z_host.items()}

    def host_step():
        for P in PS:
            of.openfft_exec_c2c_host_async(plans[P], xh, yh[P], of.FORWARD)
        for P in PS:
            of.openfft_exec_c2c_host_async(plans[P], yh[P], zh[P], of.BACKWARD)
        for P in PS:
            of.openfft_sync(plans[P])

    def host_step_sync():
        for P in PS:
            of.openfft_exec_c2c_host(plans[P], xh, yh[P], of.FORWARD)
            of.openfft_exec_c2c_host(plans[P], yh[P], zh[P], of.BACKWARD)

    import torch.distributed as dist
    # The host link and host memory are shared with the machine's other GPUs,
    # whose traffic shows up as occasional steps 1.5-2x slower: each step is
    # timed on its own and the median is reported, every step beside it.
    e2e_steps = 5
    t_e2e, t_e2e_steps = {}, {}
    for name, fn in (("sync", host_step_sync), ("async", host_step)):
        fn()
        per = []
        for _ in range(e2e_steps):
            if world > 1:
                dist.barrier()
            t0 = time.perf_counter()
            fn()
            per.append(reduce_max(time.perf_counter() - t0, world, dev))
        t_e2e[name] = float(np.median(per))
        t_e2e_steps[name] = [round(v * 1e3, 1) for v in per]
    zr = zh[PS[-1]]
    e2e_err = float(np.linalg.norm(zr - x_np) / np.linalg.norm(x_np))
    e2e = {"value": round(job_value(work_per_step, world, t_e2e["async"] * 1e3), 2), "unit": UNIT,
           "h2d_bytes_per_step": 2 * len(PS) * N * 16, "d2h_bytes_per_step": 2 * len(PS) * N * 16,
           "steps": e2e_steps, "statistic": "median of the steps, each timed on its own",
           "step_ms": t_e2e_steps["async"], "one_call_at_a_time_step_ms": t_e2e_steps["sync"],
           "mean": round(job_value(work_per_step, world, float(np.mean(t_e2e_steps["async"]))), 2),
           "calls": "openfft_exec_c2c_host_async: three forward and then three backward transforms "
                    "(three plans) enqueued, then synchronised; each backward reads its plan's forward "
                    "output in host memory, ordered by the library; the plans share one upload and one "
                    "download stream",
           "one_call_at_a_time": round(job_value(work_per_step, world, t_e2e["sync"] * 1e3), 2),
           "round_trip_rel_l2": e2e_err}
    del y_host, z_host

    # plain FP64 (the DP pipe) on the same workload, per forward / backward transform
    plain = measure_plain_f64(of, torch, plans, x, y, stream)
    for h in plans.values():
        of.openfft_destroy(h)
    del x, y, z
    torch.cuda.empty_cache()

    # other forms (not the headline): the 256^3 step, FP32, methods, batched, mixed, real, learned
    forms = {"plain_f64_512cubed": plain}
    if not args.quick:
        forms.update(measure_forms(of, torch, stream, args, world))

    arith = {c["arith"] for c in chosen.values()}
    dtype = "f64" if arith == {of.ARITH_NATIVE} else ("f32x2 (double-float, FP64-accurate)"
                                                       if arith == {of.ARITH_DOUBLE_FLOAT} else "f64 / f32x2")
    result = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD, "shape": [n, n, n], "P": list(PS), "transforms_per_step": 6,
                   "l2": "inputs larger than L2 (2.1 GB arrays), no flush", "tuning": args.tune,
                   "chosen": {str(P): c for P, c in chosen.items()}, "parallelism": "replicas"},
        "roofline": roofline, "e2e": e2e, "gpu_launches": int(m["launches"]), "clocks": clocks,
        "phases_ms": {k: round(v["ms"], 3) for k, v in phases.items()},
        "round_trip_rel_l2": rt_err, "forms": forms,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline_sample(x_np, n)
    if rank == 0:
        print(json.dumps(result), flush=True)


def measure_plain_f64(of, torch, plans, x, y, stream, reps=3):
    """The plain FP64 form (IEEE double on the FP64 units, the native candidate
    of the fused variant) of the headline workload, per forward and backward
    transform at each P, beside the tuned FP64-accurate one."""
    out = {}
    N = x.numel()
    for P, h in plans.items():
        cur = of.openfft_current_candidate(h)
        nat = [i for i in range(of.openfft_num_candidates(h))
               if of.openfft_candidate(h, i)["arith"] == of.ARITH_NATIVE
               and of.openfft_candidate(h, i)["variant"] == of.VARIANT_FUSED]
        best = None
        for ci in nat[:2]:
            of.openfft_set_tuning(h, of.TUNE_USER, ci)
            ts = {}
            for d, name in ((of.FORWARD, "fwd"), (of.BACKWARD, "bwd")):
                of.openfft_exec_c2c(h, x, y, d)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    of.openfft_exec_c2c(h, x, y, d)
                e1.record(stream)
                e1.synchronize()
                ts[name] = e0.elapsed_time(e1) / reps
            if best is None or ts["fwd"] + ts["bwd"] < best[0]["fwd"] + best[0]["bwd"]:
                best = (ts, of.openfft_candidate(h, ci))
        of.openfft_set_tuning(h, of.TUNE_USER, cur)
        ms = (best[0]["fwd"] + best[0]["bwd"]) / 2
        out[str(P)] = {"fwd_ms": round(best[0]["fwd"], 3), "bwd_ms": round(best[0]["bwd"], 3),
                       "gflops": round(flops(N) / ms / 1e6, 1),
                       "hbm_frac": round(6 * N * 16 / (ms * 1e-3) / 1e9 / load_peaks()[0], 4),
                       "chosen": best[1]}
    return out


def measure_256_step(of, torch, stream, args, world):
    """The 256^3 configuration: forward + backward at P = 16, 64, 256 per step,
    timed like the headline (its own value, roofline and round trip)."""
    from paper_1501_07350_gb300 import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    n = N256
    N = n ** 3
    x = torch.from_numpy(synth.complex_field((N,), seed=synth.config_seed(2), dist="normal")).to(dev)
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    m = time_step(of, torch, n, PS256, x, y, z, stream, args, world)
    ms_per_step = reduce_max(m["ms_total"], world, dev) / args.steps
    out = {"workload": WORKLOAD256, "value": round(job_value(2 * len(PS256) * flops(N), world, ms_per_step), 2),
           "unit": UNIT, "ms_per_step": round(ms_per_step, 4),
           "roofline": stage_roofline(of, torch, dev, n, m["chosen"], m["phases"], None),
           "round_trip_rel_l2": float(torch.linalg.vector_norm(z - x) / torch.linalg.vector_norm(x)),
           "chosen": {str(P): c for P, c in m["chosen"].items()}}
    return out, m["plans"], x, y, z


def measure_forms(of, torch, stream, args, world):
    """The 256^3 step, then per-transform GFLOP/s of each form on the 256^3
    input (median of 5), and the batched, mixed-radix, real and learned forms."""
    step256, plans_f64, x, y, z = measure_256_step(of, torch, stream, args, world)
    n = N256
    N = n ** 3
    out = {"step_256cubed": step256}

    def time_exec(h, a, b, direction, reps=5):
        ts = []
        for _ in range(2):
            of.openfft_exec_c2c(h, a, b, direction)
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            of.openfft_exec_c2c(h, a, b, direction)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    h = plans_f64[64]
    cur = of.openfft_current_candidate(h)
    for ci in range(of.openfft_num_candidates(h)):
        c = of.openfft_candidate(h, ci)
        if c["variant"] != of.VARIANT_FUSED:
            continue
        of.openfft_set_tuning(h, of.TUNE_USER, ci)
        ms = time_exec(h, x, y, of.FORWARD)
        key = "f64_%s_G%d_%s" % ("native" if c["arith"] == of.ARITH_NATIVE else "doublefloat", c["lines_per_cta"],
                                 ["auto", "warp", "tile", "generic"][c["kernel"]])
        out[key] = {"ms": round(ms, 4), "gflops": round(flops(N) / ms / 1e6, 1),
                    "hbm_frac": round(6 * N * 16 / (ms * 1e-3) / 1e9 / load_peaks()[0], 4)}
    for vi, name in [(of.VARIANT_PACK_UNPACK, "V1"), (of.VARIANT_PACK_EXCHANGE_UNPACK, "V0")]:
        for ci in range(of.openfft_num_candidates(h)):
            c = of.openfft_candidate(h, ci)
            if c["variant"] == vi and c["arith"] == of.ARITH_DOUBLE_FLOAT:
                of.openfft_set_tuning(h, of.TUNE_USER, ci)
                ms = time_exec(h, x, y, of.FORWARD)
                out["f64_doublefloat_%s" % name] = {"ms": round(ms, 4), "gflops": round(flops(N) / ms / 1e6, 1)}
    of.openfft_set_tuning(h, of.TUNE_USER, cur)
    # the paper's communication methods as transpose variants (Sec. 3.2.1), double-float
    # arithmetic, at every P of the workload: which one wins where
    names = {of.VARIANT_PACK_EXCHANGE_UNPACK: "Alltoallv (V0: pack, exchange, unpack)",
             of.VARIANT_PACK_UNPACK: "Isend_Waitsome (V1: unpack from the send segments)",
             of.VARIANT_ISEND_WAITALL: "Isend_Waitall (P exchange steps)",
             of.VARIANT_ISEND_WAITALL_BLOCK: "Isend_Waitall_Block (B_SIZE = 32 groups)",
             of.VARIANT_ISEND_WAITSOME_BLOCK: "Isend_Waitsome_Block",
             of.VARIANT_SENDRECV: "Sendrecv (P shifted steps)",
             of.VARIANT_FUSED: "fused into the stage stores (V2)"}
    methods = {}
    for P, hp in plans_f64.items():
        curp = of.openfft_current_candidate(hp)
        row = {}
        for ci in range(of.openfft_num_candidates(hp)):
            c = of.openfft_candidate(hp, ci)
            if c["arith"] != of.ARITH_DOUBLE_FLOAT or c["kernel"] != 0 or c["lines_per_cta"] != 8:
                continue
            of.openfft_set_tuning(hp, of.TUNE_USER, ci)
            row[names[c["variant"]]] = round(time_exec(hp, x, y, of.FORWARD, reps=3), 4)
        of.openfft_set_tuning(hp, of.TUNE_USER, curp)
        methods[str(P)] = {"ms": row, "fastest": min(row, key=row.get),
                           "fastest_explicit": min((k for k in row if "V2" not in k), key=row.get)}
    out["exchange_methods_256cubed_fwd"] = methods
    # the small configuration: 32^3 complex128, P = 4, one forward transform (latency-bound)
    from paper_1501_07350_gb300 import synth as _synth
    xs = torch.from_numpy(_synth.complex_field((32, 32, 32), seed=_synth.config_seed(1))).to(x.device)
    ys = torch.empty_like(xs)
    hs = of.openfft_plan(32, 32, 32, 4, of.C2C_F64)
    of.openfft_set_stream(hs, stream)
    of.openfft_set_tuning(hs, of.TUNE_EXHAUSTIVE)
    ms_s = time_exec(hs, xs, ys, of.FORWARD, reps=20)
    out["small_32cubed_P4_fwd"] = {"us": round(ms_s * 1e3, 2), "gflops": round(flops(32 ** 3) / ms_s / 1e6, 2),
                                   "chosen": of.openfft_candidate(hs, of.openfft_current_candidate(hs)),
                                   "note": "latency-bound (3 launches of 512 KiB); no roofline fraction"}
    of.openfft_destroy(hs)
    # FP32 form (complex64), auto-tuned
    x32 = x.to(torch.complex64)
    y32 = torch.empty_like(x32)
    h32 = of.openfft_plan(n, n, n, 64, of.C2C_F32)
    of.openfft_set_stream(h32, stream)
    of.openfft_set_tuning(h32, of.TUNE_EXHAUSTIVE)
    ms = time_exec(h32, x32, y32, of.FORWARD)
    ref = torch.empty_like(y)
    of.openfft_exec_c2c(h, x, ref, of.FORWARD)
    torch.cuda.synchronize()
    err = float(torch.linalg.vector_norm(y32.to(torch.complex128) - ref) / torch.linalg.vector_norm(ref))
    out["f32"] = {"ms": round(ms, 4), "gflops": round(flops(N) / ms / 1e6, 1),
                  "hbm_frac": round(6 * N * 8 / (ms * 1e-3) / 1e9 / load_peaks()[0], 4),
                  "rel_l2_vs_f64": err, "bound": 1e-5,
                  "chosen": of.openfft_candidate(h32, of.openfft_current_candidate(h32))}
    of.openfft_destroy(h32)
    del x32, y32
    # batched: 64 uneven transforms (sizes drawn from {48^3, 64^3, 96^3, 100x108x120}),
    # complex64, P = 8 each, one persistent graph launch -- against the same 64
    # transforms run one plan at a time in FP64 and in FP32
    if not args.no_batch:
        out["batch64"] = measure_batch(of, torch, stream)
    # non-power-of-two 120 x 144 x 160, P = 32: FP64 vs FP32 vs split tensor-core forms
    out["mixed_120x144x160"] = measure_mixed(of, torch, stream)
    # real transforms at 256^3 against the complex transform
    out["r2c_256cubed"] = measure_r2c(of, torch, stream)
    for hp in plans_f64.values():
        of.openfft_destroy(hp)
    del x, y, z
    torch.cuda.empty_cache()
    if not args.no_512:
        # the learned selector against exhaustive autotuning at 512^3
        out["learned_vs_exhaustive_512cubed"] = measure_learned(of, torch, stream)
    return out


def measure_mixed(of, torch, stream, reps=7):
    """Non-power-of-two 120 x 144 x 160 at P = 32: FP64 (native and double-float,
    each its best candidate), FP32, and the split tf32 / bf16 tensor-core
    DFT-GEMM forms, per forward transform.  The complex128 array (44 MB) fits
    in L2, so a 256 MiB buffer is written between timed reps.  Errors are
    against the FP64 result on the same seeded uniform[-1,1) input (complex64
    for the reduced forms) and, for a plane wave, against its closed form."""
    from paper_1501_07350_gb300 import synth
    Na, Nb, Nc, P = 120, 144, 160, 32
    N = Na * Nb * Nc
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    x64 = torch.from_numpy(synth.complex_field((N,), seed=synth.config_seed(3))).to(dev)
    x32 = x64.to(torch.complex64)
    k0 = (59, 71, 79)
    pw = torch.from_numpy(synth.plane_wave(Na, Nb, Nc, k0).reshape(-1)).to(dev)

    def timed(h, a, b):
        for _ in range(3):
            of.openfft_exec_c2c(h, a, b, of.FORWARD)
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            of.openfft_exec_c2c(h, a, b, of.FORWARD)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        of.openfft_sync(h)
        return statistics.median(ts)

    def rel(a, b):
        return float(torch.linalg.vector_norm(a.to(torch.complex128) - b) / torch.linalg.vector_norm(b))

    def plane_wave_err(h, dt):
        y = torch.empty_like(pw, dtype=dt)
        of.openfft_exec_c2c(h, pw.to(dt), y, of.FORWARD)
        of.openfft_sync(h)
        y = y.to(torch.complex128)
        # forward output is cba-ordered: (kc, kb, ka) -> index (kc * Nb + kb) * Na + ka
        idx = (k0[2] * Nb + k0[1]) * Na + k0[0]
        y[idx] -= N
        return float(torch.linalg.vector_norm(y)) / (N * math.sqrt(N))

    peak = load_peaks()[0]
    out = {"shape": [Na, Nb, Nc], "P": P, "l2": "256 MiB written between reps"}
    h = of.openfft_plan(Na, Nb, Nc, P, of.C2C_F64)
    of.openfft_set_stream(h, stream)
    ref = torch.empty_like(x64)
    for arith, name in [(of.ARITH_NATIVE, "f64_native"), (of.ARITH_DOUBLE_FLOAT, "f64_doublefloat")]:
        best = None
        for ci in range(of.openfft_num_candidates(h)):
            c = of.openfft_candidate(h, ci)
            if c["arith"] != arith or c["variant"] != of.VARIANT_FUSED:
                continue
            of.openfft_set_tuning(h, of.TUNE_USER, ci)
            ms = timed(h, x64, ref)
            if best is None or ms < best[0]:
                best = (ms, c)
        out[name] = {"ms": round(best[0], 4), "gflops": round(flops(N) / best[0] / 1e6, 1),
                     "hbm_frac": round(6 * N * 16 / (best[0] * 1e-3) / 1e9 / peak, 4), "chosen": best[1]}
    of.openfft_set_tuning(h, of.TUNE_USER, [i for i in range(of.openfft_num_candidates(h))
                                            if of.openfft_candidate(h, i)["arith"] == of.ARITH_NATIVE][0])
    of.openfft_exec_c2c(h, x64, ref, of.FORWARD)
    of.openfft_sync(h)
    out["f64_native"]["plane_wave_err"] = plane_wave_err(h, torch.complex128)
    of.openfft_destroy(h)
    for dtype, name, bound in [(of.C2C_F32, "f32", 1e-5), (of.C2C_SPLIT_TF32, "split_tf32_tc", 1e-5),
                               (of.C2C_SPLIT_BF16, "split_bf16_tc", 1e-4)]:
        h = of.openfft_plan(Na, Nb, Nc, P, dtype)
        of.openfft_set_stream(h, stream)
        of.openfft_set_tuning(h, of.TUNE_EXHAUSTIVE)
        y = torch.empty_like(x32)
        ms = timed(h, x32, y)
        out[name] = {"ms": round(ms, 4), "gflops": round(flops(N) / ms / 1e6, 1),
                     "hbm_frac": round(6 * N * 8 / (ms * 1e-3) / 1e9 / peak, 4),
                     "rel_l2_vs_f64": rel(y, ref), "plane_wave_err": plane_wave_err(h, torch.complex64),
                     "bound": bound, "chosen": of.openfft_candidate(h, of.openfft_current_candidate(h))}
        of.openfft_destroy(h)
    del flush
    torch.cuda.empty_cache()
    return out


def measure_learned(of, torch, stream, Ps=(64, 256, 1024), reps=5):
    """512^3 complex128 (held out of the cost model's training set): the
    candidate the learned selector proposes against exhaustive autotuning
    (the paper's run-time choice), both timed by the same protocol; regret =
    t_learned / t_exhaustive - 1.  Also the host time each way of choosing
    takes (exhaustive: two timed runs of every candidate; learned: one model
    evaluation per candidate)."""
    from paper_1501_07350_gb300 import learned, synth
    learned.install()
    n = 512
    N = n ** 3
    dev = torch.device("cuda", torch.cuda.current_device())
    torch.cuda.empty_cache()
    x = torch.from_numpy(synth.complex_field((N,), seed=synth.config_seed(5))).to(dev)
    y = torch.empty_like(x)

    def timed(h, ci):
        of.openfft_set_tuning(h, of.TUNE_USER, ci)
        for _ in range(2):
            of.openfft_exec_c2c(h, x, y, of.FORWARD)
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            of.openfft_exec_c2c(h, x, y, of.FORWARD)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    out = {"shape": [n, n, n], "dtype": "complex128", "held_out": True, "per_P": {}}
    regrets = []
    for P in Ps:
        h = of.openfft_plan(n, n, n, P, of.C2C_F64)
        of.openfft_set_stream(h, stream)
        t0 = time.perf_counter()
        of.openfft_set_tuning(h, of.TUNE_EXHAUSTIVE)
        tune_ex = time.perf_counter() - t0
        ci_ex = of.openfft_current_candidate(h)
        t0 = time.perf_counter()
        of.openfft_set_tuning(h, of.TUNE_LEARNED)
        tune_l = time.perf_counter() - t0
        ci_l = of.openfft_current_candidate(h)
        t_ex, t_l, t_def = timed(h, ci_ex), timed(h, ci_l), timed(h, 0)
        # the same candidate is the same launch sequence: its regret is 0 and
        # the two timings differ by measurement noise only
        same = ci_l == ci_ex
        regret = 0.0 if same else t_l / t_ex - 1.0
        regrets.append(regret)
        out["per_P"][str(P)] = {"exhaustive": {"candidate": of.openfft_candidate(h, ci_ex), "ms": round(t_ex, 3),
                                               "tuning_s": round(tune_ex, 3)},
                                "learned": {"candidate": of.openfft_candidate(h, ci_l), "ms": round(t_l, 3),
                                            "tuning_s": round(tune_l, 4)},
                                "default_ms": round(t_def, 3), "regret": round(regret, 4), "same_choice": same,
                                "timing_noise": round(t_l / t_ex - 1.0, 4) if same else None,
                                "candidates": of.openfft_num_candidates(h)}
        of.openfft_destroy(h)
    out["mean_regret"] = round(sum(regrets) / len(regrets), 4)
    out["max_regret"] = round(max(regrets), 4)
    out["target"] = "within 5% of exhaustive autotuning"
    # the committed dataset: regret on the held-out benchmark problems, and on
    # whole shape families held out of training (models trained on the GPU here)
    rows = learned.load_rows()
    tr, te = learned.split(rows)
    ps, _ = learned.train(tr)
    ev = learned.evaluate(te, ps)
    out["dataset_held_out"] = {"summary": learned.summary(ev),
                               "per_problem": [{"shape": e["shape"], "P": e["P"], "dtype": e["dtype"],
                                                "regret": round(e["regret"], 4),
                                                "speedup_vs_default": round(e["speedup_vs_default"], 4)}
                                               for e in ev]}
    out["family_held_out"] = {k: {"train_problems": v["train_problems"], "summary": v["summary"],
                                  "per_problem": [{"shape": e["shape"], "P": e["P"], "dtype": e["dtype"],
                                                   "regret": round(e["regret"], 4)} for e in v["problems"]]}
                              for k, v in learned.evaluate_families(rows).items()}
    del x, y
    torch.cuda.empty_cache()
    return out


def measure_r2c(of, torch, stream, n=256, P=64, reps=5):
    """Real transforms at n^3 (real abc array -> half spectrum [n/2+1][n][n] and
    back), FP64-accurate and FP32, against the complex transform of the same
    input.  GFLOP/s in the 2.5 N log2 N convention of real transforms;
    algorithmic bytes: the real array read (write) once plus three passes of
    the half array (stage 1 writes it, stages 2 and 3 read and write it)."""
    from paper_1501_07350_gb300 import synth
    N = n ** 3
    Nh = (n // 2 + 1) * n * n
    dev = torch.device("cuda", torch.cuda.current_device())
    x64 = torch.from_numpy(synth.normal(synth.config_seed(2), N)).to(dev)
    peak = load_peaks()[0]

    def timed(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    out = {"shape": [n, n, n], "P": P, "flops": "2.5 N log2 N"}
    for dtype, name, rt, ct, E, R in [(of.R2C_F64, "f64", torch.float64, torch.complex128, 16, 8),
                                      (of.R2C_F32, "f32", torch.float32, torch.complex64, 8, 4)]:
        x = x64.to(rt)
        h = torch.empty(Nh, dtype=ct, device=dev)
        xb = torch.empty_like(x)
        plan = of.openfft_plan(n, n, n, P, dtype)
        of.openfft_set_stream(plan, stream)
        of.openfft_set_tuning(plan, of.TUNE_EXHAUSTIVE)
        ms_f = timed(lambda: of.openfft_exec_r2c(plan, x, h))
        ms_b = timed(lambda: of.openfft_exec_c2r(plan, h, xb))
        of.openfft_sync(plan)
        err = float(torch.linalg.vector_norm(xb - x) / torch.linalg.vector_norm(x))
        alg = R * N + 5 * E * Nh
        out[name] = {"r2c_ms": round(ms_f, 4), "c2r_ms": round(ms_b, 4),
                     "r2c_gflops": round(2.5 * N * math.log2(N) / ms_f / 1e6, 1),
                     "r2c_hbm_frac": round(alg / (ms_f * 1e-3) / 1e9 / peak, 4),
                     "c2r_hbm_frac": round(alg / (ms_b * 1e-3) / 1e9 / peak, 4),
                     "round_trip_rel_l2": err,
                     "chosen": of.openfft_candidate(plan, of.openfft_current_candidate(plan))}
        of.openfft_destroy(plan)
        # the complex transform of the same (real) input, for comparison
        xc = x.to(ct)
        yc = torch.empty_like(xc)
        cp = of.openfft_plan(n, n, n, P, of.C2C_F64 if dtype == of.R2C_F64 else of.C2C_F32)
        of.openfft_set_stream(cp, stream)
        of.openfft_set_tuning(cp, of.TUNE_EXHAUSTIVE)
        out[name]["c2c_forward_ms"] = round(timed(lambda: of.openfft_exec_c2c(cp, xc, yc, of.FORWARD)), 4)
        of.openfft_destroy(cp)
        del x, h, xb, xc, yc
    torch.cuda.empty_cache()
    return out


def measure_batch(of, torch, stream, count=64, reps=5):
    from paper_1501_07350_gb300 import synth
    shapes = synth.batch_shapes(synth.config_seed(4), count)
    Ps = [8] * count
    work = sum(flops(a * b * c) for a, b, c in shapes)
    bytes64 = sum(48 * a * b * c for a, b, c in shapes)
    xs = [torch.from_numpy(synth.complex_field((a * b * c,), seed=synth.config_seed(4) + 1 + i)).cuda()
          for i, (a, b, c) in enumerate(shapes)]
    x32 = [x.to(torch.complex64) for x in xs]
    y32 = [torch.empty_like(x) for x in x32]

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    res = {"transforms": count, "points": int(sum(a * b * c for a, b, c in shapes)), "gflop": round(work / 1e9, 3)}
    hb = of.openfft_plan_many(shapes, Ps, of.C2C_F32)
    of.openfft_set_stream(hb, stream)
    ms = timed(lambda: of.openfft_exec_many(hb, x32, y32, of.FORWARD))
    of.openfft_sync(hb)
    # accuracy of the batched form against the per-transform FP64 plans (checked below)
    res["batched_c64_graph"] = {"ms": round(ms, 4), "gflops": round(work / ms / 1e6, 1),
                                "hbm_frac": round(bytes64 / (ms * 1e-3) / 1e9 / load_peaks()[0], 4)}
    plans64 = []
    for (a, b, c) in shapes:
        h = of.openfft_plan(a, b, c, 8, of.C2C_F64)
        of.openfft_set_stream(h, stream)
        of.openfft_set_tuning(h, of.TUNE_USER, [i for i in range(of.openfft_num_candidates(h))
                                                if of.openfft_candidate(h, i)["arith"] == of.ARITH_NATIVE][0])
        plans64.append(h)
    y64 = [torch.empty_like(x) for x in xs]

    def run64():
        for h, x, y in zip(plans64, xs, y64):
            of.openfft_exec_c2c(h, x, y, of.FORWARD)
    ms64 = timed(run64)
    res["per_transform_f64_native"] = {"ms": round(ms64, 4), "gflops": round(work / ms64 / 1e6, 1)}
    errs = [float(torch.linalg.vector_norm(a.to(torch.complex128) - b) / torch.linalg.vector_norm(b))
            for a, b in zip(y32, y64)]
    res["batched_c64_graph"]["max_rel_l2_vs_f64"] = max(errs)
    res["batched_c64_graph"]["bound"] = 1e-5
    for h in plans64:
        of.openfft_destroy(h)
    plans32 = []
    for (a, b, c) in shapes:
        h = of.openfft_plan(a, b, c, 8, of.C2C_F32)
        of.openfft_set_stream(h, stream)
        plans32.append(h)

    def run32():
        for h, x, y in zip(plans32, x32, y32):
            of.openfft_exec_c2c(h, x, y, of.FORWARD)
    ms32 = timed(run32)
    res["per_transform_c64"] = {"ms": round(ms32, 4), "gflops": round(work / ms32 / 1e6, 1)}
    for h in plans32:
        of.openfft_destroy(h)
    of.openfft_destroy(hb)
    return res


def host_threads(per_thread_bytes):
    """Threads for the oracle baseline: every host core this process may run on,
    fewer if the host memory would not hold one transform's working set per thread."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    avail = None
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    if avail is None:
        return 1
    return max(1, min(cores, int(avail * 0.6 // per_thread_bytes)))


def oracle_concurrent(x_box, shape, threads, first_p=0):
    """`threads` forward transforms of the array x_box (flat, `shape`) by the
    FP64 oracle, one per thread and all at once (the oracle is a C library
    called through ctypes, which releases the GIL, so the threads run on
    separate cores); P cycles over the headline's 64 / 256 / 1024.  Returns
    the wall time in seconds."""
    import threading

    import oracle
    errors = []
    Na, Nb, Nc = shape

    def work(i):
        try:
            oracle.fft3d(x_box, Na, Nb, Nc, PS[(first_p + i) % len(PS)], oracle.FORWARD)
        except Exception as e:          # reported after the join
            errors.append(e)
    ts = [threading.Thread(target=work, args=(i,)) for i in range(threads)]
    t0 = time.perf_counter()
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    dt = time.perf_counter() - t0
    if errors:
        raise errors[0]
    return dt


def oracle_bytes(shape) -> int:
    """Host bytes one oracle transform holds: input, output, two stage arrays,
    and the send / receive segments of a redistribution (values and indices)."""
    return int(np.prod(shape)) * (16 * 6 + 8 * 2)


def sample_box(x_np):
    """The oracle's sample of the headline input: its first 64 a-planes, a
    64 x 512 x 512 array (an eighth of the volume, the same 512-point lines)."""
    return np.ascontiguousarray(x_np[:int(np.prod(SAMPLE_SHAPE))])


def cpu_baseline_sample(x_np, n):
    """The FP64 oracle on the host cores, on a bounded sample of the headline
    workload: one forward transform of the 64 x 512 x 512 box per thread, all
    threads at once; and one thread on the same box for comparison."""
    box = sample_box(x_np)
    Nbox = int(np.prod(SAMPLE_SHAPE))
    threads = host_threads(oracle_bytes(SAMPLE_SHAPE))
    dt = oracle_concurrent(box, SAMPLE_SHAPE, threads)
    dt1 = oracle_concurrent(box, SAMPLE_SHAPE, 1)
    return {"value": round(threads * flops(Nbox) / dt / 1e9, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d forward transforms of the 64x512x512 box of the 512^3 input (its first 64 a-planes), "
                      "P = 64 / 256 / 1024, one per thread, run at once (%.1f s wall); one transform on one "
                      "thread: %.4f GFLOP/s (%.1f s)" % (threads, dt, flops(Nbox) / dt1 / 1e9, dt1)}


# ------------------------------------------------------------ reference --

def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    from paper_1501_07350_gb300 import synth
    n = N1D
    x = synth.complex_field((n ** 3,), seed=synth.config_seed(5))
    box = sample_box(x)
    del x
    Nbox = int(np.prod(SAMPLE_SHAPE))
    oracle.build()
    threads = host_threads(oracle_bytes(SAMPLE_SHAPE))
    times = []
    for i in range(args.warmup + args.steps):
        dt = oracle_concurrent(box, SAMPLE_SHAPE, threads, first_p=i)
        if i >= args.warmup:
            times.append(dt)
    t = sum(times) / len(times)
    value = threads * flops(Nbox) / t / 1e9
    sample = ("%d forward transforms per step of the 64x512x512 box of the 512^3 input (its first 64 a-planes), "
              "one per host thread, P cycling 64/256/1024" % threads)
    res = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t * 1e3, 2),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "shape": [n, n, n], "P": list(PS), "transforms_per_step": 6,
                      "sample": sample},
           "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)


def run_single(args, local_rank):
    """One form on one shape, forward only: a small, fixed command for profilers."""
    import torch

    from paper_1501_07350_gb300 import _build
    from paper_1501_07350_gb300 import openfft as of
    from paper_1501_07350_gb300 import synth

    _build.build()
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else (args.n,) * 3
    N = shape[0] * shape[1] * shape[2]
    dtype = {"f32": of.C2C_F32, "tf32": of.C2C_SPLIT_TF32, "bf16": of.C2C_SPLIT_BF16}.get(args.form, of.C2C_F64)
    want_arith = {"f64-df": of.ARITH_DOUBLE_FLOAT, "tf32": of.ARITH_TC_TF32,
                  "bf16": of.ARITH_TC_BF16}.get(args.form, of.ARITH_NATIVE)
    tc_form = want_arith in (of.ARITH_TC_TF32, of.ARITH_TC_BF16)
    want_variant = {"fused": of.VARIANT_FUSED, "v1": of.VARIANT_PACK_UNPACK,
                    "v0": of.VARIANT_PACK_EXCHANGE_UNPACK}[args.variant]
    x = torch.from_numpy(synth.complex_field((N,), seed=synth.config_seed(2))).cuda()
    if dtype != of.C2C_F64:
        x = x.to(torch.complex64)
    y = torch.empty_like(x)
    h = of.openfft_plan(shape[0], shape[1], shape[2], args.P, dtype)
    of.openfft_set_stream(h, stream)
    pick = None
    for ci in range(of.openfft_num_candidates(h)):
        c = of.openfft_candidate(h, ci)
        if tc_form:
            if c["arith"] == want_arith and c["lines_per_cta"] == args.G:
                pick = ci
        elif (c["variant"] == want_variant and c["arith"] == want_arith and c["lines_per_cta"] == args.G
                and (want_variant != of.VARIANT_FUSED
                     or c["kernel"] == {"auto": 0, "warp": 0, "tile": 2, "generic": 3}[args.kernel])):
            pick = ci
    if pick is None:
        raise SystemExit("no such candidate")
    of.openfft_set_tuning(h, of.TUNE_USER, pick)
    for _ in range(args.warmup):
        of.openfft_exec_c2c(h, x, y, of.FORWARD)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        of.openfft_exec_c2c(h, x, y, of.FORWARD)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    E = 16 if dtype == of.C2C_F64 else 8
    print(json.dumps({"single": args.form, "shape": list(shape), "P": args.P, "variant": args.variant,
                      "G": args.G, "kernel": args.kernel,
                      "ms": round(ms, 4), "gflops": round(flops(N) / ms / 1e6, 1),
                      "hbm_frac": round(6 * N * E / (ms * 1e-3) / 1e9 / load_peaks()[0], 4)}))
    of.openfft_destroy(h)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--tune", choices=["exhaustive", "default"], default="exhaustive")
    ap.add_argument("--quick", action="store_true", help="skip the other forms")
    ap.add_argument("--no-512", dest="no_512", action="store_true", help="skip the 512^3 form")
    ap.add_argument("--no-batch", dest="no_batch", action="store_true", help="skip the batched form")
    ap.add_argument("--only-batch", dest="only_batch", action="store_true", help="time the batched form only")
    ap.add_argument("--only-r2c", dest="only_r2c", action="store_true", help="time the real transforms only")
    ap.add_argument("--only-learned", dest="only_learned", action="store_true",
                    help="time the learned selector against exhaustive autotuning at 512^3 only")
    ap.add_argument("--only-mixed", dest="only_mixed", action="store_true",
                    help="time the 120x144x160 FP64 / FP32 / split tensor-core forms only")
    ap.add_argument("--no-cpu-baseline", dest="no_cpu_baseline", action="store_true")
    ap.add_argument("--single", action="store_true",
                    help="time one form on one n^3 shape (forward only), for profiling")
    ap.add_argument("--form", choices=["f64-native", "f64-df", "f32", "tf32", "bf16"], default="f64-df")
    ap.add_argument("--variant", choices=["fused", "v1", "v0"], default="fused")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--shape", default="", help="Na,Nb,Nc (overrides --n)")
    ap.add_argument("--P", type=int, default=64)
    ap.add_argument("--G", type=int, default=8)
    ap.add_argument("--kernel", choices=["auto", "warp", "tile", "generic"], default="auto")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)     # at least 3 warm-up steps; the count run is reported
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.single:
        run_single(args, local_rank)
        return
    if args.only_batch:
        import torch
        from paper_1501_07350_gb300 import _build
        from paper_1501_07350_gb300 import openfft as of
        _build.build()
        torch.cuda.set_device(local_rank)
        print(json.dumps({"batch64": measure_batch(of, torch, torch.cuda.current_stream())}))
        return
    if args.only_r2c:
        import torch
        from paper_1501_07350_gb300 import _build
        from paper_1501_07350_gb300 import openfft as of
        _build.build()
        torch.cuda.set_device(local_rank)
        print(json.dumps({"r2c_256cubed": measure_r2c(of, torch, torch.cuda.current_stream())}))
        return
    if args.only_learned:
        import torch
        from paper_1501_07350_gb300 import _build
        from paper_1501_07350_gb300 import openfft as of
        _build.build()
        torch.cuda.set_device(local_rank)
        print(json.dumps({"learned_vs_exhaustive_512cubed": measure_learned(of, torch, torch.cuda.current_stream())}))
        return
    if args.only_mixed:
        import torch
        from paper_1501_07350_gb300 import _build
        from paper_1501_07350_gb300 import openfft as of
        _build.build()
        torch.cuda.set_device(local_rank)
        print(json.dumps({"mixed_120x144x160": measure_mixed(of, torch, torch.cuda.current_stream())}))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
