#!/usr/bin/env python3
"""Benchmark: effective bop/s (2mkn/t) of the GF(2) and Boolean bit-matrix
products on square seeded Bernoulli inputs, through the C ABI.

One step = one GF(2) product (through the alternative-basis Strassen
recursion, depth chosen by the planner) plus one Boolean product (cubic), both
at m = k = n = 32768 by default. Inputs are resident in HBM before the timed
region; the step touches ~1.7 GB (> L2), so no L2 flush is needed between
steps. `value` counts 2*m*k*n bit operations per product.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs the same workload on its own GPU
(independent replicas, weak scaling); rank 0 prints one JSON line.
--impl reference times the CPU oracle on a bounded row sample instead.
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

METRIC = "effective bop/s (2mkn/t) Boolean & GF(2) products, tensor-core vs popcount path"

# name: (n, seed, Boolean density); GF(2) operands are dense (p = 1/2).
WORKLOADS = {
    "square32768": (32768, 2, "2^-7.5"),
    "square65536": (65536, 3, "2^-8"),
    "square524288": (524288, 4, "2^-9.5"),
    # 2048 problems, m, k, n log-uniform in [256, 8192] (multiples of 64), 50/50
    # GF(2) (p = 1/2) / Boolean (p = 1/sqrt(k)); problem i uses seed 5 * 2^16 + i
    "batched2048": (2048, 5, "1/sqrt(k)"),
    # operands and products in pinned host memory, through the host layer with
    # a device budget below the product's in-HBM footprint (out of core)
    "host65536": (65536, 3, "2^-8"),
}
HOST_DEVICE_BYTES = {"host65536": 3 << 30}
DEFAULT_WORKLOAD = "square32768"
# Matrix ids of the generator streams: GF(2) pair (0, 1), Boolean pair (4, 5).
IDS_GF2 = (0, 1)
IDS_BOOL = (4, 5)

# 32-bit LOP3 results per SM per clock on sm_103 (measured with a
# dependent-chain microbenchmark; IMAD also 64, POPC 16).
LOP3_LANES_PER_SM_CLK = 64
# Nominal dense FP8 : BF16 tensor throughput ratio (4.5 : 2.25 PFLOP/s).
FP8_PER_BF16 = 2.0
# Nominal dense FP4 : BF16 tensor throughput ratio (13.5 : 2.25 PFLOP/s).
FP4_PER_BF16 = 6.0
# FP8 MACs per clock per SM of tcgen05.mma kind::f8f6f4 on sm_103 (measured
# with back-to-back MMAs); 2 FLOP each.
FP8_MAC_PER_SM_CLK = 8192
# FP4 MACs per clock per SM of tcgen05.mma kind::mxf4 (block scale every 32 k)
# on sm_103 (measured with back-to-back MMAs: twice the FP8 rate).
FP4_MAC_PER_SM_CLK = 16384

# DRAM bytes (read + write) of the base-case launches of one step of the
# default workload, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum; profiles/tc_nt_kernel_square32768_traffic.md). It
# holds only for the kernel source it was taken on and the same launches
# (GF(2) depth 3 with one depth-first level: 7 leaf launches + 1 Boolean).
TRAFFIC_RECORD = {
    "kernel": "paper_1909_01554_gb300/csrc/tc_gemm.cu",
    "sha256": "ca977e867ceb42cea71dffdae50cae4403355d59c57737e9f8a3bc5846ee2dd2",
    "workload": "square32768", "gf2_depth": 3, "gf2_serial": 1, "base_launches": 8,
    "dram_bytes_per_step": 2781064192,
}


def recorded_traffic(workload: str, depth: int, serial: int, launches_per_step: float):
    """Bytes per base-case launch from the ncu record, or None when the kernel
    source or the launch composition differs from what was captured."""
    import hashlib

    r = TRAFFIC_RECORD
    try:
        with open(os.path.join(ROOT, r["kernel"]), "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    if (digest != r["sha256"] or workload != r["workload"] or depth != r["gf2_depth"]
            or serial != r["gf2_serial"] or launches_per_step != r["base_launches"]):
        return None
    return r["dram_bytes_per_step"] / r["base_launches"]


def tensor_pipe(achieved: float, clocks: dict, fallback_mhz: float, fp4: bool = False) -> dict:
    """The tensor pipe's own limit at the clock seen under load, beside the
    measured-peak roofline."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = (clocks or {}).get("sm_mhz") or fallback_mhz
    macs, kind = (FP4_MAC_PER_SM_CLK, "fp4") if fp4 else (FP8_MAC_PER_SM_CLK, "fp8")
    pp = sms * macs * 2 * mhz * 1e6 / 1e12
    return {"pipe_peak": pp, "pipe_frac": achieved / pp,
            "pipe_peak_source": f"{sms} SMs x {macs} {kind} MAC/clk x 2 x "
                                f"{mhz} MHz (median under load)"}


def strassen_bound(pl: dict, m: int, n: int, product_ms: float, peak: float,
                   hbm_gbs: float, pipe_peak: float = None) -> dict:
    """The Strassen path's bound for one binary product: its leaves' work at
    the base case's peak (TFLOP/s, or Tbop/s on the CUDA cores: 2 per MAC
    either way) plus its streaming passes' bytes (transpose, padding, every
    XOR pass) at the measured HBM bandwidth, against the measured product."""
    d = pl["strassen_depth"]
    work = 2 * pl["leaves"] * (m >> d) * (pl["kp"] >> d) * (n >> d)
    base_ms = work / (peak * 1e12) * 1e3
    pass_ms = pl["pass_bytes"] / (hbm_gbs * 1e9) * 1e3
    out = {"leaf_work": work, "pass_bytes": pl["pass_bytes"], "peak": peak, "hbm_gbs": hbm_gbs,
           "bound_ms": base_ms + pass_ms, "base_bound_ms": base_ms, "pass_bound_ms": pass_ms,
           "product_ms": product_ms, "frac": (base_ms + pass_ms) / product_ms}
    if pipe_peak:
        pb = work / (pipe_peak * 1e12) * 1e3 + pass_ms
        out.update({"pipe_bound_ms": pb, "pipe_frac": pb / product_ms})
    return out


def tensor_peak(pk: dict, pk_kind: str, fp4: bool):
    """Measured bf16 peak scaled to the operand type by the nominal ratio."""
    ratio, kind = (FP4_PER_BF16, "fp4") if fp4 else (FP8_PER_BF16, "fp8")
    return (pk["bf16_tflops_sustained"] * ratio,
            f"{pk_kind} bf16 sustained x {ratio} (nominal {kind}:bf16)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--path", choices=["auto", "fp8", "fp8pair", "fp4pair", "i8", "popc"],
                    default="auto")
    ap.add_argument("--depth", type=int, default=-1, help="Strassen depth of the GF(2) product")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="planner rules instead of the autotuner")
    ap.add_argument("--no-target", action="store_true",
                    help="skip the m = k = n = 2^19 record (tensor-core and CUDA-core forms, "
                         "one timed product each) the default workload adds at N = 1")
    ap.add_argument("--kernel-level", type=int, default=0, choices=[0, 1],
                    help="GF(2): run the innermost Strassen level inside the base-case kernel "
                         "(CUDA-core or e2m1 tensor path)")
    args = ap.parse_args()
    if args.kernel_level and args.path not in ("popc", "fp4pair"):
        ap.error("--kernel-level 1 runs on the CUDA-core or the e2m1 kernel: add --path popc "
                 "or --path fp4pair")
    return args


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, dist) -> float:
    """The largest x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def pipelined(torch, stream, steps: int, upload, compute, download) -> float:
    """Runs `steps` end-to-end steps over two device buffer sets and returns the
    milliseconds from the first upload to the last read-back. upload(j) runs on
    an upload stream, download(j) on a read-back stream (the two directions of
    the host link overlap) and compute(j) on `stream`. Set j is re-uploaded
    once its compute has read it, and computed into again only after its
    previous products have been read back."""
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    ready = [torch.cuda.Event() for _ in range(2)]     # inputs of set j uploaded
    done = [torch.cuda.Event() for _ in range(2)]      # compute on set j finished
    fetched = [torch.cuda.Event() for _ in range(2)]   # products of set j read back
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    up.wait_event(e0)
    down.wait_event(e0)
    with torch.cuda.stream(up):
        for j in range(min(2, steps)):
            upload(j)
            ready[j].record(up)
    for i in range(steps):
        j = i % 2
        stream.wait_event(ready[j])
        if i >= 2:
            stream.wait_event(fetched[j])
        with torch.cuda.stream(stream):
            compute(j)
        done[j].record(stream)
        down.wait_event(done[j])
        with torch.cuda.stream(down):
            download(j)
        fetched[j].record(down)
        if i + 2 < steps:
            up.wait_event(done[j])
            with torch.cuda.stream(up):
                upload(j)
            ready[j].record(up)
    stream.wait_event(fetched[(steps - 1) % 2])
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


OVERLAP = ("double-buffered: uploads and read-backs on two copy streams (both directions of "
           "the host link at once) while the other buffer set computes")


def copy_times(torch, upload, download) -> dict:
    """Milliseconds of one step's upload and one read-back alone (after a
    warm-up), to set beside the end-to-end time."""
    out = {}
    for name, fn in (("h2d_ms", upload), ("d2h_ms", download)):
        fn(0)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn(0)
        b.record()
        torch.cuda.synchronize()
        out[name] = a.elapsed_time(b)
    return out


def job_rate(world: int, units_per_step: float, steps: int, ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time."""
    return world * units_per_step * steps / (ms / 1000.0)


# ---------------------------------------------------------------- CPU oracle
def oracle_sample(n: int, seed: int, bool_p: str, rows: int):
    """Time the oracle on rows 0..rows-1 of both products (inputs generated
    outside the timed region). Returns (seconds, bit operations, threads)."""
    import bitgen
    import oracle

    Bg = bitgen.fill_cpu(n, n, seed, IDS_GF2[1])
    Bb = bitgen.fill_cpu(n, n, seed, IDS_BOOL[1], p=bool_p)
    Ag = bitgen.fill_cpu(n, n, seed, IDS_GF2[0], row0=0, nrows=rows)
    Ab = bitgen.fill_cpu(n, n, seed, IDS_BOOL[0], p=bool_p, row0=0, nrows=rows)
    th = oracle.threads()
    t0 = time.perf_counter()
    oracle.rows(oracle.GF2, Ag, Bg, n, n, th)
    oracle.rows(oracle.BOOL, Ab, Bb, n, n, th)
    dt = time.perf_counter() - t0
    return dt, 2 * (2 * rows * n * n), th


def calibrated_rows(n: int, seed: int, bool_p: str, target_s: float) -> int:
    r = 32
    dt, _, _ = oracle_sample(n, seed, bool_p, r)
    want = int(r * target_s / max(dt, 1e-3))
    want = max(32, min(n, want // 32 * 32))
    return want


def cpu_baseline(n: int, seed: int, bool_p: str) -> dict:
    rows = calibrated_rows(n, seed, bool_p, 12.0)
    dt, bops, th = oracle_sample(n, seed, bool_p, rows)
    if dt < 8.0 and rows < n:  # the small calibration run overestimated the per-row cost
        rows = max(32, min(n, int(rows * 12.0 / max(dt, 1e-3)) // 32 * 32))
        dt, bops, th = oracle_sample(n, seed, bool_p, rows)
    return {"value": bops / dt, "unit": "bop/s", "cores": th, "kind": "oracle",
            "sample": f"rows 0..{rows - 1} of the GF(2) and the Boolean product at "
                      f"m=k=n={n} ({rows} of {n} rows, {dt:.1f} s)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload.startswith("batched"):
        count, seed, _ = WORKLOADS[args.workload]
        probs = batched_problems(count, seed)
        for _ in range(args.warmup):
            oracle_batched_sample(probs, 1.0)
        tot_s, tot_b, used, th = 0.0, 0, 0, 1
        for _ in range(args.steps):
            dt, b, used, th = oracle_batched_sample(probs, 3.0)
            tot_s += dt
            tot_b += b
        value = tot_b / tot_s
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": "bop/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic (seeded SplitMix64 Bernoulli bits)",
            "config": {"workload": args.workload, "problems": count},
            "cpu_baseline": {"value": value, "unit": "bop/s", "cores": th, "kind": "oracle",
                             "sample": f"the first {used} problems of the batch per step"},
            "e2e": {"value": value, "unit": "bop/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}), flush=True)
        return 0
    n, seed, bool_p = WORKLOADS[args.workload]
    rows = calibrated_rows(n, seed, bool_p, 3.0)
    for _ in range(args.warmup):
        oracle_sample(n, seed, bool_p, rows)
    tot_s, tot_b, th = 0.0, 0, 1
    for _ in range(args.steps):
        dt, b, th = oracle_sample(n, seed, bool_p, rows)
        tot_s += dt
        tot_b += b
    value = tot_b / tot_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "bop/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * tot_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded SplitMix64 Bernoulli bits)",
        "config": {"workload": args.workload, "m": n, "k": n, "n": n,
                   "sample_rows_per_step": rows},
        "cpu_baseline": {"value": value, "unit": "bop/s", "cores": th, "kind": "oracle",
                         "sample": f"rows 0..{rows - 1} of both products per step"},
        "e2e": {"value": value, "unit": "bop/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload.startswith("batched"):
        return run_batched(args)
    if args.workload.startswith("host"):
        return run_host(args)

    import torch

    import bitgen
    import paper_1909_01554_gb300 as bmm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    n, seed, bool_p = WORKLOADS[args.workload]
    m = k = n
    path = {"auto": bmm.PATH_AUTO, "fp8": bmm.PATH_TC_FP8, "i8": bmm.PATH_TC_I8,
            "popc": bmm.PATH_POPC, "fp8pair": bmm.PATH_TC_FP8_PAIR,
            "fp4pair": bmm.PATH_TC_FP4_PAIR}[args.path]
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    # inputs resident in HBM (device generator; same stream definition as the CPU one)
    def gen(rows, cols, mid, p):
        t = bmm.empty(rows, cols)
        bitgen.fill_device(t, cols, seed, mid, p=p, stream=sh)
        return t

    Ag, Bg = gen(m, k, IDS_GF2[0], None), gen(k, n, IDS_GF2[1], None)
    Ab, Bb = gen(m, k, IDS_BOOL[0], bool_p), gen(k, n, IDS_BOOL[1], bool_p)
    Cg, Cb = bmm.empty(m, n), bmm.empty(m, n)
    kw_g = {"path": path, "depth": args.depth}
    if args.kernel_level:
        kw_g["kernel_level"] = args.kernel_level
    kw_b = {"path": path}
    # The autotuner picks base-case path and Strassen depth by measurement
    # (outside the timed region) wherever both are left to the library.
    tuned = {}
    if path == bmm.PATH_AUTO and not args.no_tune:
        if args.depth < 0:
            tuned["gf2"] = bmm.autotune(bmm.GF2, m, k, n, stream=sh)
        tuned["bool"] = bmm.autotune(bmm.BOOL, m, k, n, stream=sh)

    def step(A1, B1, C1, A2, B2, C2, mid=None):
        bmm.gf2(A1, B1, C1, m, k, n, stream=sh, **kw_g)
        if mid is not None:
            mid.record(stream)
        bmm.boolean(A2, B2, C2, m, k, n, stream=sh, **kw_b)

    for _ in range(args.warmup):
        step(Ag, Bg, Cg, Ab, Bb, Cb)
    bmm.stream_status(sh)
    torch.cuda.synchronize()
    barrier()

    sampler = ClockSampler(torch.cuda.current_device())
    bmm.trace_enable(True)
    l0 = bmm.launch_count()
    sampler.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    # step boundaries and the point between the two products of each step
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 1)]
    ev0.record(stream)
    marks[0].record(stream)
    for i in range(args.steps):
        step(Ag, Bg, Cg, Ab, Bb, Cb, mid=marks[2 * i + 1])
        marks[2 * i + 2].record(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    per_product = {
        "gf2": sum(marks[2 * i].elapsed_time(marks[2 * i + 1]) for i in range(args.steps))
        / args.steps,
        "bool": sum(marks[2 * i + 1].elapsed_time(marks[2 * i + 2]) for i in range(args.steps))
        / args.steps,
    }
    launches = bmm.launch_count() - l0
    bmm.trace_enable(False)
    bmm.stream_status(sh)
    ms = ev0.elapsed_time(ev1)
    base_n, base_ms = bmm.trace_read(bmm.PHASE_BASE)
    xor_n, xor_ms = bmm.trace_read(bmm.PHASE_XOR)
    tr_n, tr_ms = bmm.trace_read(bmm.PHASE_TRANSPOSE)
    ms = max_over_ranks(ms, dist)

    bops_step = 2 * (2 * m * k * n)
    value = job_rate(world, bops_step, args.steps, ms)

    # plan facts for the roofline of the base case (the dominant kernel)
    pg = bmm.plan(bmm.GF2, m, k, n, **kw_g)
    pb = bmm.plan(bmm.BOOL, m, k, n, **kw_b)
    depth_g, leaves = pg["strassen_depth"], pg["leaves"]
    lm, lk, ln = m >> depth_g, k >> depth_g, n >> depth_g
    flops_base_step = 2 * leaves * lm * lk * ln + 2 * m * k * n  # GF(2) leaves + Boolean
    resolved = pg["path"]
    pk, pk_kind = peaks()
    if resolved in (*bmm.TENSOR_PATHS, bmm.PATH_TC_I8):
        fp4 = resolved == bmm.PATH_TC_FP4_PAIR
        peak, peak_source = tensor_peak(pk, pk_kind, fp4)
        achieved = flops_base_step * args.steps / (base_ms / 1000.0) / 1e12
        traffic = recorded_traffic(args.workload, depth_g, pg["serial_depth"],
                                   base_n / args.steps)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "traffic_algorithmic": (7 ** depth_g * (lm * lk + ln * lk + lm * ln)
                                        + m * k + k * n + m * n) / 8 / (base_n / args.steps),
                "peak_source": peak_source,
                **tensor_pipe(achieved, clocks, pk["sm_max_mhz"], fp4)}
        dtype = "u8" if resolved == bmm.PATH_TC_I8 else "e2m1" if fp4 else "e4m3"
    else:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        peak = sms * LOP3_LANES_PER_SM_CLK * pk["sm_max_mhz"] * 1e6 * 64 / 1e12
        achieved = flops_base_step * args.steps / (base_ms / 1000.0) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tbop/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": f"{sms} SMs x {LOP3_LANES_PER_SM_CLK} LOP3/clk x "
                               f"{pk['sm_max_mhz']} MHz x 64 bop"}
        dtype = "u32"

    # end to end through the public API with pinned host buffers: every step
    # uploads its four operands and reads both products back; two device
    # buffer sets let step i+1's upload run on a copy stream while step i
    # computes
    e2e = None
    if not args.no_e2e:
        hA = [x.cpu().pin_memory() for x in (Ag, Bg, Ab, Bb)]
        hC = [[torch.empty(m * n // 64, dtype=torch.int64).pin_memory() for _ in range(2)]
              for _ in range(2)]
        dA = [[torch.empty_like(x) for x in (Ag, Bg, Ab, Bb)] for _ in range(2)]
        dC = [[bmm.empty(m, n), bmm.empty(m, n)] for _ in range(2)]

        def upload(j):
            for h, d in zip(hA, dA[j]):
                d.copy_(h, non_blocking=True)

        def compute(j):
            step(dA[j][0], dA[j][1], dC[j][0], dA[j][2], dA[j][3], dC[j][1])

        def download(j):
            for h, d in zip(hC[j], dC[j]):
                h.copy_(d, non_blocking=True)

        pipelined(torch, stream, 2, upload, compute, download)  # warm-up
        torch.cuda.synchronize()
        barrier()
        ems = pipelined(torch, stream, args.steps, upload, compute, download)
        ems = max_over_ranks(ems, dist)
        e2e = {"value": job_rate(world, bops_step, args.steps, ems), "unit": "bop/s",
               "h2d_bytes_per_step": 4 * m * k // 8, "d2h_bytes_per_step": 2 * m * n // 8,
               "ms_per_step": ems / args.steps, **copy_times(torch, upload, download),
               "overlap": OVERLAP}

    # end to end through the library's own host-memory entry points
    # (bmm_gf2_host / bmm_bool_host): pinned host arrays in and out, each call
    # blocking until its product is back in host memory
    e2e_host = None
    if not args.no_e2e and world == 1:
        e2e_host = host_api_e2e(torch, bmm, (Ag, Bg, Ab, Bb), m, k, n, args.steps, stream,
                                kw_g, kw_b)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n, seed, bool_p)

    # the largest single-GPU configuration, measured in the same run
    target = None
    if args.workload == DEFAULT_WORKLOAD and world == 1 and not args.no_target:
        del Ag, Bg, Ab, Bb, Cg, Cb
        if e2e is not None:
            del hA, hC, dA, dC
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        target = target_record(torch, bmm, bitgen, stream, pk, pk_kind,
                               no_tune=args.no_tune)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "bop/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic (seeded SplitMix64 Bernoulli bits)",
            "config": {"workload": args.workload, "m": m, "k": k, "n": n,
                       "gf2": f"p=1/2, Strassen depth {depth_g} ({leaves} leaves), "
                              f"self-inverse alternative basis"
                              + (", innermost level inside the base-case kernel"
                                 if pg["kernel_level"] else ""),
                       "bool": f"p={bool_p}, cubic", "base_case": _path_name(resolved),
                       "bool_base_case": _path_name(pb["path"]),
                       "l2": f"inputs larger than L2 (each operand {m * k // 8 // 2**20} MiB)",
                       "autotuned": {op: {"path": _path_name(t["path"]),
                                          "strassen_depth": t["strassen_depth"],
                                          "way": "whole products timed" if t["measured"]
                                          else "leaf proxies timed + pass model",
                                          "candidates": t["candidates"]}
                                     for op, t in tuned.items()} or None,
                       "parallelism": f"replicas x{world}"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "product_ms": per_product,
            "product_bops": {op: 2 * m * k * n / (t / 1000.0) for op, t in per_product.items()},
            "phases_ms_per_step": {"base": base_ms / args.steps, "xor": xor_ms / args.steps,
                                   "transpose": tr_ms / args.steps},
            "phase_launches": {"base": base_n, "xor": xor_n, "transpose": tr_n},
            "e2e_host": e2e_host,
            "gf2_strassen_bound": (strassen_bound(pg, m, n, per_product["gf2"], roof["peak"],
                                                  pk["hbm_gbs"], roof.get("pipe_peak"))
                                   if depth_g > 0 else None),
            "target_2pow19": target,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0



def host_api_e2e(torch, bmm, dev_inputs, m, k, n, steps, stream, kw_g, kw_b) -> dict:
    """The step through bmm_gf2_host / bmm_bool_host: operands and products in
    pinned host memory, every call uploading its operands, computing and
    reading its product back before it returns (host wall clock around the
    calls, which block)."""
    hAg, hBg, hAb, hBb = (x.cpu().pin_memory() for x in dev_inputs)
    hCg = torch.empty(m * n // 64, dtype=torch.int64).pin_memory()
    hCb = torch.empty(m * n // 64, dtype=torch.int64).pin_memory()
    sh = stream.cuda_stream
    dev = {key: v for key, v in kw_g.items() if key in ("path", "depth")}
    devb = {key: v for key, v in kw_b.items() if key == "path"}

    def step():
        bmm.product_host(bmm.GF2, hAg, hBg, hCg, m, k, n, stream=sh, **dev)
        bmm.product_host(bmm.BOOL, hAb, hBb, hCb, m, k, n, stream=sh, **devb)

    step()  # warm-up: pinned staging and device buffers are kept between calls
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1000.0
    pg = bmm.host_plan(bmm.GF2, m, k, n, **dev)
    pb = bmm.host_plan(bmm.BOOL, m, k, n, **devb)
    bmm.host_release()
    return {"value": 2 * (2 * m * k * n) * steps / (ms / 1000.0), "unit": "bop/s",
            "ms_per_step": ms / steps,
            "h2d_bytes_per_step": pg["upload_bytes"] + pb["upload_bytes"],
            "d2h_bytes_per_step": pg["download_bytes"] + pb["download_bytes"],
            "api": "bmm_gf2_host + bmm_bool_host (pinned host arrays, blocking calls)",
            "timer": "host wall clock around the blocking calls"}


def target_record(torch, bmm, bitgen, stream, pk, pk_kind, no_tune=False) -> dict:
    """m = k = n = 2^19 (32 GiB per operand; seed 4, GF(2) p = 1/2, Boolean
    p = 2^-9.5), one product at a time with A, B and C resident in HBM. The
    tensor-core form (the autotuned path and depth) runs one untimed and one
    timed product; the CUDA-core form (LOP3/POPC base case, the same Strassen
    depth for GF(2)) one timed product. Both forms' products are compared
    word for word on the device."""
    n, seed, bool_p = WORKLOADS["square524288"]
    sh = stream.cuda_stream
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    alu_peak = sms * LOP3_LANES_PER_SM_CLK * pk["sm_max_mhz"] * 1e6 * 64 / 1e12
    out = {"workload": "square524288", "m": n, "k": n, "n": n, "seed": seed,
           "gf2": "p=1/2", "bool": f"p={bool_p}, cubic",
           "l2": "inputs larger than L2 (each operand 32 GiB)"}
    forms = {}
    for name, op, ids, p in (("gf2", bmm.GF2, IDS_GF2, None), ("bool", bmm.BOOL, IDS_BOOL, bool_p)):
        if not no_tune:
            t = bmm.autotune(op, n, n, n, stream=sh)
            out.setdefault("autotuned", {})[name] = {
                "path": _path_name(t["path"]), "strassen_depth": t["strassen_depth"],
                "way": "whole products timed" if t["measured"] else "leaf proxies timed + pass model"}
        A, B = bmm.empty(n, n), bmm.empty(n, n)
        bitgen.fill_device(A, n, seed, ids[0], p=p, stream=sh)
        bitgen.fill_device(B, n, seed, ids[1], p=p, stream=sh)
        C = bmm.empty(n, n)
        pt = bmm.plan(op, n, n, n)
        d = pt["strassen_depth"]
        flops = 2 * pt["leaves"] * (n >> d) ** 3
        res = {}
        for form, kw, warm in (("tensor", {}, True),
                               ("popcount", {"path": bmm.PATH_POPC, "depth": d}, False)):
            if form == "popcount":
                Ct = C
                C = bmm.empty(n, n)
            if warm:
                bmm.product(op, A, B, C, n, n, n, stream=sh, **kw)
            bmm.stream_status(sh)
            bmm.trace_enable(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bmm.product(op, A, B, C, n, n, n, stream=sh, **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            bmm.trace_enable(False)
            bmm.stream_status(sh)
            ms = e0.elapsed_time(e1)
            _, base_ms = bmm.trace_read(bmm.PHASE_BASE)
            achieved = flops / (base_ms / 1000.0) / 1e12
            pl = bmm.plan(op, n, n, n, **kw)
            if form == "tensor":
                fp4 = pl["path"] == bmm.PATH_TC_FP4_PAIR
                peak, src = tensor_peak(pk, pk_kind, fp4)
                roof = {"bound": "tensor", "achieved": achieved, "peak": peak,
                        "unit": "TFLOP/s", "frac": achieved / peak, "peak_source": src}
            else:
                roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak,
                        "unit": "Tbop/s", "frac": achieved / alu_peak,
                        "peak_source": f"{sms} SMs x {LOP3_LANES_PER_SM_CLK} LOP3/clk x "
                                       f"{pk['sm_max_mhz']} MHz x 64 bop"}
            res[form] = {"product_ms": ms, "bops": 2 * n ** 3 / (ms / 1000.0),
                         "path": pl["path"], "base_case": _path_name(pl["path"]),
                         "strassen_depth": pl["strassen_depth"],
                         "base_ms": base_ms, "roofline": roof, "_plan": pl,
                         "timed": "one product" + (" after one untimed" if warm else "")}
        step = 1 << 28  # words per comparison chunk
        res["paths_agree"] = all(bool(torch.equal(C[i:i + step], Ct[i:i + step]))
                                 for i in range(0, C.numel(), step))
        res["tensor_over_popcount"] = res["popcount"]["product_ms"] / res["tensor"]["product_ms"]
        forms[name] = res
        del A, B, C, Ct
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    clocks = sampler.stop()
    for name in forms:
        t = forms[name]["tensor"]
        t["roofline"].update(tensor_pipe(t["roofline"]["achieved"], clocks, pk["sm_max_mhz"],
                                         t["path"] == bmm.PATH_TC_FP4_PAIR))
        for form in ("tensor", "popcount"):
            f = forms[name][form]
            if f["strassen_depth"] > 0:
                f["strassen_bound"] = strassen_bound(
                    f.pop("_plan"), n, n, f["product_ms"], f["roofline"]["peak"], pk["hbm_gbs"],
                    f["roofline"].get("pipe_peak"))
            else:
                f.pop("_plan")
    out["products"] = forms
    out["clocks"] = clocks
    return out


def batched_problems(count: int, seed: int):
    import bitgen

    shapes = bitgen.batched_shapes(count, seed)
    return [(m, k, n, op, (seed << 16) + i) for i, (m, k, n, op) in enumerate(shapes)]


def density_for(op: int, k: int):
    return None if op == 0 else f"1/sqrt({k})"


def oracle_batched_sample(probs, target_s: float):
    """Oracle time on whole problems of the batch, taken in order until about
    target_s seconds. Returns (seconds, bit operations, problems, threads)."""
    import bitgen
    import oracle

    tot_s, bops, used = 0.0, 0, 0
    th = oracle.threads()
    for m, k, n, op, seed in probs:
        A = bitgen.fill_cpu(m, k, seed, 0, p=density_for(op, k))
        B = bitgen.fill_cpu(k, n, seed, 1, p=density_for(op, k))
        t0 = time.perf_counter()
        oracle.cubic(oracle.GF2 if op == 0 else oracle.BOOL, A, B, m, k, n, th)
        tot_s += time.perf_counter() - t0
        bops += 2 * m * k * n
        used += 1
        if tot_s >= target_s:
            break
    return tot_s, bops, used, th


def run_host(args):
    """Host-memory products (the host layer): A, B and C in pinned host memory,
    the device limited to HOST_DEVICE_BYTES; a step is one GF(2) and one
    Boolean product, each a blocking library call from host arrays to host
    arrays (so every step moves its inputs in and its products out)."""
    import torch

    import bitgen
    import paper_1909_01554_gb300 as bmm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n, seed, bool_p = WORKLOADS[args.workload]
    m = k = n
    budget = HOST_DEVICE_BYTES[args.workload]
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    def gen(rows, cols, mid, p):
        t = bmm.empty(rows, cols)
        bitgen.fill_device(t, cols, seed, mid, p=p, stream=sh)
        h = t.cpu().pin_memory()
        del t
        return h

    Ag, Bg = gen(m, k, IDS_GF2[0], None), gen(k, n, IDS_GF2[1], None)
    Ab, Bb = gen(m, k, IDS_BOOL[0], bool_p), gen(k, n, IDS_BOOL[1], bool_p)
    Cg = torch.empty(m * n // 64, dtype=torch.int64).pin_memory()
    Cb = torch.empty(m * n // 64, dtype=torch.int64).pin_memory()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    kw = {"device_bytes": budget}
    pg = bmm.host_plan(bmm.GF2, m, k, n, **kw)
    pb = bmm.host_plan(bmm.BOOL, m, k, n, **kw)

    def step(mid=None):
        bmm.product_host(bmm.GF2, Ag, Bg, Cg, m, k, n, stream=sh, **kw)
        if mid is not None:
            mid.record(stream)
        bmm.product_host(bmm.BOOL, Ab, Bb, Cb, m, k, n, stream=sh, **kw)

    for _ in range(args.warmup):
        step()
    bmm.stream_status(sh)
    sampler = ClockSampler(torch.cuda.current_device())
    bmm.trace_enable(True)
    l0 = bmm.launch_count()
    sampler.start()
    time.sleep(0.3)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 1)]
    torch.cuda.synchronize()
    marks[0].record(stream)
    for i in range(args.steps):
        step(mid=marks[2 * i + 1])
        marks[2 * i + 2].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = bmm.launch_count() - l0
    bmm.trace_enable(False)
    bmm.stream_status(sh)
    ms = max_over_ranks(marks[0].elapsed_time(marks[-1]), dist)
    per_product = {
        "gf2": sum(marks[2 * i].elapsed_time(marks[2 * i + 1]) for i in range(args.steps))
        / args.steps,
        "bool": sum(marks[2 * i + 1].elapsed_time(marks[2 * i + 2]) for i in range(args.steps))
        / args.steps,
    }
    base_n, base_ms = bmm.trace_read(bmm.PHASE_BASE)
    bops_step = 2 * (2 * m * k * n)
    value = job_rate(world, bops_step, args.steps, ms)
    # base-case work: every device product's leaves (GF(2)) or its cubic work
    sg = bmm.plan(bmm.GF2, pg["sub_m"], pg["sub_k"], pg["sub_n"])
    d = sg["strassen_depth"]
    flops = (2 * pg["count"] * sg["leaves"] * (pg["sub_m"] >> d) * (pg["sub_k"] >> d)
             * (pg["sub_n"] >> d) + 2 * m * k * n)
    pk, pk_kind = peaks()
    fp4 = sg["path"] == bmm.PATH_TC_FP4_PAIR
    peak, peak_source = tensor_peak(pk, pk_kind, fp4)
    achieved = flops * args.steps / (base_ms / 1000.0) / 1e12 if base_ms > 0 else 0.0
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None, "peak_source": peak_source,
            **tensor_pipe(achieved, clocks, pk["sm_max_mhz"], fp4)}
    h2d = pg["upload_bytes"] + pb["upload_bytes"]
    d2h = pg["download_bytes"] + pb["download_bytes"]
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n, seed, bool_p)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "bop/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "e2m1" if fp4 else "e4m3",
            "data": "synthetic (seeded SplitMix64 Bernoulli bits), pinned host memory",
            "config": {"workload": args.workload, "m": m, "k": k, "n": n,
                       "device_bytes": budget,
                       "gf2": f"p=1/2, {pg['host_depth']} host Strassen levels: "
                              f"{pg['count']} device products of {pg['sub_m']}^3 "
                              f"(device Strassen depth {d})",
                       "bool": f"p={bool_p}, C in {pb['count']} blocks of "
                               f"{pb['sub_m']} x {pb['sub_n']}",
                       "l2": "inputs larger than L2 (each operand "
                             f"{m * k // 8 // 2**20} MiB)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "bop/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "note": "the step itself runs host arrays to host arrays"},
            "gpu_launches": launches,
            "clocks": clocks,
            "product_ms": per_product,
            "product_bops": {op: 2 * m * k * n / (t / 1000.0) for op, t in per_product.items()},
            "host_plans": {"gf2": pg, "bool": pb},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_batched(args):
    import torch

    import bitgen
    import paper_1909_01554_gb300 as bmm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    count, seed, _ = WORKLOADS[args.workload]
    probs = batched_problems(count, seed)
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    # Every problem's operands are views into one input arena and its product
    # into one output arena (each block a multiple of 512 bytes), so a step's
    # host traffic is one copy each way.
    in_words = sum(m * k // 64 + k * n // 64 for m, k, n, *_ in probs)
    out_words = sum(m * n // 64 for m, k, n, *_ in probs)
    d_in = torch.empty(in_words, dtype=torch.int64, device="cuda")
    d_out = torch.empty(out_words, dtype=torch.int64, device="cuda")
    As, Bs, Cs = [], [], []
    oi = oo = 0
    with torch.cuda.stream(stream):
        for m, k, n, op, sd in probs:
            A = d_in[oi:oi + m * k // 64]
            oi += m * k // 64
            B = d_in[oi:oi + k * n // 64]
            oi += k * n // 64
            bitgen.fill_device(A, k, sd, 0, p=density_for(op, k), stream=sh)
            bitgen.fill_device(B, n, sd, 1, p=density_for(op, k), stream=sh)
            As.append(A)
            Bs.append(B)
            Cs.append(d_out[oo:oo + m * n // 64])
            oo += m * n // 64
    torch.cuda.synchronize()
    ops = [p[3] for p in probs]
    ms, ks, ns = [p[0] for p in probs], [p[1] for p in probs], [p[2] for p in probs]
    bops_step = sum(2 * m * k * n for m, k, n, *_ in probs)

    plan = bmm.BatchedPlan(ops, As, Bs, Cs, ms, ks, ns)
    graph = torch.cuda.CUDAGraph()
    l_run = bmm.launch_count()
    plan.run(stream=sh)  # warm the kernels before capture
    torch.cuda.synchronize()
    per_run = bmm.launch_count() - l_run  # kernels one run (and one graph replay) launches
    with torch.cuda.graph(graph, stream=stream):
        plan.run(stream=sh)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            graph.replay()
    torch.cuda.synchronize()
    bmm.stream_status(sh)

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    bmm.trace_enable(True)
    l0 = bmm.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(args.steps):
            graph.replay()
        ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    bmm.trace_enable(False)
    # a graph replay launches the kernels a plan run launches: the batched
    # transpose, the row padding (when some tensor problem's k/64 is odd) and
    # the base-case launches (tensor tiles, CUDA-core tiles)
    launches = (bmm.launch_count() - l0) + per_run * args.steps
    ms_total = ev0.elapsed_time(ev1)
    ms_total = max_over_ranks(ms_total, dist)
    value = job_rate(world, bops_step, args.steps, ms_total)

    # the base-case kernels alone, timed with events on their stream (one
    # plan run; the best of three)
    base_ms = pre_ms = None
    for _ in range(3):
        bmm.trace_enable(True)
        plan.run(stream=sh)
        torch.cuda.synchronize()
        bmm.trace_enable(False)
        base_n, t = bmm.trace_read(bmm.PHASE_BASE)
        _, tp = bmm.trace_read(bmm.PHASE_TRANSPOSE)  # batched transpose and row padding
        base_ms = t if base_ms is None else min(base_ms, t)
        pre_ms = tp if pre_ms is None else min(pre_ms, tp)
    pk, pk_kind = peaks()
    fp4 = plan.path() == bmm.PATH_TC_FP4_PAIR
    peak, peak_source = tensor_peak(pk, pk_kind, fp4)
    achieved = bops_step / (base_ms / 1000.0) / 1e12 if base_ms > 0 else 0.0
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None, "peak_source": peak_source,
            **tensor_pipe(achieved, clocks, pk["sm_max_mhz"], fp4)}
    # what the plan chose per problem, and the padding its tiles carry
    pst = plan.stats()
    bmodel = bmm.batched_model(pst["tensor_path"])
    choices = [plan.choice(i) for i in range(count)]
    plan_record = {
        "problems_by_path": {_path_name(pst["tensor_path"]): pst["tensor_problems"],
                             _path_name(bmm.PATH_POPC): pst["popc_problems"]},
        "tensor_tiles": pst["tensor_tiles"], "tensor_tiles_n128": pst["tensor_tiles_n128"],
        "popc_tiles": pst["popc_tiles"],
        "half_k_stage_problems": sum(1 for c in choices
                                     if c["path"] != bmm.PATH_POPC and c["k_steps"] % 2),
        "strassen_depths": sorted({c["strassen_depth"] for c in choices}),
        "macs_issued_over_needed": pst["macs_issued"] / pst["macs_needed"],
        "model_est_base_ms": pst["est_ms"], "measured_base_ms": base_ms,
        "transpose_and_pad_ms": pre_ms,
        "model": {k_: v for k_, v in bmodel.items() if k_ != "path"},
    }

    # the same products as one library call per problem
    def per_problem():
        for (m, k, n, op, _), A, B, C in zip(probs, As, Bs, Cs):
            bmm.product(op, A, B, C, m, k, n, stream=sh)

    per_problem()
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    p0.record(stream)
    per_problem()
    p1.record(stream)
    torch.cuda.synchronize()
    per_ms = p0.elapsed_time(p1)
    per_wall = (time.perf_counter() - t0) * 1000

    # end to end: inputs from pinned host memory, products back to the host
    e2e = None
    if not args.no_e2e:
        h_in = d_in.cpu().pin_memory()
        h_outs = [torch.empty_like(d_out, device="cpu").pin_memory() for _ in range(2)]
        # a second arena pair with its own plan and graph, so that one set
        # uploads while the other computes
        d_in2, d_out2 = torch.empty_like(d_in), torch.empty_like(d_out)
        As2, Bs2, Cs2 = [], [], []
        oi = oo = 0
        for m_, k_, n_, *_ in probs:
            As2.append(d_in2[oi:oi + m_ * k_ // 64])
            oi += m_ * k_ // 64
            Bs2.append(d_in2[oi:oi + k_ * n_ // 64])
            oi += k_ * n_ // 64
            Cs2.append(d_out2[oo:oo + m_ * n_ // 64])
            oo += m_ * n_ // 64
        plan2 = bmm.BatchedPlan(ops, As2, Bs2, Cs2, ms, ks, ns)
        graph2 = torch.cuda.CUDAGraph()
        plan2.run(stream=sh)
        torch.cuda.synchronize()
        with torch.cuda.graph(graph2, stream=stream):
            plan2.run(stream=sh)
        sets = [(d_in, d_out, graph), (d_in2, d_out2, graph2)]

        def upload(j):
            sets[j][0].copy_(h_in, non_blocking=True)

        def compute(j):
            sets[j][2].replay()

        def download(j):
            h_outs[j].copy_(sets[j][1], non_blocking=True)

        pipelined(torch, stream, 2, upload, compute, download)  # warm-up
        torch.cuda.synchronize()
        ems = max_over_ranks(pipelined(torch, stream, args.steps, upload, compute, download),
                             dist)
        copies = copy_times(torch, upload, download)
        plan2.destroy()
        e2e = {"value": job_rate(world, bops_step, args.steps, ems), "unit": "bop/s",
               "h2d_bytes_per_step": d_in.numel() * 8, "d2h_bytes_per_step": d_out.numel() * 8,
               "ms_per_step": ems / args.steps, **copies, "overlap": OVERLAP}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        tot_s, b, used, th = oracle_batched_sample(probs, 12.0)
        cpu = {"value": b / tot_s, "unit": "bop/s", "cores": th, "kind": "oracle",
               "sample": f"the first {used} of {count} problems, whole ({tot_s:.1f} s)"}
    plan.destroy()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "bop/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "e2m1" if fp4 else "e4m3",
            "data": "synthetic (seeded SplitMix64 Bernoulli bits)",
            "config": {"workload": args.workload, "problems": count,
                       "shapes": "m, k, n log-uniform in [256, 8192], multiples of 64",
                       "ops": "50/50 GF(2) (p=1/2) / Boolean (p=1/sqrt(k))",
                       "sum_2mkn": bops_step, "launch": "one CUDA-graph replay of a batch plan "
                       "(batched transpose, row padding, persistent tcgen05 base case; a "
                       "persistent CUDA-core launch for problems the plan sends there)",
                       "l2": "inputs larger than L2 (~4 GB per step)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks,
            "per_problem_launches": {"value": bops_step / (per_ms / 1000.0), "unit": "bop/s",
                                     "ms": per_ms, "host_wall_ms": per_wall,
                                     "launches": None},
            "plan": plan_record,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _path_name(p) -> str:
    return {1: "tcgen05 fp8 (e4m3, f32 accumulate)", 2: "tcgen05 int8 (u8, s32 accumulate)",
            3: "CUDA-core LOP3/POPC",
            4: "tcgen05 fp8 (e4m3, f32 accumulate), SM pairs (cta_group::2)",
            5: "tcgen05 fp4 (e2m1, block-scaled kind::mxf4, f32 accumulate), SM pairs "
               "(cta_group::2)"}.get(p, str(p))


if __name__ == "__main__":
    sys.exit(main())
