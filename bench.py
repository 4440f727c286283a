"""Benchmark of the sliding-window-sum hot path on GB300.

Workload (the configuration the headline metric is quoted on): the generic sliding-sum sweep
over 2^28 elements -- int32 uniform in [-2^20, 2^20) for + mod 2^32, min, max, xor; affine maps
(a, b) uniform uint32 (non-commutative composition); fp32 N(0,1) for +; windows
w in {4, 16, 64, 256, 1024}.  One step = all 30 (operator, w) sliding sums, inputs resident in
HBM.  Every input and output is larger than L2 (no flush needed).

Printed: ONE JSON line with the whole-job GB/s (algorithmic bytes: input + output of every call),
the roofline of the sliding-sum kernels against the measured HBM copy bandwidth, the same metric
end to end (pinned host buffers, copies inside the timed region), the oracle timed on host cores
on a bounded sample, secondary minimizer measurements, and the SM clocks seen while timing.

``--impl reference`` times the oracle (the plain CPU statement of Eq. 2) instead.
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
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

OPS = ["add_i32", "min_i32", "max_i32", "xor_i32", "affine_u32", "add_f32"]
WS = [4, 16, 64, 256, 1024]
ESIZE = {"affine_u32": 8}
METRIC = "minimizer Gbp/s & sliding-sum GB/s vs HBM peak; batched vs plain; p99 latency"
# DRAM traffic of the sliding-sum kernels, from one ncu capture of the full 30-case sweep at 2^26
# elements (dram__bytes_read.sum + dram__bytes_write.sum, mean per launch), scaled to the run's n
# by the elements processed.  Valid only for the kernel sources it was taken on: the hash below
# covers them, and a mismatch reports the traffic as null.
TRAFFIC_PROFILE = {"bytes_per_launch": 578392021.3, "n": 1 << 26, "sources_sha256_16": "7f8da2f2d001f10f",
                   "summary": "profiles/sliding_sum_sweep_2e26_dram_traffic.md"}
TRAFFIC_SOURCES = ["paper_1811_10074_gb300/csrc/sliding_sum.cu", "paper_1811_10074_gb300/csrc/common.cuh",
                   "paper_1811_10074_gb300/csrc/tma.cuh"]
WORKLOAD = ("sliding-sum sweep: 2^28 elements; int32 U[-2^20,2^20) for +,min,max,xor; affine (a,b) uint32; "
            "fp32 N(0,1) for +; w in {4,16,64,256,1024}")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1 << 28, help="elements per sliding-sum input")
    ap.add_argument("--no-extras", action="store_true", help="skip the secondary measurements")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuners (AUTO uses its fixed rule; a read batch takes its default path)")
    ap.add_argument("--ops", default=",".join(OPS), help="comma list of operators to time")
    ap.add_argument("--ws", default=",".join(map(str, WS)), help="comma list of window sizes to time")
    ap.add_argument("--keys-n", type=int, default=1 << 28, help="keys of the --section keys measurement")
    ap.add_argument("--keys-ws", default="4,5,6,7,8,9,10,11,12,13,14,15,16,17", help="window lengths of --section keys")
    ap.add_argument("--section", default="all",
                    choices=["all", "sliding", "minimizers", "fused", "keys", "table", "table-skew", "batch", "serve"],
                    help="'minimizers' runs only the secondary minimizer measurements")
    ap.add_argument("--cpu-sample", type=int, default=1 << 20, help="elements per case for the CPU baseline")
    ap.add_argument("--mini-n", type=int, default=1 << 31, help="bases of the long minimizer measurement")
    ap.add_argument("--genome-n", type=int, default=3_100_000_000, help="bases of the genome-scale table measurement")
    ap.add_argument("--table-hits", type=int, default=100_000_000, help="hits of the --section table-skew measurement")
    ap.add_argument("--fused", default="15,10", help="k,w of the --section fused measurement (--mini-n bases)")
    ap.add_argument("--batch-plain", type=int, default=20_000,
                    help="reads of the plain per-read comparison of --section batch (0: skip it)")
    args = ap.parse_args()
    args.ops = [o for o in args.ops.split(",") if o]
    args.ws = [int(v) for v in args.ws.split(",") if v]
    return args


# ------------------------------------------------------------------------------------------
# distributed plumbing (one process per GPU, launched by torchrun for N > 1)
# ------------------------------------------------------------------------------------------

def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available() and args.impl == "ours":
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v: float) -> float:
    if world <= 1:
        return v
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def sweep_traffic(n: int, cases) -> float | None:
    """Mean DRAM bytes per launch of the full sweep (ncu), or None when it does not apply."""
    import hashlib
    if sorted(cases) != sorted((op, w) for op in OPS for w in WS):
        return None
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != TRAFFIC_PROFILE["sources_sha256_16"]:
        return None
    return TRAFFIC_PROFILE["bytes_per_launch"] * n / TRAFFIC_PROFILE["n"]


def case_bytes(op: str, w: int, n: int) -> int:
    es = ESIZE.get(op, 4)
    return es * (n + (n - w + 1))


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------

def make_inputs(n: int, device, seed: int):
    from paper_1811_10074_gb300 import synth
    x32 = synth.int32_uniform(n, seed=seed, device=device)
    xa = synth.affine_pairs(n, seed=seed, device=device)
    xf = synth.f32_normal(n, seed=seed, device=device)
    return {"add_i32": x32, "min_i32": x32, "max_i32": x32, "xor_i32": x32, "affine_u32": xa, "add_f32": xf}


def host_cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:  # lscpu missing: fall through
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(n_sample: int, seed: int = 42):
    """The oracle (plain O(wN) Eq. 2, single thread) on n_sample elements per case."""
    import oracle
    xs = make_inputs(n_sample, "cpu", seed)
    total_bytes = 0
    t0 = time.perf_counter()
    for op in OPS:
        for w in WS:
            oracle.sliding_sum(op, w, xs[op])
            total_bytes += case_bytes(op, w, n_sample)
    dt = time.perf_counter() - t0
    return total_bytes / dt / 1e9, dt


def run_ours(args, world, rank, local):
    import paper_1811_10074_gb300 as P
    from paper_1811_10074_gb300 import build as B
    B.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    n = args.n
    xs = make_inputs(n, dev, seed=42 + rank)
    outs = {}
    for op in OPS:
        x = xs[op]
        outs[op] = torch.empty((n,) + tuple(x.shape[1:]), dtype=x.dtype, device=dev)
    ctx = P.default_context(dev.index)
    stream = torch.cuda.current_stream()
    cases = [(op, w) for op in args.ops for w in args.ws]
    step_bytes = sum(case_bytes(op, w, n) for op, w in cases)

    def step(events=None):
        for i, (op, w) in enumerate(cases):
            if events is not None:
                events[i][0].record(stream)
            P.sliding_sum(op, w, xs[op], out=outs[op][: n - w + 1], ctx=ctx, stream=stream)
            if events is not None:
                events[i][1].record(stream)

    tuned = {}
    if not args.no_tune:  # the library's autotuner picks the variant AUTO uses for each (op, w)
        for op, w in cases:
            tuned[f"{op}/w{w}"] = P.tune_sliding_sum(op, w, n, ctx=ctx, stream=stream)[0]
    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in cases]
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for s in range(args.steps):
        step(ev[s])
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms_total = t_start.elapsed_time(t_end)
    ms_total = max_over_ranks(world, ms_total)
    ms_step = ms_total / args.steps
    value = world * step_bytes / (ms_step / 1e3) / 1e9
    ctx.sync()

    # roofline of the sliding-sum kernels, per launch
    per_case = {}
    tot_b, tot_ms = 0, 0.0
    for i, (op, w) in enumerate(cases):
        d = [ev[s][i][0].elapsed_time(ev[s][i][1]) for s in range(args.steps)]
        ms = sum(d) / len(d)
        b = case_bytes(op, w, n)
        per_case[f"{op}/w{w}"] = round(b / (ms / 1e3) / 1e9, 1)
        tot_b += b * len(d)
        tot_ms += sum(d)
    peak, peak_kind = measured_peaks()
    achieved = tot_b / (tot_ms / 1e3) / 1e9
    traffic = sweep_traffic(n, cases)

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        e2e = e2e_leg(args, world, xs, outs, ctx, stream, step_bytes)

    result = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32,u32x2,f32",
        "data": "synthetic (SplitMix64 seed 42, generated on the device)",
        "config": {"workload": WORKLOAD, "n": n, "ops": args.ops, "w": args.ws, "calls_per_step": len(cases),
                   "bytes_per_step": step_bytes, "l2": "inputs and outputs larger than L2 (no flush)",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"kernel": "sliding-sum block combine (k_slide_small for w=4, warp-private k_slide_warp / k_slide_wblk otherwise)",
                     "bound": "hbm",
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                     "traffic": None if traffic is None else round(traffic),
                     "algorithmic_bytes_per_launch": round(step_bytes / len(cases)),
                     "traffic_source": TRAFFIC_PROFILE["summary"] + " (2^26 capture scaled by elements)",
                     "per_case_gbs": per_case, "variant_per_case": tuned or "fixed rule (no tuning)"},
        "e2e": e2e,
        "gpu_launches": len(cases) * args.steps,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        v, dt = cpu_baseline(args.cpu_sample)
        result["cpu_baseline"] = {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                                  "sample": f"{args.cpu_sample} elements per (op, w) case, all {len(OPS) * len(WS)} cases, "
                                            f"{dt:.1f} s single-threaded naive O(wN)",
                                  "cpu_model": host_cpu_model(), "host_cores": os.cpu_count()}
    if not args.no_extras and rank == 0:
        result["minimizers"] = minimizer_extras(dev, ctx, args.mini_n, with_cpu=not args.no_cpu)
        result["genome_table"] = genome_table_extras(dev, ctx, args.genome_n)
        result["batched_reads"] = batch_extras(dev, ctx)
        result["serving"] = serve_extras(ctx)
    del xs, outs
    torch.cuda.empty_cache()
    return result


def e2e_leg(args, world, xs, outs, ctx, stream, step_bytes):
    """The same sweep through the public API from pinned host buffers: every step copies each
    operator's input to the device, runs its sliding sums and copies every output back.  The
    copies run on their own streams (one per direction) and the outputs alternate between two
    device buffers per operator, so copies in both directions overlap the kernels; events order
    every reuse of a buffer."""
    import paper_1811_10074_gb300 as P
    n = args.n
    ops = list(dict.fromkeys(args.ops))
    srcs = {op: ("add_i32" if op in ("min_i32", "max_i32", "xor_i32") else op) for op in ops}
    hx = {src: xs[src].cpu().pin_memory() for src in dict.fromkeys(srcs.values())}
    hy = {op: torch.empty(outs[op].shape, dtype=outs[op].dtype).pin_memory() for op in ops}
    dy = {op: [outs[op], torch.empty_like(outs[op])] for op in ops}
    s_h2d, s_d2h = torch.cuda.Stream(), torch.cuda.Stream()
    nbytes = {"h2d": 0, "d2h": 0}
    ev = lambda: torch.cuda.Event()
    state = {"used": {src: None for src in hx}, "slot_free": {op: [None, None] for op in ops}}

    def e2e_step():
        nbytes["h2d"] = nbytes["d2h"] = 0
        loaded = {}
        for src in hx:  # inputs: all uploads first, each after the previous step's last read of it
            if state["used"][src] is not None:
                s_h2d.wait_event(state["used"][src])
            with torch.cuda.stream(s_h2d):
                xs[src].copy_(hx[src], non_blocking=True)
            loaded[src] = ev()
            loaded[src].record(s_h2d)
            nbytes["h2d"] += hx[src].numel() * hx[src].element_size()
        k = 0
        for op in ops:
            stream.wait_event(loaded[srcs[op]])
            for w in args.ws:
                m = n - w + 1
                slot = k & 1
                k += 1
                if state["slot_free"][op][slot] is not None:
                    stream.wait_event(state["slot_free"][op][slot])
                P.sliding_sum(op, w, xs[op], out=dy[op][slot][:m], ctx=ctx, stream=stream)
                done = ev()
                done.record(stream)
                s_d2h.wait_event(done)
                with torch.cuda.stream(s_d2h):
                    hy[op][:m].copy_(dy[op][slot][:m], non_blocking=True)
                free = ev()
                free.record(s_d2h)
                state["slot_free"][op][slot] = free
                nbytes["d2h"] += hy[op][:m].numel() * hy[op].element_size()
            last = ev()
            last.record(stream)
            state["used"][srcs[op]] = last
        join = ev()
        join.record(s_d2h)
        stream.wait_event(join)

    e2e_step()
    torch.cuda.synchronize()
    barrier(world)
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    s_h2d.wait_event(e_start)  # the first upload starts inside the timed region
    for _ in range(args.steps):
        e2e_step()
    e_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    e_ms = max_over_ranks(world, e_start.elapsed_time(e_end)) / args.steps
    del dy
    return {"value": round(world * step_bytes / (e_ms / 1e3) / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": nbytes["h2d"], "d2h_bytes_per_step": nbytes["d2h"], "ms_per_step": round(e_ms, 3),
            "copies": "each distinct input array uploaded once per step and read there by every operator of "
                      "its type (the one int32 array by add, min, max and xor); every output copied back; one "
                      "stream per direction, two device output buffers per operator"}


def time_call(fn, reps: int, stream):
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def minimizer_extras(dev, ctx, long_n: int = 1 << 31, with_cpu: bool = True):
    """Secondary numbers: fused minimizers (Gbp/s) and the paper-equivalent sliding minimum over
    precomputed hashes (GB/s vs HBM)."""
    import paper_1811_10074_gb300 as P
    from paper_1811_10074_gb300 import synth
    stream = torch.cuda.current_stream()
    out = {}
    peak, _ = measured_peaks()
    # plain workload: 1,000,000 bases, k=15, w=10
    n = 1_000_000
    seq = synth.acgt_uniform_packed(n, seed=42, device=dev)
    h, p, cnt = P.minimizers(seq, n, 15, 10, ctx=ctx, stream=stream, sync=False)
    ms = time_call(lambda: P.minimizers(seq, n, 15, 10, ctx=ctx, stream=stream, sync=False), 50, stream)
    out["plain_1e6"] = {"ms_per_call": round(ms, 4), "gbp_s": round(n / (ms / 1e3) / 1e9, 2),
                        "picks": int(cnt.item()), "k": 15, "w": 10,
                        "per_call": "1 cudaMemsetAsync (workspace header and tile status words) + 1 kernel "
                                    "(the single-pass kernel on packed bases: 245 tiles, one per CTA); no host "
                                    "sync; output buffers from the caching allocator"}
    # long sequence: uniform bases (default 2^31), k=15 w=10, k=19 w=10, k=15 w=50
    n = long_n
    tag = f"2^{n.bit_length() - 1}" if n & (n - 1) == 0 else str(n)
    seq = synth.acgt_uniform_packed(n, seed=43, device=dev)
    for k, w in ((15, 10), (19, 10), (15, 50)):
        out[f"fused_{tag}_k{k}_w{w}"] = fused_case(dev, ctx, n, k, w, seq=seq)
    del seq
    torch.cuda.empty_cache()
    # paper-equivalent (Sec. 4): sliding minimum over the hashed canonical 15-mers of a uniform
    # genome, 2^28 of them (sws_kmers with the hash), w = 10 and the sweep w = 4..17 (the window
    # lengths of the paper's timing figure)
    m = 1 << 28
    keys, sweep = keys_sweep(dev, ctx, m, range(4, 18))
    out["sliding_min_keys_2^28_w10"] = sweep[10]
    out["sliding_min_keys_2^28_w4_17"] = {str(w): {"ms": v["ms"], "gbs": v["gbs"], "frac_hbm": v["frac_hbm"]}
                                          for w, v in sweep.items()}
    out["keys_input"] = "2^28 hashed canonical 15-mers (sws_kmers, hash) of a uniform ACGT sequence, seed 44"
    if with_cpu:
        out["cpu_baseline"] = minimizer_cpu_baseline(keys, m, sweep)
    return out


def fused_case(dev, ctx, n: int, k: int, w: int, seq=None, reps: int = 3):
    """Minimizers of n uniform bases (seed 43) in one call: one warm-up call, then reps timed."""
    import paper_1811_10074_gb300 as P
    from paper_1811_10074_gb300 import synth
    stream = torch.cuda.current_stream()
    if seq is None:
        seq = synth.acgt_uniform_packed(n, seed=43, device=dev)
    cap = int(n * 2.6 / (w + 1)) + 1024
    ms = time_call(lambda: P.minimizers(seq, n, k, w, capacity=cap, ctx=ctx, stream=stream, sync=False), reps, stream)
    _, _, cnt = P.minimizers(seq, n, k, w, capacity=cap, ctx=ctx, stream=stream, sync=False)
    picks = int(cnt.item())
    hb = 4 if 2 * k <= 32 else 8
    bytes_ = n / 4 + picks * (hb + 4)
    return {"ms": round(ms, 3), "gbp_s": round(n / (ms / 1e3) / 1e9, 1),
            "hbm_gbs": round(bytes_ / (ms / 1e3) / 1e9, 1), "picks": picks}


def keys_sweep(dev, ctx, m: int, ws, reps: int = 5):
    """The sliding minimum with deduplicated picks over m hashed canonical 15-mers of a uniform
    sequence (seed 44) for each w in ws: ms per call (CUDA events over `reps` calls), GB/s of the
    algorithmic bytes (4 B per key in, 8 B per pick out) and their fraction of the measured HBM
    bandwidth.  Returns (keys, {w: figures})."""
    import paper_1811_10074_gb300 as P
    from paper_1811_10074_gb300 import synth
    stream = torch.cuda.current_stream()
    peak, _ = measured_peaks()
    gseq = synth.acgt_uniform_packed(m + 14, seed=44, device=dev)
    keys = P.kmers(gseq, m + 14, 15, "hash", ctx=ctx, stream=stream)
    del gseq
    sweep = {}
    for w in ws:
        cap = int(m * 2.6 / (w + 1)) + 1024
        ms = time_call(lambda: P.minimizers_from_keys(keys, w, capacity=cap, ctx=ctx, stream=stream, sync=False), reps,
                       stream)
        _, _, cnt = P.minimizers_from_keys(keys, w, capacity=cap, ctx=ctx, stream=stream, sync=False)
        picks = int(cnt.item())
        b = 4 * m + 8 * picks
        sweep[w] = {"ms": round(ms, 3), "gbs": round(b / (ms / 1e3) / 1e9, 1),
                    "frac_hbm": round(b / (ms / 1e3) / 1e9 / peak, 4), "picks": picks}
    ctx.sync(stream)
    return keys, sweep


def minimizer_cpu_baseline(keys, m, sweep, sample_keys: int = 1 << 24, sample_bases: int = 1 << 22):
    """The oracle on the host cores, on bounded samples of the same inputs: the sliding minimum
    over the first `sample_keys` hashed 15-mers for w = 4..17 as the naive per-window scan (the
    paper's "Array"), the queue-based scan ("Dequeue"), each on one core, and the naive scan
    chunked over all cores; fused minimizers (k = 15, w = 10) of `sample_bases` uniform bases on
    one core and chunked over all cores.  Units as the GPU figures (GB/s of 4 B per key in + 8 B
    per pick out; Gbp/s)."""
    import oracle
    from paper_1811_10074_gb300 import synth
    cores = os.cpu_count() or 1
    ks = keys[:sample_keys].cpu().numpy().view(np.uint32).astype(np.uint64)
    res = {"cpu_model": host_cpu_model(), "host_cores": cores, "kind": "oracle",
           "sample": f"first {sample_keys} of the GPU's 2^28 keys per w; {sample_bases} uniform bases (seed 45) "
                     f"for the fused k=15 w=10 row", "keys": {}}
    for w in range(4, 18):
        row = {}
        for name, fn, cs in (("array_1core", lambda: oracle.minimizers_from_keys(ks, w), 1),
                             ("dequeue_1core", lambda: oracle.minimizers_from_keys(ks, w, deque=True), 1),
                             (f"array_{cores}cores", lambda: oracle.minimizers_from_keys_chunked(ks, w, cores), cores)):
            t0 = time.perf_counter()
            h, _ = fn()
            dt = time.perf_counter() - t0
            row[name] = {"s": round(dt, 3), "gbs": round((4 * ks.size + 8 * h.size) / dt / 1e9, 4), "cores": cs}
        row["gpu_vs_best_cpu"] = round(sweep[w]["gbs"] / max(v["gbs"] for v in row.values()), 1)
        res["keys"][str(w)] = row
    seq = synth.acgt_uniform_packed(sample_bases, seed=45)
    fused = {}
    for name, fn, cs in (("naive_1core", lambda: oracle.minimizers(seq, sample_bases, 15, 10), 1),
                         ("dequeue_1core", lambda: oracle.minimizers(seq, sample_bases, 15, 10, deque=True), 1),
                         (f"naive_{cores}cores", lambda: oracle.minimizers_chunked(seq, sample_bases, 15, 10, cores),
                          cores)):
        t0 = time.perf_counter()
        fn()
        dt = time.perf_counter() - t0
        fused[name] = {"s": round(dt, 3), "gbp_s": round(sample_bases / dt / 1e9, 4), "cores": cs}
    res["fused_k15_w10"] = fused
    return res


def genome_table_extras(dev, ctx, n: int = 3_100_000_000, reps: int = 3, bucket_bits: int = 24):
    """Genome-scale seed table: a synthetic 3.1e9-base genome (GC 41% i.i.d., 5% of bases in
    N-blocks of log-uniform length 10 kb - 1 Mb that break windows); for k=19 w=10 and k=15 w=50
    the minimizers of the whole sequence, then the (hash, pos) hits radix-sorted into a table with
    2^bucket_bits buckets.  Gbp/s counts genome bases over minimizers + table build."""
    import paper_1811_10074_gb300 as P
    from paper_1811_10074_gb300 import synth
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    seq, iv = synth.genome_packed(n, device=dev)
    nb = torch.from_numpy(iv).to(dev)
    gen_s = time.perf_counter() - t0
    out = {"workload": f"{n} bases, GC 41%, {len(iv)} N-blocks covering {int((iv[:, 1] - iv[:, 0]).sum())} bases; "
                       f"table of 2^{bucket_bits} buckets", "generate_s": round(gen_s, 1)}
    for k, w in ((19, 10), (15, 50)):
        cap = int(n * 2.6 / (w + 1)) + 1024
        mini = lambda: P.minimizers(seq, n, k, w, nblocks=nb, capacity=cap, ctx=ctx, stream=stream, sync=False)
        ms_m = time_call(mini, reps, stream)
        h, p, cnt = mini()
        m = int(cnt.item())
        h, p = h[:m], p[:m]
        tab = lambda: P.kmer_table(h, p, 2 * k, bucket_bits, ctx=ctx, stream=stream)
        ms_t = time_call(tab, reps, stream)
        hb = h.element_size()
        out[f"k{k}_w{w}"] = {"hits": m, "minimizers_ms": round(ms_m, 2), "table_ms": round(ms_t, 2),
                             "minimizers_gbp_s": round(n / (ms_m / 1e3) / 1e9, 1),
                             "table_mhits_s": round(m / (ms_t / 1e3) / 1e6, 1),
                             "gbp_s": round(n / ((ms_m + ms_t) / 1e3) / 1e9, 1),
                             "hit_bytes": hb + 4}
        if k == 19:
            out["seeding_k19_w10"] = seeding_extras(seq, n, k, w, h, p, bucket_bits, ctx, stream, reps)
        del h, p, cnt
        torch.cuda.empty_cache()
    del seq, nb
    torch.cuda.empty_cache()
    return out


def table_skew_extras(dev, ctx, m: int, reps: int = 3, hash_bits: int = 38, bucket_bits: int = 24):
    """Seed table of m synthetic 38-bit hits spread like w = 10 minimizer picks (small hashes far
    more frequent) in the lowest quarter of the hash range, so that its buckets range from empty
    to ~4x the genome's largest: the table sort alone, a few GB on the device."""
    import paper_1811_10074_gb300 as P
    from paper_1811_10074_gb300 import synth
    stream = torch.cuda.current_stream()
    h = synth.minimizer_skew_hashes(m, hash_bits=hash_bits, w=10, drop_bits=2, device=dev)
    p = torch.arange(m, dtype=torch.int32, device=dev)
    tab = lambda: P.kmer_table(h, p, hash_bits, bucket_bits, ctx=ctx, stream=stream)
    ms = time_call(tab, reps, stream)
    return {"workload": f"{m} hits, {hash_bits}-bit hashes with the w=10 pick density in the lowest quarter "
                        f"of the range, 2^{bucket_bits} buckets", "hits": m, "table_ms": round(ms, 3),
            "table_mhits_s": round(m / (ms / 1e3) / 1e6, 1),
            "algorithmic_gb_s": round(m * 24 / (ms / 1e3) / 1e9, 1)}


def seeding_extras(seq, n, k, w, gh, gp, bucket_bits, ctx, stream, reps, n_reads: int = 1_000_000):
    """Seeding (Sec. 2.3) against the genome's seed table: 1e6 reads of 100-248 bases (multiples
    of 4) cut from the genome at byte boundaries, their minimizers in one batch, each minimizer
    looked up in the table, hits expanded with a repeat filter of 1000."""
    import paper_1811_10074_gb300 as P
    dev = seq.device
    sh, sp, off = P.kmer_table(gh, gp, 2 * k, bucket_bits, ctx=ctx, stream=stream)
    g = torch.Generator(device=dev)
    g.manual_seed(42)
    lens_b = torch.randint(25, 63, (n_reads,), generator=g, device=dev)          # bytes (4 bases each)
    starts_b = torch.randint(0, n // 4 - 64, (n_reads,), generator=g, device=dev)
    ends = torch.cumsum(lens_b, 0)
    idx = torch.repeat_interleave(starts_b - (ends - lens_b), lens_b) + torch.arange(int(ends[-1]), device=dev)
    rseq = seq[idx]
    offs = torch.cat([torch.zeros(1, dtype=torch.int64, device=dev), ends * 4])
    total = int(offs[-1])
    qh, qp, po = P.minimizers_batch(rseq, offs, total, k, w, ctx=ctx, stream=stream)
    nq = qh.shape[0]
    look = lambda: P.seed_lookup(sh, off, 2 * k, bucket_bits, qh, ctx=ctx, stream=stream)
    ms_l = time_call(look, reps, stream)
    first, count = look()
    cap = int(count.to(torch.int64).sum().item())
    hitsf = lambda: P.seed_hits(first, count, sp, 1000, capacity=cap, ctx=ctx, stream=stream, sync=False)
    ms_h = time_call(hitsf, reps, stream)
    _, _, hc = hitsf()
    nh = int(hc.item())
    return {"reads": n_reads, "read_bases": total, "query_seeds": nq, "seeds_with_hits": int((count > 0).sum().item()),
            "lookup_ms": round(ms_l, 3), "lookups_per_s": round(nq / (ms_l / 1e3) / 1e6, 1),
            "hits": nh, "hits_ms": round(ms_h, 3), "hits_per_s_m": round(nh / (ms_h / 1e3) / 1e6, 1),
            "unit": "lookups_per_s and hits_per_s_m in millions per second"}


def batch_extras(dev, ctx, n_short: int = 1_000_000, n_long: int = 20_000, plain_sample: int = 20_000, reps: int = 5,
                 tune: bool = True):
    """Batched reads: 1e6 short reads U[100,250] + 2e4 log-normal long reads (median 10 kb, max
    200 kb), k=15 w=10, in one replayed graph (autotuned unless tune is off), against plain per-read
    launches through the C ABI on a sample of reads with the same length distribution (none when
    plain_sample is 0)."""
    import ctypes
    import paper_1811_10074_gb300 as P
    from paper_1811_10074_gb300 import binding as Bd
    from paper_1811_10074_gb300 import synth
    stream = torch.cuda.current_stream()
    lens = synth.read_lengths(n_short, n_long)
    packed, offs = synth.read_batch(lens, device=dev)
    total, nreads = int(offs[-1]), len(lens)
    bt = P.Batch(nreads, total, 15, 10, options="tune" if tune else "default", ctx=ctx)
    bt.load(packed, torch.from_numpy(offs).to(dev))
    bt.run(nreads, total)
    _, _, _ = bt.results()
    picks = int(bt.count.item())
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        bt.run(nreads, total, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    bms = a.elapsed_time(b) / reps
    batched = {"reads": nreads, "bases": total, "picks": picks, "ms": round(bms, 3),
               "gbp_s": round(total / (bms / 1e3) / 1e9, 1),
               "path": ["specialized staged", "look-back", "single pass"][bt.path],
               "tuned_ms": [round(v, 3) for v in bt.tuned_ms], "graph": True}
    bt.close()
    del packed
    workload = "1e6 reads U[100,250] + 2e4 reads ln L ~ N(ln 1e4, 1), L <= 2e5; uniform ACGT; k=15 w=10"
    if plain_sample <= 0:
        return {"workload": workload, "batched_graph": batched}
    # plain: one sws_minimizers call per read, each read packed from a 16-byte boundary
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(nreads, size=min(plain_sample, nreads), replace=False))
    slens = lens[idx]
    poffs = np.zeros(len(slens) + 1, dtype=np.int64)
    np.cumsum((slens + 63) // 64 * 64, out=poffs[1:])
    pseq = synth.acgt_uniform_packed(int(poffs[-1]), seed=8, device=dev)
    cap = int(slens.max())
    hbuf = torch.empty(cap, dtype=torch.int32, device=dev)
    pbuf = torch.empty(cap, dtype=torch.int32, device=dev)
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    lib = Bd.load()
    vp = ctypes.c_void_p
    base = pseq.data_ptr()
    sh = vp(stream.cuda_stream)
    args = [(vp(base + int(poffs[i]) // 4), int(slens[i])) for i in range(len(slens))]
    hp, pp, cp = vp(hbuf.data_ptr()), vp(pbuf.data_ptr()), vp(cnt.data_ptr())

    def plain():
        for sp, L in args:
            lib.sws_minimizers(ctx.handle, sp, L, 15, 10, 0, vp(0), 0, hp, pp, cap, cp, sh)

    plain()
    torch.cuda.synchronize()
    a.record(stream)
    t0 = time.perf_counter()
    plain()
    b.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    pms = a.elapsed_time(b)
    pbases = int(slens.sum())
    plain_r = {"reads_timed": len(slens), "bases_timed": pbases, "us_per_read": round(pms * 1e3 / len(slens), 2),
               "gbp_s": round(pbases / (pms / 1e3) / 1e9, 3), "host_wall_s": round(wall, 3)}
    return {"workload": workload,
            "batched_graph": batched, "plain_per_read_launches": plain_r,
            "speedup_batched_vs_plain": round(batched["gbp_s"] / max(plain_r["gbp_s"], 1e-9), 1)}


def serve_extras(ctx, n_requests: int = 3000, duration_s: float = 1.5, p99_bound_ms: float = 20.0):
    """Serving: requests of log-uniform length in [150 bp, 1 Mbp] (k=15, w=10).  A drainer thread
    collects answers as they come (sws_server_collect: many per call, read in place in the
    server's pinned memory) and releases them.  Poisson arrivals at growing rates, each due request
    submitted as soon as its arrival time has passed (those due together in one call): p50/p99
    latency (submission to answer on the host), the client's submission lateness and the bases per
    second answered; the capacity is the highest rate still answered in full with a bounded p99."""
    import paper_1811_10074_gb300 as P
    from paper_1811_10074_gb300 import synth
    lens = synth.loguniform_lengths(n_requests, 150, 1_000_000, seed=42)
    starts = np.zeros(n_requests + 1, dtype=np.int64)
    np.cumsum((lens + 3) // 4 * 4, out=starts[1:])
    pool = synth.acgt_uniform_packed(int(starts[-1]), seed=43).numpy()
    reqs = [(pool[starts[i] // 4: (starts[i] + lens[i] + 3) // 4], int(lens[i])) for i in range(n_requests)]
    srv = P.Server(15, 10, slots=4, max_requests_per_batch=128, max_bases_per_batch=1 << 24, ctx=ctx)

    def run(arrivals, per_call=None):
        """Submit reqs[i % n] at arrivals[i] (at most per_call requests per call); return (server
        stats, bases, lateness, client span)."""
        srv.reset_stats()
        total = len(arrivals)
        state = {"got": 0, "t_last": 0.0}

        def drainer():
            while state["got"] < total:
                ids = srv.collect_raw(4096, 0.05)[0]
                if ids.size:
                    srv.release(ids)
                    state["got"] += ids.size
                    state["t_last"] = time.perf_counter()

        th = threading.Thread(target=drainer)
        th.start()
        late, bases, nxt = [], 0, 0
        t0 = time.perf_counter()
        while nxt < total:
            now = time.perf_counter() - t0
            if arrivals[nxt] > now:
                time.sleep(min(arrivals[nxt] - now, 0.001))
                continue
            due = nxt
            while due < total and arrivals[due] <= now and (per_call is None or due - nxt < per_call):
                due += 1
            batch = [reqs[i % n_requests] for i in range(nxt, due)]
            srv.submit_many(batch)
            t_sub = time.perf_counter() - t0
            late += [t_sub - arrivals[i] for i in range(nxt, due)]
            bases += sum(L for _, L in batch)
            nxt = due
        th.join()
        return srv.stats(), bases, np.array(late), state["t_last"] - t0

    run([0.0] * 256)  # warm up
    mean_len = float(np.mean(lens))

    def load(gbps, seed):
        rate = gbps * 1e9 / mean_len
        count = max(64, int(rate * duration_s))
        arrivals = list(synth.poisson_arrivals(count, rate, seed=seed))
        st, bases, late, span = run(arrivals)
        return {"offered_gbp_s": round(gbps, 3), "requests": count, "arrival_rate_per_s": round(rate, 1),
                "p50_ms": round(st["p50_s"] * 1e3, 3), "p99_ms": round(st["p99_s"] * 1e3, 3),
                "max_ms": round(st["max_s"] * 1e3, 3), "gbp_s": round(bases / span / 1e9, 3),
                "batches": int(st["batches"]),
                "client_late_p99_ms": round(float(np.percentile(late, 99)) * 1e3, 3)}

    # capacity: the highest offered rate (Poisson arrivals, rates growing by 1.15x) that is served,
    # i.e. answered at >= 97% of the offered rate with p99 within p99_bound_ms.  The ladder goes on
    # past a step whose p99 alone misses (a stall of the client or the host can do that once) and
    # stops after two steps in a row that are not answered at the offered rate.
    ladder, cap, g, step, short = [], 0.0, 8.0, 0, 0
    while step < 16 and short < 2:
        r = load(g, 100 + step)
        kept_up = r["gbp_s"] >= 0.97 * g
        ok = kept_up and r["p99_ms"] <= p99_bound_ms
        ladder.append(dict(r, sustained=ok))
        short = 0 if kept_up else short + 1
        if ok:
            cap = max(cap, r["gbp_s"])
        g *= 1.15
        step += 1
    out = {"workload": "requests log-uniform 150 bp - 1 Mbp, uniform ACGT, k=15 w=10; 4 slots, <=128 requests "
                       "and <=16 Mbp per batch; answers collected in place and released by a client thread",
           "capacity_gbp_s": round(cap, 3),
           "capacity_definition": f"highest offered rate of a ladder of Poisson loads (x1.15 steps from 8 Gbp/s, "
                                  f"{duration_s} s each, until two steps in a row fall short) answered at >= 97% "
                                  f"of it with p99 <= {p99_bound_ms} ms",
           "loads": []}
    for r in ladder:
        out["loads"].append(dict(r, offered_x_capacity=round(r["offered_gbp_s"] / cap, 3) if cap else None))
    srv.close()
    return out


# ------------------------------------------------------------------------------------------
# reference arm: the oracle on host cores
# ------------------------------------------------------------------------------------------

def run_reference(args, world, rank):
    import oracle
    oracle.build()
    ns = max(args.cpu_sample // 2, 1 << 12)
    xs = make_inputs(ns, "cpu", 42)
    cases = [(op, w) for op in OPS for w in WS]
    step_bytes = sum(case_bytes(op, w, ns) for op, w in cases)

    def step():
        for op, w in cases:
            oracle.sliding_sum(op, w, xs[op])

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    v = step_bytes / dt / 1e9
    return {
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32,u32x2,f32", "data": "synthetic (SplitMix64 seed 42)",
        "config": {"workload": WORKLOAD, "n": ns, "sample": f"{ns} elements per case (bounded sample of 2^28)"},
        "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"{ns} elements per (op, w) case, all 30 cases per step",
                         "cpu_model": host_cpu_model(), "host_cores": os.cpu_count()},
        "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse_args()
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, world, rank)), flush=True)
        return
    if args.section in ("minimizers", "fused", "keys", "table", "table-skew", "batch", "serve"):
        from paper_1811_10074_gb300 import build as B
        import paper_1811_10074_gb300 as P
        B.build()
        dev = torch.device("cuda", torch.cuda.current_device())
        ctx = P.default_context(dev.index)
        if rank == 0:
            if args.section == "keys":
                ws = [int(v) for v in args.keys_ws.split(",") if v]
                _, sweep = keys_sweep(dev, ctx, args.keys_n, ws)
                print(json.dumps({"keys": {"n": args.keys_n, "sweep": sweep}}), flush=True)
            elif args.section == "fused":
                k, w = (int(v) for v in args.fused.split(","))
                print(json.dumps({"fused": fused_case(dev, ctx, args.mini_n, k, w)}), flush=True)
            elif args.section == "minimizers":
                print(json.dumps({"minimizers": minimizer_extras(dev, ctx, args.mini_n, with_cpu=not args.no_cpu)}), flush=True)
            elif args.section == "table":
                print(json.dumps({"genome_table": genome_table_extras(dev, ctx, args.genome_n)}), flush=True)
            elif args.section == "table-skew":
                print(json.dumps({"table_skew": table_skew_extras(dev, ctx, args.table_hits)}), flush=True)
            elif args.section == "batch":
                print(json.dumps({"batched_reads": batch_extras(dev, ctx, plain_sample=args.batch_plain,
                                                                tune=not args.no_tune)}), flush=True)
            else:
                print(json.dumps({"serving": serve_extras(ctx)}), flush=True)
        return
    res = run_ours(args, world, rank, local)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
