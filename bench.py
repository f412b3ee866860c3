#!/usr/bin/env python3
"""Throughput of the spike-stream reconstruction (FSR / SSR, arXiv 2412.11639) on GB300.

A step is one reconstruction of the whole workload: the default is the moving-scene
sensor stream of 250 x 400 pixels x 20000 steps with a frame every 10 steps (fp32),
SSR (order 2).  Inputs (250 MB) and outputs (800 MB) are both larger than the 129 MB L2,
so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one rank per GPU, each rank reconstructing its own replica
(weak scaling, no data-path collective); the time is the maximum over ranks.
--impl reference times the fp64 CPU oracle (the only reference implementation of this
method here) on the host cores, on a bounded sample of the same workload per step.
Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpixel-frames/s at 1 GB300 and % HBM roofline; refiner PSNR gain vs plain"
UNIT = "Gpixel-frames/s"
KERNEL = "spk_scan_kernel"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "spk_scan_traffic.txt")


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="dynamic_250x400x20000")
    ap.add_argument("--T", type=int, default=0,
                    help="cut the workload (refine mode: the evaluation stream) to its first T steps "
                         "(profiling a smaller case)")
    ap.add_argument("--rows", type=int, default=0,
                    help="reconstruct only the first ROWS rows of the same stream (fewer blocks "
                         "per SM: shows whether the scan is bound per warp or per SM)")
    ap.add_argument("--order", type=int, default=2, choices=[1, 2, 3, 4, 5],
                    help="method: 1 FSR, 2 SSR (default), 3 TFI, 4 TFP (window --tfp-window), "
                         "5 the n-order tree (--stability-order levels)")
    ap.add_argument("--tfp-window", type=int, default=32)
    ap.add_argument("--stability-order", type=int, default=3, choices=[3, 4, 5])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", choices=["single", "batch", "serve", "refine"], default="single",
                    help="single: the headline workload; batch: 64 uneven streams per launch "
                         "(CUDA graph, autotuned tile); serve: live streams arriving over time; "
                         "refine: train the learned refiner on simulated clips, then evaluate it")
    ap.add_argument("--no-refiner", action="store_true",
                    help="single mode: skip the refiner evaluation on the headline stream")
    ap.add_argument("--no-large", action="store_true",
                    help="single mode: skip the large-sensor sub-record (1000x1000x20000, fp16 "
                         "frame every step) timed after the headline workload")
    ap.add_argument("--refine-clips", type=int, default=200,
                    help="refine mode: clips to train on from scratch (0: load the packaged checkpoint)")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ distributed ----
def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(value: float, world: int) -> float:
    """Maximum of a float over all ranks (identity for a single process)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------- clocks ----
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="spk_clocks_", suffix=".csv")
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self, t0: float, t1: float):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                    ts += float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                except ValueError:
                    continue
                rows.append((ts, parts))
            os.unlink(self.path)
        except OSError:
            pass
        inside = [p for ts, p in rows if t0 - 0.05 <= ts <= t1 + 0.05] or [p for _, p in rows]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(p[2]) for p in inside if num(p[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for p in inside:
            for name, v in zip(names, p[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": num(inside[0][3]), "samples": len(inside),
                "power_w_max": max((num(p[4]) or 0.0) for p in inside),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------- inputs ----
def workload_stream(name: str, rank: int, world: int, device: int | None = None, T_cut: int = 0):
    """The workload's packed stream as a host array: made by the GPU generator when a device
    is given (the same bits as the C generator), else by the C generator (rank 0, cached in
    the temp dir)."""
    import numpy as np
    import spkgen
    w = spkgen.WORKLOADS[name]
    if T_cut:
        w = w.resized(T=T_cut, name=f"{w.name}[:{T_cut}]")
    if device is not None:
        st, _ = spkgen.make_stream_cuda(w, device=device)
        return w, st.cpu().numpy()
    cache = os.path.join(tempfile.gettempdir(), f"spk_stream_{name}_{w.T}.npy")
    if rank == 0 and not os.path.exists(cache):
        st, _ = spkgen.make_stream(w)
        tmp = cache + f".{os.getpid()}.tmp.npy"
        np.save(tmp, st)
        os.replace(tmp, cache)
    barrier(world)
    return w, np.load(cache, mmap_mode=None)


def cut_rows(w, st, rows: int):
    """The first `rows` rows of every frame of a packed stream, repacked at their own pitch
    (pixel p < rows * W keeps its bit; the bits past it in the last byte are padding)."""
    import numpy as np
    import spkgen
    if not 0 < rows <= w.H:
        raise SystemExit(f"--rows must be in 1..{w.H}")
    n = (rows * w.W + 7) // 8
    out = np.zeros((st.shape[0], spkgen.pitch(rows, w.W)), dtype=np.uint8)
    out[:, :n] = st[:, :n]
    return w.resized(H=rows, name=f"{w.name}[rows:{rows}]"), out


def measured_peak():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    cdir = os.path.join(ROOT, "paper_2412_11639_gb300", "csrc")
    for f in ("spk.cu", "spk_scan.cuh"):           # the scan kernel's translation unit
        h.update(open(os.path.join(cdir, f), "rb").read())
    return h.hexdigest()


def recorded_profile(workload: str, order: int):
    """Figures of the committed ncu capture, if it matches this source and workload (an empty
    dict otherwise): DRAM bytes per launch, ALU-pipe busy % of peak, ALU-pipe warp
    instructions per launch and the pipe's peak warp instructions per cycle (whole GPU)."""
    try:
        kv = {}
        for line in open(TRAFFIC_FILE):
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                kv[k.strip()] = v.strip()
        if (kv.get("workload") == workload and int(kv.get("order", -1)) == order
                and kv.get("source_sha256") == kernel_source_sha()):
            out = {"traffic": float(kv["dram_bytes_per_launch"])}
            for key, name in (("alu_pipe_active_pct", "alu_pct"), ("alu_warp_inst_per_launch", "alu_inst"),
                              ("alu_peak_warp_inst_per_cycle", "alu_peak_per_cycle")):
                if kv.get(key):
                    out[name] = float(kv[key])
            return out
    except (OSError, ValueError, KeyError):
        pass
    return {}


def alu_roofline(rec: dict, kern_ms: float, clk) -> dict | None:
    """The scan's binding unit, the integer ALU pipe: ALU-pipe warp instructions per launch
    (from the committed capture of this source) over the live kernel time, against the
    pipe's peak (warp instructions per cycle for the whole GPU, from the same capture) at
    the SM clock sampled during the timed region (2070 MHz, the maximum, if unsampled)."""
    if "alu_inst" not in rec or "alu_peak_per_cycle" not in rec:
        return None
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    achieved = rec["alu_inst"] / (kern_ms / 1e3) / 1e9
    peak = rec["alu_peak_per_cycle"] * mhz * 1e6 / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gwarp-inst/s",
            "frac": achieved / peak, "kernel": KERNEL, "kernel_ms": kern_ms,
            "alu_warp_inst_per_launch": rec["alu_inst"], "sm_mhz": mhz,
            "peak_source": "sm__inst_executed_pipe_alu.sum.peak_sustained x sampled SM clock",
            "from_committed_capture": os.path.relpath(TRAFFIC_FILE, ROOT)}


# ------------------------------------------------------------------ CPU oracle ----
def oracle_rate(st, w, order, pixels=None, window=32, n=3):
    """Gpixel-frames/s of the fp64 CPU oracle over the given pixels (all by default)."""
    import oracle
    t0 = time.perf_counter()
    if order == 3:
        r = oracle.tfi(st, w.H, w.W, w.T, 1.0, w.stride, pixels=pixels)
    elif order == 4:
        r = oracle.tfp(st, w.H, w.W, w.T, window, 1.0, w.stride, pixels=pixels)
    else:
        r = oracle.reconstruct(st, w.H, w.W, w.T, 1.0, n if order == 5 else order, w.stride, pixels=pixels,
                               frames=True)
    dt = time.perf_counter() - t0
    npix = w.P if pixels is None else len(pixels)
    del r
    return npix * w.T_out / dt / 1e9, dt, npix


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# --------------------------------------------------------------------- arms ----
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import numpy as np
    w, st = workload_stream(args.workload, 0, 1, T_cut=args.T)
    chunk = 1024
    starts = np.arange(0, w.P, chunk)
    for i in range(args.warmup):
        s0 = starts[i % len(starts)]
        oracle_rate(st, w, args.order, np.arange(s0, min(s0 + chunk, w.P)), args.tfp_window, args.stability_order)
    t0 = time.perf_counter()
    units = 0
    for i in range(args.steps):
        s0 = starts[i % len(starts)]
        pix = np.arange(s0, min(s0 + chunk, w.P))
        oracle_rate(st, w, args.order, pix, args.tfp_window, args.stability_order)
        units += len(pix) * w.T_out
    dt = time.perf_counter() - t0
    value = units / dt / 1e9
    cores = host_cores()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": config_of(w, args.order, args.tfp_window, args.stability_order),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{chunk} pixels x {w.T_out} frames per step, rotating over the "
                                   f"{w.P} pixels of {w.name}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


METHODS = {1: "FSR", 2: "SSR", 3: "TFI", 4: "TFP", 5: "n-order"}


def config_of(w, order, window=32, n=3):
    name = METHODS[order] + (f"-{window}" if order == 4 else "") + (f" n={n}" if order == 5 else "")
    return {"workload": w.name, "H": w.H, "W": w.W, "T": w.T, "frame_stride": w.stride,
            "T_out": w.T_out, "out_dtype": w.out_dtype, "method": name,
            "threshold": 1.0, "parallelism": "replicas, one per GPU",
            "l2": "inputs and outputs larger than the 129 MB L2 (no flush)"}


def large_sensor_record(local_rank: int, order: int, steps: int = 3, warmup: int = 2):
    """The HBM-heaviest workload, 1000 x 1000 pixels x 20000 steps with an fp16 frame every
    step (2.5 GB in, 40 GB out per launch), timed with CUDA events on the launching stream,
    with its own HBM roofline."""
    import torch

    import paper_2412_11639_gb300 as pkg
    import spkgen
    from paper_2412_11639_gb300 import spk
    w = spkgen.WORKLOADS["large_1000x1000x20000"]
    dev, _ = spkgen.make_stream_cuda(w, device=local_rank)
    R = pkg.Reconstructor(order=order, stride=w.stride, dtype=torch.float16, device=local_rank)
    out = R.alloc_frames(w.H, w.W, w.T)
    for _ in range(warmup):
        R(dev, w.H, w.W, w.T, 1.0, out=out)
    R.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    n0 = spk.spk_launch_count(R.ctx)
    for a, b in ev:
        a.record(R.stream)
        R(dev, w.H, w.W, w.T, 1.0, out=out)
        b.record(R.stream)
    torch.cuda.synchronize()
    R.synchronize()
    launches = spk.spk_launch_count(R.ctx) - n0
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    R.close()
    del out, dev
    torch.cuda.empty_cache()
    alg_bytes = w.P * w.T / 8 + w.P * w.T_out * 2
    peak, peak_kind = measured_peak()
    achieved = alg_bytes / (ms / 1e3) / 1e9
    return {"workload": w.name, "method": METHODS[order], "out_dtype": "f16", "frame_stride": 1,
            "value": w.P * w.T_out / (ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "warmup": warmup, "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
                         "kernel": KERNEL, "kernel_ms": ms, "algorithmic_bytes_per_launch": alg_bytes}}


def host_link(h_in, h_out, units: int, reps: int = 5) -> dict:
    """This machine's host link, measured with the e2e's own page-locked buffers: plain copies of
    the step's input to the device and of its frames back, each timed alone (CUDA events, a
    side stream; the link is shared with other users of the machine, so the best and the
    median of the copies are given), and the throughput a step could reach if it were only
    those copies, overlapped, at the best rates."""
    import statistics

    import torch
    s = torch.cuda.Stream()
    d_in = torch.empty(h_in.numel(), dtype=h_in.dtype, device="cuda")
    d_out = torch.empty(h_out.numel(), dtype=h_out.dtype, device="cuda")
    best, med = {}, {}
    with torch.cuda.stream(s):
        for name, f, nbytes in (("h2d", lambda: d_in.copy_(h_in.view(-1), non_blocking=True),
                                 h_in.numel() * h_in.element_size()),
                                ("d2h", lambda: h_out.view(-1).copy_(d_out, non_blocking=True),
                                 h_out.numel() * h_out.element_size())):
            f()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            for a, b in ev:
                a.record(s)
                f()
                b.record(s)
            s.synchronize()
            rates = [nbytes / (a.elapsed_time(b) / 1e3) / 1e9 for a, b in ev]
            best[name], med[name] = max(rates), statistics.median(rates)
    del d_in, d_out
    t = max(h_in.numel() * h_in.element_size() / (best["h2d"] * 1e9),      # seconds per step
            h_out.numel() * h_out.element_size() / (best["d2h"] * 1e9))
    return {"h2d_GBps": best["h2d"], "d2h_GBps": best["d2h"], "h2d_GBps_median": med["h2d"],
            "d2h_GBps_median": med["d2h"], "copy_bound_value": units / t / 1e9, "unit": UNIT}


def methods_record(dev, w, local_rank: int, steps: int = 5, warmup: int = 3):
    """The other reconstruction methods on the same resident stream and frame layout (FSR,
    the TFI and TFP baselines, the n-order tree at n = 3, 4, 5), each timed with CUDA events
    on its launching stream."""
    import torch

    import paper_2412_11639_gb300 as pkg
    from paper_2412_11639_gb300 import spk
    dtype = torch.float16 if w.out_dtype == "f16" else torch.float32
    rec = {}
    for name, order, n in (("FSR", 1, 3), ("TFI", 3, 3), ("TFP-32", 4, 3), ("n-order n=3", 5, 3),
                           ("n-order n=4", 5, 4), ("n-order n=5", 5, 5)):
        R = pkg.Reconstructor(order=order, stride=w.stride, dtype=dtype, device=local_rank,
                              tfp_window=32, stability_order=n)
        out = R.alloc_frames(w.H, w.W, w.T)
        for _ in range(warmup):
            R(dev, w.H, w.W, w.T, 1.0, out=out)
        R.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        n0 = spk.spk_launch_count(R.ctx)
        for a, b in ev:
            a.record(R.stream)
            R(dev, w.H, w.W, w.T, 1.0, out=out)
            b.record(R.stream)
        torch.cuda.synchronize()
        R.synchronize()
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        rec[name] = {"ms_per_step": ms, "value": w.P * w.T_out / (ms / 1e3) / 1e9, "unit": UNIT,
                     "gpu_launches": spk.spk_launch_count(R.ctx) - n0, "steps": steps}
        R.close()
        del out
    return {"workload": w.name, "out_dtype": w.out_dtype, "frame_stride": w.stride, "methods": rec}


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2412_11639_gb300 as pkg
    from paper_2412_11639_gb300 import spk

    torch.cuda.set_device(local_rank)
    w, st = workload_stream(args.workload, rank, world, device=local_rank, T_cut=args.T)
    if args.rows:
        w, st = cut_rows(w, st, args.rows)
    dtype = torch.float16 if w.out_dtype == "f16" else torch.float32
    esz = 2 if dtype == torch.float16 else 4
    R = pkg.Reconstructor(order=args.order, stride=w.stride, dtype=dtype, device=local_rank,
                          tfp_window=args.tfp_window, stability_order=args.stability_order)
    dev = torch.from_numpy(st).cuda()
    out = R.alloc_frames(w.H, w.W, w.T)
    stream = R.stream

    for _ in range(args.warmup):
        R(dev, w.H, w.W, w.T, 1.0, out=out)
    R.synchronize()

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local_rank) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    n0 = spk.spk_launch_count(R.ctx)
    t0 = time.time()
    e0.record(stream)
    for i in range(K):
        ev[i][0].record(stream)
        R(dev, w.H, w.W, w.T, 1.0, out=out)
        ev[i][1].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    barrier(world)
    R.synchronize()
    launches = spk.spk_launch_count(R.ctx) - n0
    total_ms = max_over_ranks(e0.elapsed_time(e1), world)
    kern_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    clk = clocks.stop(t0, t1) if clocks else None

    units = w.P * w.T_out * K * world
    value = units / (total_ms / 1e3) / 1e9
    alg_bytes = w.P * w.T / 8 + w.P * w.T_out * esz
    peak, peak_kind = measured_peak()
    achieved = alg_bytes / (kern_ms / 1e3) / 1e9

    # end to end through the public C ABI with pinned host buffers (copies timed)
    e2e = None
    if args.e2e_steps > 0:
        # every step copies its input from pinned host memory and its frames back; the calls
        # are asynchronous and alternate between two lanes, so that a step's device-to-host
        # copy overlaps the next step's input copy and scan
        h_in = torch.from_numpy(st).pin_memory()
        h_out = [torch.empty((w.T_out, w.H, w.W), dtype=dtype).pin_memory() for _ in range(2)]
        for k in range(2):
            spk.spk_reconstruct_host_async(R.ctx, h_in, w.H, w.W, w.T, 1.0, h_out[k])
        spk.spk_synchronize(R.ctx)
        barrier(world)
        te0 = time.perf_counter()
        for k in range(args.e2e_steps):
            spk.spk_reconstruct_host_async(R.ctx, h_in, w.H, w.W, w.T, 1.0, h_out[k % 2])
        spk.spk_synchronize(R.ctx)
        te_dt = max_over_ranks(time.perf_counter() - te0, world)
        t1 = time.perf_counter()
        spk.spk_reconstruct_host(R.ctx, h_in, w.H, w.W, w.T, 1.0, h_out[0])
        one_call = time.perf_counter() - t1
        e2e = {"value": w.P * w.T_out * args.e2e_steps * world / te_dt / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(st.nbytes), "d2h_bytes_per_step": int(h_out[0].numel() * esz),
               "api": "spk_reconstruct_host_async x steps, then spk_synchronize",
               "single_call_ms": one_call * 1e3,
               "link": host_link(h_in, h_out[0], w.P * w.T_out)}
    R.close()

    refined = None
    if (rank == 0 and not args.no_refiner and w.name == "dynamic_250x400x20000" and args.order == 2):
        from paper_2412_11639_gb300 import refiner
        if os.path.exists(refiner.CHECKPOINT):
            rec2 = pkg.Reconstructor(order=2, stride=w.stride, device=local_rank)
            ref = refiner.Refiner(device=local_rank)
            ref.load(refiner.CHECKPOINT)
            refined = refiner_eval(ref, rec2, w)
            ref.close()
            rec2.close()
        else:
            refined = {"unavailable": "no trained checkpoint in the package"}

    large = methods = None
    if (rank == 0 and not args.no_large and w.name == "dynamic_250x400x20000" and not args.T
            and not args.rows and args.order in (1, 2)):
        methods = methods_record(dev, w, local_rank)
        large = large_sensor_record(local_rank, args.order)

    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        import numpy as np

        import oracle
        v, dt, npix = oracle_rate(st, w, args.order, window=args.tfp_window, n=args.stability_order)
        cpu = {"value": v, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
               "sample": f"the whole workload once ({npix} pixels x {w.T_out} frames, {dt:.1f} s)"}
        oracle.set_threads(1)   # the same oracle on one core, on the first 2048 pixels
        v1, dt1, n1 = oracle_rate(st, w, args.order, np.arange(min(2048, w.P)), args.tfp_window,
                                  args.stability_order)
        oracle.set_threads(0)
        cpu["single_core"] = {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": f"{n1} pixels x {w.T_out} frames, {dt1:.1f} s"}
    rec = recorded_profile(w.name, args.order)
    traffic, alu_pct = rec.get("traffic"), rec.get("alu_pct")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "input_Gpixel_steps_per_s": w.P * w.T * K * world / (total_ms / 1e3) / 1e9,
        "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i32+f32", "data": "synthetic",
        "config": config_of(w, args.order, args.tfp_window, args.stability_order),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "kernel": "spk_tfp_kernel" if args.order == 4 else KERNEL, "kernel_ms": kern_ms,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     # traffic and the ALU-pipe load are not measured by this run: they come
                     # from the ncu capture committed under profiles/ for this same kernel
                     # source and workload (null once the kernel has changed)
                     "from_committed_capture": {
                         "file": os.path.relpath(TRAFFIC_FILE, ROOT), "fields": ["traffic"],
                         "alu_pipe_busy_pct_of_peak": alu_pct}},
        "alu_roofline": alu_roofline(rec, kern_ms, clk),
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "refiner": refined,
        "large_sensor": large,
        "other_methods": methods,
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------- learned refiner ----
# multiply-adds per pixel-frame of the network as defined (inputs: the plain value and four
# interval rates): 3x3 x (5*32 + 3*32*32 + 32*1); the kernels pad 5 -> 16 input and 1 -> 16
# output channels to the tensor-core k16/n8 shapes and so execute 3x3 x (16*32 + 3*32*32 + 32*16)
REFINER_MACS = 9 * (5 * 32 + 3 * 32 * 32 + 32 * 1)
REFINER_MACS_PADDED = 9 * (16 * 32 + 3 * 32 * 32 + 32 * 16)


def refiner_eval(ref, rec, w, chunk: int = 0, reps: int = 3, ssim_every: int = 20, skip: int = 20):
    """Refined vs plain frames of workload w against its ground truth, and the refiner's
    device throughput (features + forward) with CUDA events.  chunk: frames per forward
    call (0: all frames in one call, the fastest; smaller chunks leave SMs idle at the end of
    every layer)."""
    chunk = chunk or w.T_out
    import numpy as np
    import torch

    import spkgen
    from paper_2412_11639_gb300 import quality, refiner
    stream, gt = spkgen.make_stream_cuda(w, gt_stride=w.stride, device=ref.device)
    gt = gt.view(w.T_out, w.H, w.W)
    plain = rec(stream, w.H, w.W, w.T)
    x0 = refiner.features(rec, stream, w.H, w.W, w.T, plain)
    out = torch.empty_like(plain)
    cs = rec.stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def run():
        ev[0].record(cs)
        refiner.spk.spk_features(rec.ctx, stream, w.H, w.W, w.T, 1.0, plain, x0)
        ev[1].record(cs)
        for k in range(0, w.T_out, chunk):
            n = min(chunk, w.T_out - k)
            refiner.spk.spk_refiner_forward(ref.r, cs.cuda_stream, x0[k:k + n], plain[k:k + n], n, w.H, w.W,
                                            out[k:k + n])
        ev[2].record(cs)
    run()
    torch.cuda.synchronize()
    feat_ms, fwd_ms = [], []
    for _ in range(reps):
        run()
        torch.cuda.synchronize()
        feat_ms.append(ev[0].elapsed_time(ev[1]))
        fwd_ms.append(ev[1].elapsed_time(ev[2]))
    fm, gm = statistics.median(feat_ms), statistics.median(fwd_ms)
    pf = w.P * w.T_out

    def psnr_dev(a):
        mse = torch.mean((a[skip:].double() - gt[skip:].double()) ** 2).item()
        return 10 * np.log10(1.0 / mse)
    sel = slice(skip, w.T_out, ssim_every)
    g_h = gt[sel].cpu().numpy()
    res = {"checkpoint": os.path.relpath(refiner.CHECKPOINT, ROOT),
           "eval_stream": w.name, "frames_scored": w.T_out - skip,
           "psnr_plain_db": psnr_dev(plain), "psnr_refined_db": psnr_dev(out),
           "ssim_plain": quality.ssim(plain[sel].cpu().numpy(), g_h),
           "ssim_refined": quality.ssim(out[sel].cpu().numpy(), g_h),
           "ssim_frames": len(range(w.T_out)[sel]),
           "throughput_Gpf_s": pf / ((fm + gm) / 1e3) / 1e9,
           "features_ms": fm, "forward_ms": gm, "forward_launches": 5 * ((w.T_out + chunk - 1) // chunk)}
    res["psnr_gain_db"] = res["psnr_refined_db"] - res["psnr_plain_db"]
    peak = bf16_peak()
    tf = pf * 2 * REFINER_MACS / (gm / 1e3) / 1e12
    tfp = pf * 2 * REFINER_MACS_PADDED / (gm / 1e3) / 1e12
    res["roofline"] = {"bound": "tensor", "achieved": tf, "peak": peak[0], "unit": "TFLOP/s", "frac": tf / peak[0],
                       "peak_source": peak[1], "executed_TFLOP_s": tfp,
                       "flop_per_pixel_frame": 2 * REFINER_MACS,
                       "executed_flop_per_pixel_frame": 2 * REFINER_MACS_PADDED}
    del x0, stream
    return res


def bf16_peak():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["bf16_tflops"]), "measured bf16_tflops (burst)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def run_refine(args):
    """Train the refiner on freshly simulated clips, then evaluate it on the headline stream."""
    import torch

    import paper_2412_11639_gb300 as pkg
    import spkgen
    from paper_2412_11639_gb300 import refiner
    base = spkgen.WORKLOADS["dynamic_250x400x20000"]
    if args.T:                           # evaluate on the stream's first T steps (profiling)
        base = base.resized(T=args.T, name=f"{base.name}[:{args.T}]")
    rec = pkg.Reconstructor(order=2, stride=base.stride)
    ref = refiner.Refiner(seed=0)
    if args.refine_clips == 0:           # evaluate (and time) the committed checkpoint
        ref.load(refiner.CHECKPOINT)
    clip = base.resized(T=2000)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = refiner.train_on_simulator(ref, rec, clip, args.refine_clips, steps_per_clip=2, batch=16) or [None]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    res = refiner_eval(ref, rec, base)
    # the training step alone (features and clips excluded), timed with CUDA events on a
    # copy of the refiner (the timing steps must not move the evaluated weights)
    ref.save(os.path.join(tempfile.gettempdir(), f"spk_refiner_{os.getpid()}.npy"))
    ref.close()
    ref = refiner.Refiner(seed=0)
    x0, plain, gt = refiner.simulator_clip(rec, clip.resized(seed=999))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        ref.train_step(x0[:16], plain[:16], gt[:16], 1e-5, want_loss=False)
    e0.record(ref.stream)
    for _ in range(10):
        ref.train_step(x0[:16], plain[:16], gt[:16], 1e-5, want_loss=False)
    e1.record(ref.stream)
    torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / 10
    line = {"mode": "refine", "metric": "refiner PSNR gain vs plain (dB) and throughput",
            "training": {"clips": args.refine_clips, "clip": f"{clip.H}x{clip.W}x{clip.T} stride {clip.stride}",
                         "steps": 2 * args.refine_clips, "batch_frames": 16, "seconds": dt,
                         "first_loss": losses[0], "last_loss": losses[-1],
                         "train_step_ms": step_ms,
                         "train_Gpf_s": 16 * clip.P / (step_ms / 1e3) / 1e9},
            "refiner": res, "data": "synthetic"}
    print(json.dumps(line), flush=True)
    ref.close()
    rec.close()
    return 0


# ------------------------------------------------------------- extra modes ----
def _distinct_streams(specs):
    """Moving-scene streams of the given sizes and seeds, made by the GPU generator (the
    same bits as the C generator), as host arrays."""
    import spkgen
    out = []
    for (H, W, T, seed) in specs:
        w = spkgen.WORKLOADS["dynamic_250x400x20000"].resized(H=H, W=W, T=T, seed=seed)
        out.append((H, W, T, spkgen.make_stream_cuda(w)[0].cpu().numpy()))
    return out


def run_batch(args):
    """64 distinct streams of uneven size and length reconstructed in one launch per step."""
    import numpy as np
    import torch

    import paper_2412_11639_gb300 as pkg
    import spkgen
    from paper_2412_11639_gb300 import spk
    rng = np.random.default_rng(11)
    # 64 seeded moving-scene streams, sizes from 128 x 128 to 1000 x 1000 (both ends
    # included), lengths 2000 .. 20000 steps; each made on the device by the GPU generator
    specs = [(int(rng.integers(128, 1001)), int(rng.integers(128, 1001)), int(rng.integers(2000, 20001)), 40 + k)
             for k in range(64)]
    specs[0] = (128, 128) + specs[0][2:]
    specs[-1] = (1000, 1000) + specs[-1][2:]
    base = spkgen.WORKLOADS["dynamic_250x400x20000"]
    dev = [spkgen.make_stream_cuda(base.resized(H=H, W=W, T=T, seed=seed))[0] for (H, W, T, seed) in specs]
    side = torch.cuda.Stream()
    R = pkg.Reconstructor(order=args.order, stride=10, dtype=torch.float16, stream=side)
    jobs, outs = [], []
    for (H, W, T, _), d in zip(specs, dev):
        o = R.alloc_frames(H, W, T)
        jobs.append((d, H, W, T, 1.0, o, None))
        outs.append(o)
    tile = spk.spk_autotune(R.ctx, jobs)
    with torch.cuda.stream(side):
        pkg.spk_run(R.ctx, jobs)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        pkg.spk_run(R.ctx, jobs)
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(1, min(args.steps, 20))
    e0.record()
    for _ in range(steps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    R.synchronize()
    ms = e0.elapsed_time(e1) / steps
    units = sum(o.numel() for o in outs)
    # every one of the 64 jobs equals its stream reconstructed alone
    R1 = pkg.Reconstructor(order=args.order, stride=10, dtype=torch.float16)
    same = 0
    for (H, W, T, _), d, o in zip(specs, dev, outs):
        alone = R1(d, H, W, T, 1.0)
        R1.synchronize()
        same += bool(torch.equal(alone.view(torch.int16), o.view(torch.int16)))
        del alone
    alg_bytes = sum(d.numel() for d in dev) + 2 * units
    peak, peak_kind = measured_peak()
    line = {"mode": "batch", "metric": "Gpixel-frames/s, 64 uneven streams per launch", "value": units / ms / 1e6,
            "unit": "Gpixel-frames/s", "ms_per_step": ms, "steps": steps, "tile": tile, "graph": True,
            "streams": len(specs), "distinct_streams": len(set(s[3] for s in specs)),
            "sizes": [s[:3] for s in specs], "input_bytes": int(sum(d.numel() for d in dev)),
            "frame_stride": 10, "out_dtype": "f16", "method": "SSR" if args.order == 2 else "FSR",
            "alg_GBps": alg_bytes / ms / 1e6, "hbm_frac": alg_bytes / ms / 1e6 / peak,
            "peak_source": f"{peak_kind} hbm_gbs", "jobs_equal_to_alone": same,
            "same_as_alone": same == len(specs), "data": "synthetic"}
    print(json.dumps(line), flush=True)
    R1.close()
    R.close()
    return 0


def run_serve(args):
    """Live 250x400 streams arriving over time at the camera's real-time 20 kHz."""
    import numpy as np

    from paper_2412_11639_gb300.serving import Request, Server
    rng = np.random.default_rng(12)
    distinct = _distinct_streams([(250, 400, 20000, 60 + k) for k in range(3)])
    reqs, t = [], 0.0
    for k in range(24):
        H, W, T, st = distinct[k % len(distinct)]
        T_k = int(rng.integers(2000, 20001))
        t += float(rng.exponential(1.0 / 12.0))
        reqs.append(Request(k, np.ascontiguousarray(st[:T_k]), H, W, arrival=t, rate=20000.0))
    srv = Server(order=args.order, stride=10, mem_budget=4 << 30, max_streams=32, max_piece=2048)
    st = srv.run(reqs)
    line = {"mode": "serve", "metric": "per-frame latency at 20 kHz live streams", "requests": len(reqs),
            "sensor": "250x400", "rate_steps_per_s": 20000, "arrivals_per_s": 12.0,
            "p50_ms": st.p50_ms, "p99_ms": st.p99_ms, "max_ms": st.max_ms,
            "pixel_frames": st.pixel_frames, "wall_s": st.wall_s, "busy_s": st.busy_s,
            "throughput_Gpf_s": st.pixel_frames / st.wall_s / 1e9,
            "device_throughput_Gpf_s": st.pixel_frames / st.busy_s / 1e9,
            "launches": st.launches, "peak_active": st.peak_active, "admission_wait_s": st.admitted_late_s,
            "frame_stride": 10, "method": "SSR" if args.order == 2 else "FSR", "data": "synthetic"}
    print(json.dumps(line), flush=True)
    srv.close()
    return 0


def main(argv=None):
    args = parse_args(argv)
    rank, world, local_rank = dist_env()
    if args.mode != "single" and args.impl == "ours":
        if world > 1 and rank != 0:
            return 0
        return {"batch": run_batch, "serve": run_serve, "refine": run_refine}[args.mode](args)
    if world > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl" if torch.cuda.is_available() and args.impl == "ours" else "gloo")
    try:
        if args.impl == "reference":
            return run_reference(args, rank, world)
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
