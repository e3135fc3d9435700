#!/usr/bin/env python
"""Benchmark: MAP reconstructions per second of the layered collimated-beam
model on one GB300 (and N independent replicas under torchrun).

Workload (one step = one full reconstruction): the 4-layer scan of 256 x 512
pixels at 0.5 mm (water 20 mm / steel 12 mm / cement 40 mm / rock), 64 Tx x
16 receivers, 2048 samples at 20 MHz, 2 MHz 2-cycle pulse, direct arrivals on,
depth-varying QGGMRF prior, 50 iterations in FP32.  Synthetic data
y = A x + D g + w (SNR 20 dB) is made on the device by the library itself.

Reported: recons/s (device time of the timed steps, L2 flushed between steps),
p50/p99 latency, an end-to-end figure through the host-buffer C ABI call, the
roofline of the dominant kernel, GPU clocks sampled during the timed region,
and (rank 0, one GPU) the FP64 oracle timed on a bounded sample on the host
cores.  ``--impl reference`` times only the oracle.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP32_LANES_PER_SM = 128            # FP32 FMA lanes per SM (Blackwell)
SMEM_BYTES_PER_CLK = 128           # shared-memory load bandwidth per SM per clock
WORKLOAD = ("4-layer water/steel/cement/rock, 256x512 image @0.5 mm, 64 Tx x 16 Rx, 2048 samples "
            "@20 MHz, 2 MHz pulse, direct arrivals, depth-varying QGGMRF prior, 50 MAP iterations")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--mode", default="auto", choices=["auto", "otf", "tab"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--apply-only", type=int, default=0,
                    help="run only A x and A^T r this many times (for profiler captures) and exit")
    ap.add_argument("--workload", default="cfg1", choices=["cfg1", "batched", "served", "saft", "icd"],
                    help="cfg1: the headline workload; batched: uneven scenes through the engine vs serial "
                         "solves; served: Poisson arrivals of mixed sizes through the engine vs a serial queue")
    ap.add_argument("--requests", type=int, default=0, help="requests for the batched / served workloads")
    ap.add_argument("--source-hash", default="",
                    help="print the hash profiles/traffic.txt records for these comma-separated sources and exit")
    ap.add_argument("--scene", default="cfg1", choices=["cfg1", "cfg2"], help="workload of --apply-only")
    ap.add_argument("--spacing", type=int, default=8, help="colour spacing of --workload icd")
    ap.add_argument("--sweeps", type=int, default=10, help="sweeps of --workload icd")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"],
                    help="storage precision of the --apply-only geometry")
    return ap.parse_args()


def measured_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if none of the
    kernel's source files changed since the capture (else None)."""
    try:
        for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
            if line.startswith("#") or not line.strip():
                continue
            name, srcs, sha, rd, wr = line.split()[:5]
            if name.startswith(kernel):
                return float(rd) + float(wr) if source_hash(srcs) == sha else None
    except OSError:
        return None
    return None


def source_hash(srcs: str) -> str:
    """sha256 (first 16 hex digits) over comma-separated source files, in order."""
    import hashlib
    h = hashlib.sha256()
    for src in srcs.split(","):
        h.update(open(os.path.join(ROOT, src), "rb").read())
    return h.hexdigest()[:16]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# FP64 oracle on the host (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(scene, budget_s: float, x_img, gpu_rows=None):
    """Times the oracle on a bounded sample and extrapolates one reconstruction.

    Sample: the forward operator on a few A-scans (legs cached separately) and
    the adjoint on a block of pixels.  Returns (seconds per reconstruction,
    description, threads, rel. L2 of the GPU's sampled A-scans vs the oracle)."""
    import numpy as np
    from oracle import oracle as O
    from paper_2202_09703_gb300 import synth as S

    nthreads = os.cpu_count() or 1
    plan = O.Plan(scene, nthreads=nthreads)
    K, N = scene.K, scene.N
    ks = [0, K // 2, K - 1]
    t0 = time.perf_counter()
    yk = [plan.forward(x_img, k, k + 1)[0] for k in ks]       # legs for these positions + taps
    t_first = time.perf_counter() - t0
    t0 = time.perf_counter()
    for k in ks:
        plan.forward(x_img, k, k + 1)
    t_fwd = (time.perf_counter() - t0) / len(ks)              # one A-scan, legs cached
    legs_first = max(t_first - t_fwd * len(ks), 0.0)
    n_pos_first = len({i for k in ks for i in (k // scene.n_rx,)}) + len(ks)
    t_leg_per_pos = legs_first / max(n_pos_first, 1)          # all pixels, one position
    # adjoint on a block of pixels inside the record, sized to the budget
    rng = S.SplitMix64(7)
    npix = 256
    while True:
        pix = np.unique(rng.integers(0, min(N, 300 * scene.img_w) - 1, npix))
        bp = O.Plan(scene, pix=pix, nthreads=nthreads)
        r = S.random_vector(K * scene.M, 3)
        t0 = time.perf_counter()
        bp.backproject(r)                                      # legs for these pixels + taps
        t_b1 = time.perf_counter() - t0
        t0 = time.perf_counter()
        bp.backproject(r)
        t_b2 = time.perf_counter() - t0
        bp.close()
        if t_b1 + t_b2 > 0.3 * budget_s or npix >= N:
            break
        npix = min(N, npix * 4)
    active = min(N, 344 * scene.img_w)                        # rows whose vertical time is inside the record
    t_bwd = t_b2 * active / len(pix)
    legs_all = (t_b1 - t_b2) * active / len(pix)               # every position, every active pixel
    t_fwd_full = t_fwd * K
    n_iter = scene.n_iter
    recon = legs_all + (n_iter + 1) * t_fwd_full + n_iter * t_bwd
    desc = (f"oracle A on {len(ks)} A-scans and A^T on {len(pix)} pixels of the workload, "
            f"extrapolated to one {n_iter}-iteration reconstruction (legs once, {n_iter + 1} A, {n_iter} A^T); "
            f"{nthreads} OpenMP threads")
    err = None
    if gpu_rows is not None:
        num = sum(float(np.sum((gpu_rows[i] - yk[i]) ** 2)) for i in range(len(ks)))
        den = sum(float(np.sum(yk[i] ** 2)) for i in range(len(ks)))
        err = math.sqrt(num / den)
    plan.close()
    return recon, desc, nthreads, err, ks


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2202_09703_gb300 import synth as S
    scene = S.cfg1()
    x_img = S.phantom(scene, 0)
    times = []
    desc, nth = "", 1
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        recon, desc, nth, _, _ = oracle_sample(scene, args.cpu_seconds / 3, x_img)
        if step >= args.warmup:
            times.append(recon)
    val = len(times) / sum(times)
    out = {"impl": "reference", "metric": "recons/s", "value": val, "unit": "recons/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD},
           "cpu_baseline": {"value": val, "unit": "recons/s", "cores": nth, "kind": "oracle", "sample": desc},
           "e2e": {"value": val, "unit": "recons/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def combine_ranks(t_dev: float, wall: float, steps: int, world: int, dist=None):
    """Whole-job figures from one rank's timings: every rank takes the slowest
    rank's device time and wall time (the timed region is fenced by barriers
    on both sides), and the throughput is steps x world over that time
    (N independent replicas, weak scaling)."""
    if dist is not None and world > 1:
        import torch
        tt = torch.tensor([t_dev, wall], dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_dev, wall = float(tt[0]), float(tt[1])
    return t_dev, wall, steps * world / t_dev


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2202_09703_gb300 import build as B
    B.build()
    from paper_2202_09703_gb300 import mbir as M
    from paper_2202_09703_gb300 import synth as S

    scene = S.cfg1()
    stream = torch.cuda.current_stream()
    geo = M.Geometry(scene, mode=args.mode)
    K, Mn, N = scene.K, scene.M, scene.N

    # synthetic scan: y = A x_true + D g + w at 20 dB SNR, made by the library
    x_true = torch.as_tensor(S.phantom(scene, rank).reshape(-1), dtype=torch.float32, device=dev)
    y = torch.empty(K * Mn, dtype=torch.float32, device=dev)
    geo.forward(x_true, y)
    g_true = torch.as_tensor(S.direct_gains(scene, rank), dtype=torch.float32, device=dev) * y.abs().max()
    geo.add_direct(g_true, y)
    noise = torch.as_tensor(S.unit_noise(scene, rank).reshape(-1), dtype=torch.float32, device=dev)
    sigma = math.sqrt(float((y.double() ** 2).sum()) / (100.0 * K * Mn))
    y += sigma * noise
    x = torch.empty(N, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)

    def step():
        geo.reconstruct(y, sigma, scene.n_iter, x)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    geo.set_profiling(True)
    geo.kernel_times(reset=True)
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    kt = geo.kernel_times(reset=True)
    geo.set_profiling(False)
    lat = [a.elapsed_time(b) for a, b in ev]                 # ms per reconstruction
    t_dev = sum(lat) / 1e3
    t_dev, wall, value = combine_ranks(t_dev, wall, args.steps, world, dist)

    # end to end through the host-buffer call: H2D of y, D2H of x and g
    y_h = y.cpu().pin_memory()
    x_h = torch.empty(N, dtype=torch.float32).pin_memory()
    g_h = torch.empty(K, dtype=torch.float32).pin_memory()
    geo.reconstruct_host(y_h, sigma, scene.n_iter, x_h, g_h)
    if dist:
        dist.barrier()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(0.0)
        torch.cuda.synchronize()
        geo.reconstruct_host(y_h, sigma, scene.n_iter, x_h, g_h)
    e_wall = time.perf_counter() - e0
    if dist:
        tt = torch.tensor([e_wall], dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e_wall = float(tt[0])
    e2e = {"value": args.steps * world / e_wall, "unit": "recons/s",
           "h2d_bytes_per_step": y_h.numel() * 4, "d2h_bytes_per_step": (x_h.numel() + g_h.numel()) * 4}

    # roofline of the dominant apply kernel.  CUDA-core kernels: each tap reads
    # the four bilinear corners of the pulse table (4 x 4 B) from shared memory
    # and does 4 FMA; shared-memory bandwidth (128 B/clk/SM) binds before the
    # FP32 pipes (128 FMA/clk/SM) do, so it is their primary roofline.
    # Tensor-core kernels (taps become MMAs): the record stream is the
    # algorithmic traffic, the TAB-mode bound of the path (HBM).
    pk, src = peaks()
    pairs, taps = geo.count_taps()
    fwd_ms = kt["forward_ms"] / max(kt["forward_launches"], 1)
    bwd_ms = kt["backproject_ms"] / max(kt["backproject_launches"], 1)
    dom, dom_ms = ("forward", fwd_ms) if fwd_ms >= bwd_ms else ("backproject", bwd_ms)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = float(pk.get("sm_max_mhz", 2070.0))
    smem_peak = sm_count * SMEM_BYTES_PER_CLK * clk_mhz * 1e6 / 1e9            # GB/s
    smem_bytes = 16.0 * taps
    fp32_peak = sm_count * FP32_LANES_PER_SM * 2 * clk_mhz * 1e6 / 1e12       # TFLOP/s
    flops = 8.0 * taps
    algo_bytes = 4.0 * (N + K * Mn)                      # x and one A-scan array in HBM
    tc_dom = bool(geo.info.forward_tensor_cores if dom == "forward" else geo.info.adjoint_tensor_cores)
    roofline = {"bound": "alu", "resource": "shared-memory load bandwidth (pulse-table corners per tap)",
                "kernel": dom, "achieved": smem_bytes / (dom_ms * 1e-3) / 1e9, "peak": smem_peak,
                "unit": "GB/s", "frac": smem_bytes / (dom_ms * 1e-3) / 1e9 / smem_peak,
                "traffic": measured_traffic("forward_sorted_kernel" if dom == "forward" else
                                            "bwd_tc32_kernel" if geo.info.adjoint_tensor_cores else
                                            "backproject_kernel"),
                "traffic_note": "DRAM read+write bytes per launch (ncu); the kernel streams from L2/shared memory",
                "peak_source": f"{sm_count} SMs x {SMEM_BYTES_PER_CLK} B/clk x {clk_mhz:.0f} MHz "
                               f"(sm_max_mhz, {src})",
                "algorithmic_bytes_per_launch": smem_bytes, "taps_per_launch": taps, "active_pairs": pairs,
                "forward_ms": fwd_ms, "backproject_ms": bwd_ms,
                "fp32": {"algorithmic_flops_per_launch": flops, "achieved_tflops": flops / (dom_ms * 1e-3) / 1e12,
                         "peak_tflops": fp32_peak, "frac": flops / (dom_ms * 1e-3) / 1e12 / fp32_peak},
                "hbm": {"algorithmic_bytes_per_launch": algo_bytes,
                        "achieved_gbs": algo_bytes / (dom_ms * 1e-3) / 1e9,
                        "peak_gbs": float(pk.get("hbm_gbs", 6800.0)),
                        "frac": algo_bytes / (dom_ms * 1e-3) / 1e9 / float(pk.get("hbm_gbs", 6800.0))}}
    if tc_dom:
        # 12 B per active pair is the smallest FP32 record (delay, weight, attenuation coordinate); the
        # stored records hold 24 B (pixel, first tap | table row | flag, four bilinear weights x w) and
        # the apply reads 4 B more of gathered x (A x) or writes 4 B of contribution (A^T r)
        rec_bytes = 12.0 * pairs + algo_bytes
        hbm_peak = float(pk.get("hbm_gbs", 6800.0))
        name = "fwd_tc32_kernel" if dom == "forward" else "bwd_tc32_kernel"
        roofline = {"bound": "hbm", "resource": "HBM: the TAB record stream (latency-bound record scatter)",
                    "kernel": dom + " (tensor cores)", "achieved": rec_bytes / (dom_ms * 1e-3) / 1e9,
                    "peak": hbm_peak, "unit": "GB/s", "frac": rec_bytes / (dom_ms * 1e-3) / 1e9 / hbm_peak,
                    "traffic": measured_traffic(name),
                    "traffic_note": "DRAM read+write bytes per launch (ncu)",
                    "peak_source": f"hbm_gbs ({src})", "algorithmic_bytes_per_launch": rec_bytes,
                    "bytes_per_pair_minimum": 12, "bytes_per_pair_used": 28, "active_pairs": pairs,
                    "taps_per_launch": taps, "forward_ms": fwd_ms, "backproject_ms": bwd_ms,
                    "shared_memory_tap_model": {"achieved_gbs": smem_bytes / (dom_ms * 1e-3) / 1e9,
                                                "peak_gbs": smem_peak,
                                                "frac": smem_bytes / (dom_ms * 1e-3) / 1e9 / smem_peak}}

    # per timed reconstruction: the projection of y, then per iteration A^T r and its group reduction,
    # prior gradient, PR+ scalars, direction, A x (with the tensor cores: the record-order gather of the
    # direction, then the product kernel), projection, step, update; the ncu launch list of this command
    # agrees (501 for 50 iterations with the tensor-core A x)
    per_it = 10 if geo.info.forward_tensor_cores else 9
    launches = args.steps * (per_it * scene.n_iter + 1)

    out = {"metric": "recons/s", "value": value, "unit": "recons/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "mode": geo.mode, "iterations": scene.n_iter,
                      "forward_window_spans": geo.info.forward_window_spans,
                      "forward_window_ms": [round(t, 4) for t in geo.info.forward_window_ms],
                      "adjoint_groups": geo.info.adjoint_groups,
                      "l2": "flushed between steps (256 MB write); device time from CUDA events per step",
                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
           "latency_ms": {"p50": statistics.median(lat), "p99": float(np.percentile(lat, 99)),
                          "wall_s": wall},
           "e2e": e2e, "roofline": roofline, "clocks": clk, "gpu_launches": launches}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        xr = S.phantom(scene, 0)
        yg = torch.empty(K * Mn, dtype=torch.float32, device=dev)
        geo.forward(torch.as_tensor(xr.reshape(-1), dtype=torch.float32, device=dev), yg)
        ygn = yg.cpu().numpy().reshape(K, Mn)
        ks = [0, K // 2, K - 1]
        recon, desc, nth, err, _ = oracle_sample(scene, args.cpu_seconds, xr, gpu_rows=[ygn[k] for k in ks])
        out["cpu_baseline"] = {"value": 1.0 / recon, "unit": "recons/s", "cores": nth, "kind": "oracle",
                               "sample": desc}
        out["oracle_rel_l2_sampled_A"] = err
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def run_apply_only(args):
    import torch
    from paper_2202_09703_gb300 import build as B
    B.build()
    from paper_2202_09703_gb300 import mbir as M
    from paper_2202_09703_gb300 import synth as S
    scene = (S.cfg2() if args.scene == "cfg2" else S.cfg1()).copy(precision=args.precision)
    dev = torch.device("cuda:0")
    geo = M.Geometry(scene, mode=args.mode)
    x = torch.as_tensor(S.phantom(scene, 0).reshape(-1), dtype=torch.float32, device=dev)
    y = torch.empty(scene.K * scene.M, dtype=torch.float32 if args.precision == "fp32" else torch.bfloat16,
                    device=dev)
    b = torch.empty(scene.N, dtype=torch.float32, device=dev)
    for _ in range(args.apply_only):
        geo.forward(x, y)
        geo.backproject(y, b)
    torch.cuda.synchronize()
    # then per-apply device times: CUDA events around single calls, median of 5
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    tf, tb = [], []
    for _ in range(5):
        ev[0].record()
        geo.forward(x, y)
        ev[1].record()
        torch.cuda.synchronize()
        tf.append(ev[0].elapsed_time(ev[1]))
        ev[0].record()
        geo.backproject(y, b)
        ev[1].record()
        torch.cuda.synchronize()
        tb.append(ev[0].elapsed_time(ev[1]))
    print(json.dumps({"apply_only": args.apply_only, "scene": scene.name, "mode": geo.mode, "precision": geo.precision,
                      "forward_tensor_cores": geo.info.forward_tensor_cores,
                      "adjoint_tensor_cores": geo.info.adjoint_tensor_cores,
                      "forward_ms": sorted(tf)[2], "backproject_ms": sorted(tb)[2],
                      "y_norm": float(y.float().norm()),
                      "b_norm": float(b.norm())}))


def _synth_request(M, S, torch, scene, seed, dev, precision=None):
    """Geometry + synthetic y = A x + D g + w (20 dB) made with the library."""
    geo = M.Geometry(scene, mode="tab", precision=precision)
    K, Mn = scene.K, scene.M
    xt = torch.as_tensor(S.phantom(scene, seed).reshape(-1), dtype=torch.float32, device=dev)
    y = torch.empty(K * Mn, dtype=torch.float32, device=dev)
    geo_f = geo if geo.precision == "fp32" else M.Geometry(scene, mode="tab", precision="fp32", records=False)
    geo_f.forward(xt, y)
    if scene.direct_arrival:
        gt = torch.as_tensor(S.direct_gains(scene, seed), dtype=torch.float32, device=dev) * y.abs().max()
        geo_f.add_direct(gt, y)
    sig = math.sqrt(float((y.double() ** 2).sum()) / (100.0 * K * Mn)) + 1e-12
    y += sig * torch.as_tensor(S.unit_noise(scene, seed).reshape(-1), dtype=torch.float32, device=dev)
    if geo.precision == "bf16":
        y = y.to(torch.bfloat16)
    return geo, y, sig


def run_batched(args):
    """Uneven scenes (image sides 64-512, 2-5 layers, 8-32 receivers, 512-4096
    samples): all submitted at once to the engine, against the same solves run
    one after another through mbir_reconstruct."""
    import numpy as np
    import torch
    from paper_2202_09703_gb300 import build as B
    B.build()
    from paper_2202_09703_gb300 import mbir as M
    from paper_2202_09703_gb300 import synth as S
    dev = torch.device("cuda:0")
    n = args.requests or 48
    scenes = S.cfg3_scenes(n, seed=0)
    out = {"workload": f"batched: {n} uneven scenes (cfg3 recipe), 50 iterations each"}
    truth = [torch.as_tensor(S.phantom(sc, i).reshape(-1), dtype=torch.float32, device=dev)
             for i, sc in enumerate(scenes)]

    def image_err(xs_):
        """mean over requests of |x - x_true| / |x_true| (the synthetic phantom)"""
        return float(np.mean([float((a - t).norm() / max(float(t.norm()), 1e-30)) for a, t in zip(xs_, truth)]))
    for prec in ("fp32", "bf16"):
        reqs = [_synth_request(M, S, torch, sc, i, dev, precision=prec) for i, sc in enumerate(scenes)]
        xs = [torch.empty(sc.N, device=dev) for sc in scenes]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if prec == "fp32":
            for (geo, y, sig), x, sc in zip(reqs, xs, scenes):
                geo.reconstruct(y, sig, sc.n_iter, x)
            torch.cuda.synchronize()
            t_serial = time.perf_counter() - t0
            x_serial = [x.clone() for x in xs]
        eng = M.Engine(120 << 30)
        xe = [torch.empty(sc.N, device=dev) for sc in scenes]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for (geo, y, sig), x, sc in zip(reqs, xe, scenes):
            eng.submit(geo, y, sig, sc.n_iter, x)
        eng.run_until_idle()
        torch.cuda.synchronize()
        t_eng = time.perf_counter() - t0
        err = max(float((a - b).norm() / max(float(b.norm()), 1e-30)) for a, b in zip(xe, x_serial))
        out[prec] = {"engine_recons_per_s": n / t_eng, "engine_s": t_eng, "max_rel_diff_vs_serial_fp32": err,
                     "engine_image_rel_err_vs_truth": image_err(xe)}
        if prec == "fp32":
            out[prec]["serial_recons_per_s"] = n / t_serial
            out[prec]["serial_s"] = t_serial
            out[prec]["serial_image_rel_err_vs_truth"] = image_err(x_serial)
        eng.close()
        for geo, _, _ in reqs:          # each pass's geometries (records, tables) go before the next pass
            geo.close()
        del reqs
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "recons/s", "value": out["bf16"]["engine_recons_per_s"], "unit": "recons/s",
                      "higher_is_better": True, "data": "synthetic", "config": out}), flush=True)


def run_served(args):
    """Poisson arrivals mixing the three workload sizes (60/30/10 %), each a
    50-iteration reconstruction, served by the engine (admission capped at
    120 GB) in FP32 and in the BF16 storage form, against a serial FIFO of
    FP32 mbir_reconstruct calls on the same GPU; image error against the
    phantom reported for each."""
    import numpy as np
    import torch
    from paper_2202_09703_gb300 import build as B
    B.build()
    from paper_2202_09703_gb300 import mbir as M
    from paper_2202_09703_gb300 import synth as S
    dev = torch.device("cuda:0")
    n = args.requests or 24
    classes = [S.cfg0(), S.cfg1(), S.cfg2().copy(precision="fp32")]
    for c in classes:
        c.n_iter = 50
    pool = {ci: _synth_request(M, S, torch, c, ci, dev) for ci, c in enumerate(classes)}
    # the BF16 storage form of the same requests (same phantoms, noise and sigma)
    pool_bf = {ci: _synth_request(M, S, torch, c, ci, dev, precision="bf16") for ci, c in enumerate(classes)}
    truth = {ci: torch.as_tensor(S.phantom(c, ci).reshape(-1), dtype=torch.float32, device=dev)
             for ci, c in enumerate(classes)}
    rng = S.SplitMix64(4242)
    results = {}
    for rate in (20.0, 200.0):
        u = rng.uniform(n)
        kinds = np.where(u < 0.6, 0, np.where(u < 0.9, 1, 2))
        gaps = -np.log(1.0 - rng.uniform(n)) / rate
        arrive = np.cumsum(gaps)
        res = {}
        for mode in ("engine", "engine_bf16", "serial"):
            src = pool_bf if mode == "engine_bf16" else pool
            xs = [torch.empty(classes[k].N, device=dev) for k in kinds]
            done = [None] * n
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if mode != "serial":
                eng = M.Engine(120 << 30)
                tickets = {}
                nxt = 0
                while True:
                    now = time.perf_counter() - t0
                    while nxt < n and arrive[nxt] <= now:
                        geo, y, sig = src[kinds[nxt]]
                        tickets[nxt] = eng.submit(geo, y, sig, classes[kinds[nxt]].n_iter, xs[nxt])
                        nxt += 1
                    na, nq = eng.step()
                    for i, t in tickets.items():
                        if done[i] is None and eng.poll(t) == M.Engine.DONE:
                            done[i] = time.perf_counter() - t0
                    if nxt >= n and na == 0 and nq == 0 and all(d is not None for d in done):
                        break
                    if na == 0 and nq == 0 and nxt < n:
                        time.sleep(max(0.0, arrive[nxt] - (time.perf_counter() - t0)))
                eng.close()
            else:
                for i in range(n):
                    wait = arrive[i] - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(wait)
                    geo, y, sig = pool[kinds[i]]
                    geo.reconstruct(y, sig, classes[kinds[i]].n_iter, xs[i])
                    done[i] = time.perf_counter() - t0
            lat = np.array(done) - arrive
            torch.cuda.synchronize()
            img = float(np.mean([float((xs[i] - truth[k]).norm() / truth[k].norm()) for i, k in enumerate(kinds)]))
            res[mode] = {"recons_per_s": n / max(done), "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                         "p99_ms": 1e3 * float(np.percentile(lat, 99)), "makespan_s": float(max(done)),
                         "image_rel_err_vs_truth": img}
        results[f"{rate:g}_req_per_s"] = res
    cfg = {"workload": f"served: {n} Poisson requests per rate, sizes 64x64 / 256x512 / 512x1024 at 60/30/10 %",
           "rates": results}
    best = results["200_req_per_s"]["engine_bf16"]["recons_per_s"]
    print(json.dumps({"metric": "recons/s", "value": best, "unit": "recons/s", "higher_is_better": True,
                      "data": "synthetic", "config": cfg}), flush=True)


def run_saft(args):
    """The paper's comparison axis on the 4-layer 256x512 workload: SAFT
    (delay-and-sum, A^T y with the beam profile phi = 1, one pass) against the
    50-iteration MAP reconstruction, both from the same synthetic scan; image
    error against the phantom after the least-squares scale for SAFT (whose
    values are not reflectivities)."""
    import numpy as np
    import torch
    from paper_2202_09703_gb300 import build as B
    B.build()
    from paper_2202_09703_gb300 import mbir as M
    from paper_2202_09703_gb300 import synth as S
    dev = torch.device("cuda:0")
    scene = S.cfg1()
    geo, y, sig = _synth_request(M, S, torch, scene, 0, dev)
    saft = M.Geometry(scene.copy(beta=0.0), mode="tab")
    xt = torch.as_tensor(S.phantom(scene, 0).reshape(-1), dtype=torch.float32, device=dev)
    img = torch.empty(scene.N, device=dev)
    for _ in range(3):
        saft.backproject(y, img)
    steps = max(args.steps, 5) * 10
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(steps):
        saft.backproject(y, img)
    ev[1].record()
    torch.cuda.synchronize()
    t_saft = ev[0].elapsed_time(ev[1]) / 1e3 / steps
    x = torch.empty(scene.N, device=dev)
    ev[0].record()
    geo.reconstruct(y, sig, scene.n_iter, x)
    ev[1].record()
    torch.cuda.synchronize()
    t_mbir = ev[0].elapsed_time(ev[1]) / 1e3

    def err(a):
        a = a.double()
        t = xt.double()
        scale = float((a @ t) / max(float(a @ a), 1e-300))
        return float((scale * a - t).norm() / t.norm())

    cfg = {"workload": "SAFT vs MAP on the 4-layer 256x512 scan (64 Tx x 16 Rx, 2048 samples), synthetic phantom",
           "saft_ms_per_image": 1e3 * t_saft, "mbir_ms_per_image": 1e3 * t_mbir,
           "saft_image_rel_err_vs_truth_ls_scaled": err(img), "mbir_image_rel_err_vs_truth": float(
               (x.double() - xt.double()).norm() / xt.double().norm()),
           "mbir_image_rel_err_vs_truth_ls_scaled": err(x)}
    print(json.dumps({"metric": "SAFT images/s", "value": 1.0 / t_saft, "unit": "images/s", "higher_is_better": True,
                      "data": "synthetic", "config": cfg}), flush=True)


def run_icd(args):
    """The paper's optimiser on the 4-layer 256x512 workload: coloured ICD
    (default spacing 8: 64 colours per sweep) for 10 sweeps against the default
    50-iteration conjugate-gradient reconstruction, both from the same
    synthetic scan.  Convergence is the cost's excess over a 200-iteration
    conjugate-gradient cost, relative to that cost; image error against the
    phantom.  Device time from CUDA events, L2 flushed before each run."""
    import numpy as np
    import torch
    from paper_2202_09703_gb300 import build as B
    B.build()
    from paper_2202_09703_gb300 import mbir as M
    from paper_2202_09703_gb300 import synth as S
    dev = torch.device("cuda:0")
    scene = S.cfg1()
    geo, y, sig = _synth_request(M, S, torch, scene, 0, dev)
    xt = torch.as_tensor(S.phantom(scene, 0).reshape(-1), dtype=torch.float32, device=dev)
    x = torch.empty(scene.N, device=dev)
    spacing, sweeps = args.spacing, args.sweeps
    geo.reconstruct_icd(y, sig, 1, spacing, x)              # builds the colour lists once
    flush = torch.empty(64 * 1024 * 1024, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            flush.fill_(0.0)
            torch.cuda.synchronize()
            ev[0].record()
            out = fn()
            ev[1].record()
            torch.cuda.synchronize()
            ts.append(ev[0].elapsed_time(ev[1]))
        return float(np.median(ts)), out

    reps = max(args.steps, 3)
    for _ in range(max(args.warmup, 1)):
        geo.reconstruct_icd(y, sig, sweeps, spacing, x)
    t_icd, out = timed(lambda: geo.reconstruct_icd(y, sig, sweeps, spacing, x, want_cost=True), reps)
    e_icd = float((x - xt).norm() / xt.norm())
    c_icd = out["cost"][-1]
    t_cg, out = timed(lambda: geo.reconstruct(y, sig, scene.n_iter, x, want_cost=True), reps)
    e_cg = float((x - xt).norm() / xt.norm())
    c_cg = out["cost"][-1]
    c_ref = geo.reconstruct(y, sig, 200, x, want_cost=True)["cost"][-1]
    ex_icd, ex_cg = (c_icd - c_ref) / abs(c_ref), (c_cg - c_ref) / abs(c_ref)
    cfg = {"workload": f"coloured ICD, spacing {spacing}, {sweeps} sweeps, on the 4-layer 256x512 scan "
                       "(64 Tx x 16 Rx, 2048 samples), synthetic phantom",
           "icd_ms": t_icd, "icd_cost_excess": ex_icd, "icd_image_rel_err_vs_truth": e_icd,
           "cg_iterations": scene.n_iter, "cg_ms": t_cg, "cg_cost_excess": ex_cg, "cg_image_rel_err_vs_truth": e_cg,
           "cost_reference": "200 conjugate-gradient iterations",
           "l2": "flushed before each run (256 MB write); device time from CUDA events"}
    print(json.dumps({"metric": "ICD recons/s", "value": 1e3 / t_icd, "unit": "recons/s", "higher_is_better": True,
                      "dtype": "f32", "data": "synthetic", "config": cfg}), flush=True)


def main():
    args = parse()
    if args.source_hash:
        print(source_hash(args.source_hash))
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "served":
        run_served(args)
        return
    if args.workload == "saft":
        run_saft(args)
        return
    if args.workload == "icd":
        run_icd(args)
        return
    if args.apply_only:
        run_apply_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
