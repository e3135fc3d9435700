#!/usr/bin/env python
"""Benchmark: MAP reconstructions per second of the layered collimated-beam
model on one GB300 (and N independent replicas under torchrun).

Workload (one step = one full reconstruction): the 4-layer scan of 512 x 1024
pixels at 0.25 mm (water 20 mm / steel 12 mm / cement 40 mm / rock), 128 Tx x
32 receivers, 4096 samples at 20 MHz, 2 MHz 2-cycle pulse, direct arrivals on,
depth-varying QGGMRF prior, 50 iterations in FP32 - the largest of the
workloads that fits one GPU.  Synthetic data y = A x + D g + w (SNR 20 dB) is
made on the device by the library itself.

Reported: recons/s (device time of the timed steps, L2 flushed between steps),
p50/p99 latency, an end-to-end figure through the host-buffer C ABI call, the
roofline of the dominant kernel, GPU clocks sampled during the timed region,
the geometry set-up time, and (rank 0, one GPU) the FP64 oracle timed on a
bounded sample on the host cores.  Beside the headline (one GPU): the same
workload in the BF16 storage form with its image error against the FP32 form,
the 256 x 512 workload, the on-the-fly (OTF) applies, and a served stream of
Poisson arrivals through the engine against serial FP32 solves.
``--impl reference`` times only the oracle.
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
WORKLOADS = {
    "cfg2": ("4-layer water/steel/cement/rock, 512x1024 image @0.25 mm, 128 Tx x 32 Rx, 4096 samples "
             "@20 MHz, 2 MHz pulse, direct arrivals, depth-varying QGGMRF prior, 50 MAP iterations, FP32"),
    "cfg1": ("4-layer water/steel/cement/rock, 256x512 image @0.5 mm, 64 Tx x 16 Rx, 2048 samples "
             "@20 MHz, 2 MHz pulse, direct arrivals, depth-varying QGGMRF prior, 50 MAP iterations, FP32"),
}


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
    ap.add_argument("--workload", default="cfg2", choices=["cfg2", "cfg1", "batched", "served", "saft", "icd"],
                    help="cfg2: the headline workload (512x1024); cfg1: the 256x512 workload; batched: uneven "
                         "scenes through the engine vs serial solves; served: Poisson arrivals of mixed sizes "
                         "through the engine vs a serial queue")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only: skip the BF16 form, the 256x512 and OTF figures and the served stream")
    ap.add_argument("--served-requests", type=int, default=100, help="requests per rate of the served figure")
    ap.add_argument("--requests", type=int, default=0, help="requests for the batched / served workloads")
    ap.add_argument("--rates", default="20,200", help="arrival rates (req/s) of --workload served")
    ap.add_argument("--geometries", type=int, default=1, help="distinct scans per size class of --workload served")
    ap.add_argument("--source-hash", default="",
                    help="print the hash profiles/traffic.txt records for these comma-separated sources and exit")
    ap.add_argument("--scene", default="cfg1", choices=["cfg1", "cfg2"], help="workload of --apply-only")
    ap.add_argument("--spacing", type=int, default=8, help="colour spacing of --workload icd")
    ap.add_argument("--sweeps", type=int, default=10, help="sweeps of --workload icd")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"],
                    help="storage precision of the --apply-only geometry")
    return ap.parse_args()


def measured_traffic(kernel: str, pairs: float):
    """DRAM bytes per launch from the committed ncu summary (a capture of a
    smaller workload, scaled to this one by its active pairs: the record
    stream is the traffic), if none of the kernel's source files changed
    since the capture (else None)."""
    try:
        for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
            if line.startswith("#") or not line.strip():
                continue
            name, srcs, sha, rd, wr, cap_pairs = line.split()[:6]
            if name == kernel:
                if source_hash(srcs) != sha:
                    return None
                return (float(rd) + float(wr)) * pairs / float(cap_pairs)
    except (OSError, ValueError):
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
def oracle_sample(scene, budget_s: float, x_img):
    """Times the oracle on a bounded sample and extrapolates one reconstruction.

    Sample: a uniformly random set P of pixels, grown until the sample takes
    about half the budget: the oracle's legs from every transducer position to
    P, its A over every A-scan with the image restricted to P, and its A^T on
    P.  Each cost is proportional to the pixels (pairs) it covers, so one
    reconstruction (legs once, n_iter + 1 A, n_iter A^T) is the sample scaled
    by N / |P|.  Returns (seconds per reconstruction, description, threads,
    P, the oracle's A of the image restricted to P)."""
    import numpy as np
    from oracle import oracle as O
    from paper_2202_09703_gb300 import synth as S

    nthreads = os.cpu_count() or 1
    K, N = scene.K, scene.N
    r = S.random_vector(K * scene.M, 3)
    xf = np.asarray(x_img, np.float64).reshape(-1)
    npix = 64
    while True:
        pix = np.unique(S.SplitMix64(7).integers(0, N - 1, npix))
        plan = O.Plan(scene, pix=pix, nthreads=nthreads)
        t0 = time.perf_counter()
        plan.backproject(r)                                    # legs of every position to P, then the taps
        t_b1 = time.perf_counter() - t0
        t0 = time.perf_counter()
        plan.backproject(r)
        t_b2 = time.perf_counter() - t0
        t0 = time.perf_counter()
        y_p = plan.forward(xf)                                 # every A-scan, the image on P only
        t_f = time.perf_counter() - t0
        plan.close()
        if t_b1 + t_b2 + t_f > 0.5 * budget_s or npix >= N:
            break
        npix = min(N, npix * 4)
    scale = N / len(pix)
    n_iter = scene.n_iter
    recon = scale * ((t_b1 - t_b2) + (n_iter + 1) * t_f + n_iter * t_b2)
    desc = (f"oracle legs (every transducer position), A (all {K} A-scans) and A^T on {len(pix)} random pixels "
            f"of the workload, scaled by N/|P| = {scale:.1f} to one {n_iter}-iteration reconstruction (legs once, "
            f"{n_iter + 1} A, {n_iter} A^T); {nthreads} OpenMP threads")
    return recon, desc, nthreads, pix, y_p


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2202_09703_gb300 import synth as S
    scene = S.cfg1() if args.workload == "cfg1" else S.cfg2().copy(precision="fp32")
    x_img = S.phantom(scene, 0)
    times, walls = [], []
    desc, nth = "", 1
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        recon, desc, nth, _, _ = oracle_sample(scene, args.cpu_seconds / 3, x_img)
        if step >= args.warmup:
            times.append(recon)
            walls.append(time.perf_counter() - t0)
    val = len(times) / sum(times)
    wl = "cfg1" if args.workload == "cfg1" else "cfg2"
    # a step is one bounded sample of the workload (its wall time is ms_per_step); the value is the
    # reconstructions per second that the samples extrapolate to
    out = {"impl": "reference", "metric": "recons/s", "value": val, "unit": "recons/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(walls),
           "extrapolated_ms_per_recon": 1e3 * statistics.mean(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOADS[wl]},
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
def headline_scene(S, workload: str):
    return S.cfg1() if workload == "cfg1" else S.cfg2().copy(precision="fp32")


def synth_scan(M, S, torch, geo, scene, seed, dev):
    """y = A x_true + D g + w at 20 dB SNR, made by the library (FP32 storage)."""
    K, Mn = scene.K, scene.M
    x_true = torch.as_tensor(S.phantom(scene, seed).reshape(-1), dtype=torch.float32, device=dev)
    y = torch.empty(K * Mn, dtype=torch.float32, device=dev)
    geo.forward(x_true, y)
    if scene.direct_arrival:
        g_true = torch.as_tensor(S.direct_gains(scene, seed), dtype=torch.float32, device=dev) * y.abs().max()
        geo.add_direct(g_true, y)
    noise = torch.as_tensor(S.unit_noise(scene, seed).reshape(-1), dtype=torch.float32, device=dev)
    sigma = math.sqrt(float((y.double() ** 2).sum()) / (100.0 * K * Mn))
    y += sigma * noise
    return x_true, y, sigma


def timed_reconstructions(torch, geo, y, sigma, n_iter, x, steps, warmup, flush, stream):
    """Device time per reconstruction (CUDA events on the launching stream), L2 flushed before each."""
    for _ in range(warmup):
        flush.fill_(1.0)
        geo.reconstruct(y, sigma, n_iter, x)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        geo.reconstruct(y, sigma, n_iter, x)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def apply_times(torch, geo, scene, dev, reps=5):
    """Median device time of single A x and A^T r calls (CUDA events, after warm-up)."""
    bf = geo.precision == "bf16"
    x = torch.ones(scene.N, dtype=torch.float32, device=dev)
    y = torch.empty(scene.K * scene.M, dtype=torch.bfloat16 if bf else torch.float32, device=dev)
    b = torch.empty(scene.N, dtype=torch.float32, device=dev)
    geo.forward(x, y)
    geo.backproject(y, b)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    tf, tb = [], []
    for _ in range(reps):
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
    return float(sorted(tf)[reps // 2]), float(sorted(tb)[reps // 2])


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

    wl = "cfg1" if args.workload == "cfg1" else "cfg2"
    scene = headline_scene(S, wl)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    geo = M.Geometry(scene, mode=args.mode)
    torch.cuda.synchronize()
    geometry_ms = 1e3 * (time.perf_counter() - t0)
    K, Mn, N = scene.K, scene.M, scene.N

    x_true, y, sigma = synth_scan(M, S, torch, geo, scene, rank, dev)
    x = torch.empty(N, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        geo.reconstruct(y, sigma, scene.n_iter, x)
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
        geo.reconstruct(y, sigma, scene.n_iter, x)
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
    x_fp32 = x.clone()
    img_err_fp32 = float((x_fp32 - x_true).norm() / x_true.norm())

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

    # roofline of the dominant apply kernel.  Tensor-core kernels (TAB mode): the record stream is the
    # algorithmic traffic - 12 B per active pair is the smallest FP32 record (delay, weight, attenuation
    # coordinate) - plus x and one A-scan array, against the measured HBM copy bandwidth.  CUDA-core kernels:
    # each tap reads the four bilinear corners of the pulse table (4 x 4 B) from shared memory and does 4 FMA;
    # shared-memory bandwidth (128 B/clk/SM) binds before the FP32 pipes (128 FMA/clk/SM) do.
    pk, src = peaks()
    pairs, taps = geo.count_taps()
    fwd_ms = kt["forward_ms"] / max(kt["forward_launches"], 1)
    bwd_ms = kt["backproject_ms"] / max(kt["backproject_launches"], 1)
    dom, dom_ms = ("forward", fwd_ms) if fwd_ms >= bwd_ms else ("backproject", bwd_ms)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = float(pk.get("sm_max_mhz", 2070.0))
    smem_peak = sm_count * SMEM_BYTES_PER_CLK * clk_mhz * 1e6 / 1e9            # GB/s
    smem_bytes = 16.0 * taps
    algo_bytes = 4.0 * (N + K * Mn)                      # x and one A-scan array in HBM
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    tc_dom = bool(geo.info.forward_tensor_cores if dom == "forward" else geo.info.adjoint_tensor_cores)
    if tc_dom:
        rec_bytes = 12.0 * pairs + algo_bytes
        name = "fwd_tcs_kernel" if dom == "forward" else "bwd_tcs_kernel"
        roofline = {"bound": "hbm", "resource": "HBM: the TAB record stream",
                    "kernel": name, "achieved": rec_bytes / (dom_ms * 1e-3) / 1e9,
                    "peak": hbm_peak, "unit": "GB/s", "frac": rec_bytes / (dom_ms * 1e-3) / 1e9 / hbm_peak,
                    "traffic": measured_traffic(name, pairs),
                    "traffic_note": "DRAM read+write bytes per launch: ncu capture of the 256x512 workload scaled "
                                    "by active pairs; null if the kernel changed since",
                    "peak_source": f"hbm_gbs ({src})", "algorithmic_bytes_per_launch": rec_bytes,
                    "bytes_per_pair_minimum": 12,
                    "bytes_per_pair_stored": geo.info.record_bytes / max(geo.info.n_records, 1), "active_pairs": pairs,
                    "taps_per_launch": taps,
                    "forward_ms": fwd_ms, "backproject_ms": bwd_ms,
                    "forward_frac": (12.0 * pairs + algo_bytes) / (fwd_ms * 1e-3) / 1e9 / hbm_peak,
                    "backproject_frac": (12.0 * pairs + algo_bytes) / (bwd_ms * 1e-3) / 1e9 / hbm_peak}
    else:
        roofline = {"bound": "alu", "resource": "shared-memory load bandwidth (pulse-table corners per tap)",
                    "kernel": dom, "achieved": smem_bytes / (dom_ms * 1e-3) / 1e9, "peak": smem_peak,
                    "unit": "GB/s", "frac": smem_bytes / (dom_ms * 1e-3) / 1e9 / smem_peak,
                    "traffic": None, "peak_source": f"{sm_count} SMs x {SMEM_BYTES_PER_CLK} B/clk x "
                                                     f"{clk_mhz:.0f} MHz (sm_max_mhz, {src})",
                    "algorithmic_bytes_per_launch": smem_bytes, "taps_per_launch": taps, "active_pairs": pairs,
                    "forward_ms": fwd_ms, "backproject_ms": bwd_ms}

    # per iteration: A^T r (tensor cores: the previous step's residual update with max |e|, the pool, the
    # fixed-point sums into b; CUDA cores: the residual update, the partial images and their reduction), the
    # prior stencil with the previous step's image update, PR+ scalars, direction, A x, projection, step; per
    # reconstruction the projection of y and the residual's sum of squares first, the last image update after
    per_iter = 3 + 6
    launches = args.steps * (per_iter * scene.n_iter + 3)

    out = {"metric": "recons/s", "value": value, "unit": "recons/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOADS[wl], "mode": geo.mode, "iterations": scene.n_iter,
                      "image": [scene.img_w, scene.img_h], "ascans": K, "samples": Mn,
                      "adjoint_groups": geo.info.adjoint_groups,
                      "tensor_core_variants": {"forward": geo.info.tc_forward_variant,
                                               "adjoint": geo.info.tc_adjoint_variant,
                                               "timed_ms": [round(t, 4) for t in geo.info.tc_variant_ms]},
                      "l2": "flushed between steps (256 MB write); device time from CUDA events per step",
                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
           "latency_ms": {"p50": statistics.median(lat), "p99": float(np.percentile(lat, 99)),
                          "wall_s": wall},
           "geometry_create_ms": geometry_ms,
           "image_rel_err_vs_phantom": img_err_fp32,
           "e2e": e2e, "roofline": roofline, "clocks": clk, "gpu_launches": launches}

    extras = world == 1 and rank == 0 and not args.no_extras
    cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    if cpu:
        xr = S.phantom(scene, 0)
        recon, desc, nth, pix, y_p = oracle_sample(scene, args.cpu_seconds, xr)
        out["cpu_baseline"] = {"value": 1.0 / recon, "unit": "recons/s", "cores": nth, "kind": "oracle",
                               "sample": desc}
        # full-size parity on the same sample: every A-scan of A x for the image restricted to P
        xm = np.zeros(N)
        xm[pix] = np.asarray(xr, np.float64).reshape(-1)[pix]
        yg = torch.empty(K * Mn, dtype=torch.float32, device=dev)
        geo.forward(torch.as_tensor(xm, dtype=torch.float32, device=dev), yg)
        d = yg.cpu().numpy().astype(np.float64).reshape(K, Mn) - y_p
        out["oracle_rel_l2_A_sampled_pixels_all_ascans"] = float(np.linalg.norm(d) / np.linalg.norm(y_p))
        del yg

    if extras:
        out["extras"] = run_extras(args, M, S, torch, np, scene, geo, y, sigma, x_true, x_fp32, flush, stream, dev)
    geo.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def run_extras(args, M, S, torch, np, scene, geo, y, sigma, x_true, x_fp32, flush, stream, dev):
    """Figures beside the headline (one GPU): the BF16 storage form of the same scan, per-apply times, the
    256 x 512 workload, the on-the-fly applies of that workload, and the served stream."""
    ex = {}
    steps = max(2, min(args.steps, 5))
    fwd, bwd = apply_times(torch, geo, scene, dev)
    ex["fp32_apply_ms"] = {"forward": fwd, "backproject": bwd}
    ex["fp32_geometry_bytes"] = geo.nbytes
    ex["fp32_record_bytes_per_pair"] = geo.info.record_bytes / max(geo.info.n_records, 1)
    geo.close()                                  # the headline's tables go before the next geometries
    torch.cuda.empty_cache()
    # BF16 storage form: same data rounded to BF16, same sigma
    t0 = time.perf_counter()
    g16 = M.Geometry(scene.copy(precision="bf16"), mode="tab")
    torch.cuda.synchronize()
    g16_ms = 1e3 * (time.perf_counter() - t0)
    ex["bf16_geometry_bytes"] = g16.nbytes
    ex["bf16_record_bytes_per_pair"] = g16.info.record_bytes / max(g16.info.n_records, 1)
    x16 = torch.empty(scene.N, dtype=torch.float32, device=dev)
    lat16 = timed_reconstructions(torch, g16, y.to(torch.bfloat16), sigma, scene.n_iter, x16, steps, 1, flush,
                                  stream)
    f16, b16 = apply_times(torch, g16, scene, dev)
    ex["bf16_storage"] = {"recons_per_s": 1e3 * len(lat16) / sum(lat16), "ms_per_step": sum(lat16) / len(lat16),
                          "steps": len(lat16), "geometry_create_ms": g16_ms,
                          "apply_ms": {"forward": f16, "backproject": b16},
                          "image_rel_diff_vs_fp32": float((x16 - x_fp32).norm() / x_fp32.norm()),
                          "image_rel_err_vs_phantom": float((x16 - x_true).norm() / x_true.norm())}
    g16.close()
    del x16
    torch.cuda.empty_cache()
    # the 256 x 512 workload, TAB (tensor cores) and OTF
    s1 = S.cfg1()
    t0 = time.perf_counter()
    g1 = M.Geometry(s1, mode="tab")
    torch.cuda.synchronize()
    g1_ms = 1e3 * (time.perf_counter() - t0)
    xt1, y1, sig1 = synth_scan(M, S, torch, g1, s1, 0, dev)
    x1 = torch.empty(s1.N, dtype=torch.float32, device=dev)
    lat1 = timed_reconstructions(torch, g1, y1, sig1, s1.n_iter, x1, max(args.steps, 5), args.warmup, flush, stream)
    f1, b1 = apply_times(torch, g1, s1, dev)
    pairs1, taps1 = g1.count_taps()
    ex["cfg1"] = {"workload": WORKLOADS["cfg1"], "recons_per_s": 1e3 * len(lat1) / sum(lat1),
                  "ms_per_step": sum(lat1) / len(lat1), "geometry_create_ms": g1_ms,
                  "apply_ms": {"forward": f1, "backproject": b1}, "active_pairs": pairs1, "taps": taps1,
                  "image_rel_err_vs_phantom": float((x1 - xt1).norm() / xt1.norm())}
    g1.close()
    go = M.Geometry(s1, mode="otf")
    fo, bo = apply_times(torch, go, s1, dev)
    ex["cfg1_otf"] = {"apply_ms": {"forward": fo, "backproject": bo},
                      "note": "travel times solved in registers on every apply (eq. 4-6); no records"}
    go.close()
    torch.cuda.empty_cache()
    if args.served_requests > 0:
        ex["served"] = served_measure(M, S, torch, np, dev, args.served_requests, (20.0, 200.0))
    return ex


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
    n = args.requests or 96
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


def served_measure(M, S, torch, np, dev, n, rates, n_geo=1):
    """Poisson arrivals mixing the three workload sizes (64x64 / 256x512 / 512x1024 at 60/30/10 %), each a
    50-iteration reconstruction, served by the engine (admission capped at 120 GB) in FP32 and in the BF16
    storage form, against a serial FIFO of FP32 mbir_reconstruct calls on the same GPU.  Each size class has
    n_geo distinct scans (geometries with their own layer thicknesses and speeds, phantoms and noise), a
    request drawing one of them, so admission sees different geometries' tables come and go.  Latency runs from a
    request's arrival to its completion seen by the host; image error against the phantom."""
    base = [S.cfg0(), S.cfg1(), S.cfg2().copy(precision="fp32")]

    def variant(c, v):
        s_ = c.copy(name=f"{c.name}_v{v}")
        for li, L in enumerate(s_.layers):            # +/- a few per cent per variant, layer by layer
            f = 1.0 + 0.02 * ((v + li) % 3 - 1) * (1 if v else 0)
            L.thickness *= f
            L.speed *= 2.0 - f
        s_.n_iter = 50
        return s_

    classes = [[variant(c, v) for v in range(n_geo)] for c in base]
    pool = {(ci, v): _synth_request(M, S, torch, classes[ci][v], 10 * ci + v, dev)
            for ci in range(3) for v in range(n_geo)}
    # the BF16 storage form of the same requests (same phantoms, noise and sigma)
    pool_bf = {(ci, v): _synth_request(M, S, torch, classes[ci][v], 10 * ci + v, dev, precision="bf16")
               for ci in range(3) for v in range(n_geo)}
    truth = {(ci, v): torch.as_tensor(S.phantom(classes[ci][v], 10 * ci + v).reshape(-1), dtype=torch.float32,
                                      device=dev) for ci in range(3) for v in range(n_geo)}
    rng = S.SplitMix64(4242)
    results = {}
    for rate in rates:
        u = rng.uniform(n)
        cls = np.where(u < 0.6, 0, np.where(u < 0.9, 1, 2))
        var = np.minimum((rng.uniform(n) * n_geo).astype(int), n_geo - 1)
        kinds = [(int(c), int(v)) for c, v in zip(cls, var)]
        gaps = -np.log(1.0 - rng.uniform(n)) / rate
        arrive = np.cumsum(gaps)
        res = {"mix": [int(np.sum(cls == c)) for c in range(3)]}
        for mode in ("engine", "engine_bf16", "serial"):
            src = pool_bf if mode == "engine_bf16" else pool
            xs = [torch.empty(classes[k[0]][k[1]].N, device=dev) for k in kinds]
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
                        tickets[nxt] = eng.submit(geo, y, sig, 50, xs[nxt])
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
                    geo.reconstruct(y, sig, 50, xs[i])
                    done[i] = time.perf_counter() - t0
            lat = np.array(done) - arrive
            torch.cuda.synchronize()
            img = float(np.mean([float((xs[i] - truth[k]).norm() / truth[k].norm()) for i, k in enumerate(kinds)]))
            res[mode] = {"recons_per_s": n / max(done), "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                         "p99_ms": 1e3 * float(np.percentile(lat, 99)), "makespan_s": float(max(done)),
                         "image_rel_err_vs_truth": img}
        results[f"{rate:g}_req_per_s"] = res
    for p_ in (pool, pool_bf):
        for geo, _, _ in p_.values():
            geo.close()
    torch.cuda.empty_cache()
    return {"workload": f"served: {n} Poisson requests per rate, sizes 64x64 / 256x512 / 512x1024 at 60/30/10 %, "
                        f"{n_geo} distinct scan(s) per size, 50 iterations each", "rates": results}


def run_served(args):
    """The served stream alone (see served_measure)."""
    import numpy as np
    import torch
    from paper_2202_09703_gb300 import build as B
    B.build()
    from paper_2202_09703_gb300 import mbir as M
    from paper_2202_09703_gb300 import synth as S
    dev = torch.device("cuda:0")
    rates = tuple(float(r) for r in args.rates.split(","))
    cfg = served_measure(M, S, torch, np, dev, args.requests or 100, rates, args.geometries)
    best = cfg["rates"][f"{rates[-1]:g}_req_per_s"]["engine_bf16"]["recons_per_s"]
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
