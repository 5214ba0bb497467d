"""Benchmark of the InfiniteDiffusion sampling path on GB300.

One step = one cold query of a 4096 x 4096 heightmap in metres through the
two-level stack (coarse UNet 64/128/128 at 1/8 resolution conditioning a fine
UNet 64/128/256/256 with bottom attention, 128-pixel windows at stride 64, 20
blended steps per level, Laplacian decode): noise, scheduler, window gather,
tensor-core UNets (TF32 by default), blend/update/re-noise and decode all run
per step.  Weights are seeded random-init (synthetic data); every step
queries a fresh location with an emptied tile cache, so nothing is reused
across steps.  Beside the headline the run measures: the end-to-end rate
into a host buffer, a second precision, the plain FP32 sampler on a cold
query of the same size, and each precision's error against the FP64
oracle's stored values of the full configuration on a 256^2 crop.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl idf|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank serves its
own queries (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

QUERY = 4096
METRIC = "final heightmap px/s, BF16/FP8+batched vs plain FP32 at stated error"
WORKLOAD = ("2-level hierarchy (coarse 64/128/128 @1/8, fine 64/128/256/256 + attention), "
            "128x128 windows stride 64, 20 steps, 4096x4096 metres query, tensor-core convs")
# FP64 oracle values of the full 20-step configuration on a 256^2 crop,
# written once by tests/golden/make_config2_crop.py (oracle only)
CROP_FIXTURE = os.path.join(ROOT, "tests", "golden", "config2_crop_k20.npz")


def bench_config(q: int, precision: str, windows_per_step=None, world: int = 1) -> dict:
    c = {"workload": WORKLOAD, "query": q, "steps_per_level": 20, "precision": precision,
         "cache": "emptied every step; working set of several GB per step exceeds L2",
         "parallelism": f"{world} independent worlds" if world > 1 else "single GPU"}
    if windows_per_step:
        c["windows_per_step"] = windows_per_step
    return c


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="idf", choices=["idf", "reference"])
    p.add_argument("--query", type=int, default=QUERY)
    p.add_argument("--precision", default="tf32", choices=["bf16", "bf16x3", "tf32", "fp32"])
    p.add_argument("--also", default="bf16", choices=["", "bf16", "bf16x3", "tf32", "fp32"],
                   help="second precision timed on the same workload beside the headline ('' = none)")
    p.add_argument("--workspace-gb", type=float, default=0.0, help="UNet workspace (0: library default)")
    p.add_argument("--cache-gb", type=float, default=0.0, help="tile cache (0: library default)")
    p.add_argument("--pairs", type=int, default=1,
                   help="1: tensor-core convolutions on CTA pairs (cta_group::2) where the shape allows")
    p.add_argument("--graphs", type=int, default=1,
                   help="1: the end-to-end leg replays repeated UNet forwards as CUDA graphs")
    p.add_argument("--autotune", type=int, default=1,
                   help="1: tensor-core tile shapes picked by the library's autotuner during the warm-up")
    p.add_argument("--student", type=int, default=0,
                   help="distillation mode: train the student on N pairs from the plain sampler, judge it")
    p.add_argument("--epochs", type=int, default=4)
    p.add_argument("--student-query", type=int, default=2048)
    p.add_argument("--student-window", type=int, default=128,
                   help="student window side (128: the 128/64 student; 32: one teacher tile per window)")
    p.add_argument("--serve", type=int, default=0,
                   help="serving mode: N random-access queries on the plain 16-channel stack, batched vs one by one")
    p.add_argument("--in-flight", type=int, default=64)
    p.add_argument("--earth", type=int, default=0,
                   help="Earth-scale mode: an N x N metres query on the 16-channel stack with a 2048^2 fBm low band")
    p.add_argument("--small-precision", default="fp8", choices=["fp32", "bf16", "fp8"],
                   help="precision of the 16-channel network in --earth and --serve (fp8 / bf16: the fused "
                        "tensor-core kernel; fp32: the plain sampler)")
    p.add_argument("--profile-unet", type=int, default=0,
                   help="profiling mode: one warm-up and one timed fine-level UNet forward on N windows")
    p.add_argument("--profile-small", type=int, default=0,
                   help="profiling mode: two forwards of the fused 16-channel UNet on N 32x32 windows "
                        "(--small-precision)")
    p.add_argument("--clocks-dir", default=tempfile.gettempdir(),
                   help="where the nvidia-smi clock samples of the timed region are written")
    p.add_argument("--ref-seconds", type=float, default=10.0,
                   help="reference arm: seconds of oracle window evaluations sampled per step")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--fp32-steps", type=int, default=1,
                   help="cold queries timed through the plain FP32 sampler (0 = skip)")
    return p.parse_args()


def dist_setup(n):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def query_origin(rank: int, i: int):
    """Origin of step i's query on a rank: distinct, far-apart 4096^2 regions
    for every (rank, step), so no rank reuses another's (or its own) tiles."""
    return (rank * 7919 + i) * (1 << 22) - (1 << 30), ((rank * 104729 + 3 * i) % 1000) * (1 << 21)


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- workload

def stack_and_weights():
    import synth
    st = synth.config2_stack()
    # the library reports its own parameter layout; weights are drawn for it
    import paper_2512_08309_gb300 as idf
    wts = [synth.weights(idf.param_shapes(lv), 0, i) for i, lv in enumerate(st["level"])]
    return st, wts


def oracle_window_counts(st, q):
    """Windows a cold metres query of a q x q region evaluates per level, by
    the oracle's own geometry: the fine cone of the decode's H rect
    (oracle.laplacian.decode_rects, oracle.kappa), and the coarse cone of
    every coarse pixel that the fine cone's conditioning or the decode's low
    band reads."""
    from oracle import kappa as OK
    from oracle import laplacian as OL
    fine, coarse = st["level"][1], st["level"][0]
    (ly0, lx0, lh, lw), (hy0, hx0, hh, hw) = OL.decode_rects(0, 0, q, q, factor=st["lap_factor"],
                                                             radius=st["lap_radius"])
    H, s, K = fine["window"], fine["stride"], fine["steps"]
    nf = sum(OK.cone_window_counts(hy0, hx0, hh, hw, H, s, K))
    y0, x0, h, w = hy0, hx0, hh, hw
    for _ in range(K):
        ri, rj = OK.kappa_1d(y0, y0 + h, H, s), OK.kappa_1d(x0, x0 + w, H, s)
        y0, x0, h, w = ri[0] * s, rj[0] * s, (ri[1] - ri[0]) * s + H, (rj[1] - rj[0]) * s + H
    f = fine["scale_to_parent"]
    cy0, cx0 = min(y0 // f, ly0), min(x0 // f, lx0)
    cy1, cx1 = max((y0 + h - 1) // f, ly0 + lh - 1), max((x0 + w - 1) // f, lx0 + lw - 1)
    nc = sum(OK.cone_window_counts(cy0, cx0, cy1 - cy0 + 1, cx1 - cx0 + 1, coarse["window"],
                                   coarse["stride"], coarse["steps"]))
    return nf, nc


# ---------------------------------------------------------------- clocks

class Clocks:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, device_index=0):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9 or parts[0] != str(device_index):
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- oracle timing

def oracle_sample(seconds=15.0):
    """Time the FP64 oracle on a bounded sample of the workload: fine and coarse
    window evaluations (Phi: UNet + preconditioning + re-noise), interleaved
    in the workload's fine:coarse ratio, until `seconds` have passed.  Returns
    (px/s estimate, description, threads)."""
    import numpy as np

    import synth
    from oracle import sampler as OS
    from oracle import unet as OU
    st = synth.config2_stack()
    wts = [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]
    nf, nc = oracle_window_counts(st, QUERY)
    world = OS.World(0, st, wts)
    fine, coarse = world.levels[1], world.levels[0]
    # coarse result the fine conditioning reads: a constant stand-in avoids
    # recursing into the coarse cone inside the timed fine evaluations
    fine.cond = lambda y0, x0, h, w: np.zeros((h, w))
    H = fine.H
    t0 = time.perf_counter()
    done_f = done_c = 0
    i = 0
    while True:
        x = [np.random.default_rng(i).standard_normal((H, H)) * 80.0]
        if done_c * nf < done_f * nc:
            coarse.phi(0, x, [(0, i * 64, H, H)])
            done_c += 1
        else:
            fine.phi(0, x, [(0, i * 64, H, H)])
            done_f += 1
        i += 1
        if time.perf_counter() - t0 > seconds and done_f >= 1:
            break
    dt = time.perf_counter() - t0
    # time per query = per-window times scaled to the cone's window counts
    est = dt * (nf / max(done_f, 1))
    if done_c:
        # split the measured time in proportion to FLOPs of the windows done
        ff = OU.flops_per_window(st["level"][1])
        fc = OU.flops_per_window(st["level"][0])
        tf = dt * done_f * ff / (done_f * ff + done_c * fc)
        tc = dt - tf
        est = tf / done_f * nf + tc / done_c * nc
    px_s = QUERY * QUERY / est
    desc = (f"FP64 NumPy oracle: {done_f} fine + {done_c} coarse 128x128 window evaluations "
            f"(preconditioned UNet + re-noise; the fine level's conditioning read replaced by "
            f"zeros) in {dt:.1f} s, extrapolated to the {nf} fine + {nc} coarse windows of one "
            f"cold {QUERY}x{QUERY} query (oracle kappa cone)")
    threads = os.cpu_count()
    return px_s, desc, threads, est


# ---------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return 0
    cores = os.cpu_count()
    vals = []
    desc = None
    for _ in range(args.warmup):
        oracle_sample(seconds=min(2.0, args.ref_seconds))   # untimed: pages in the oracle and BLAS
    t_all = time.perf_counter()
    for _ in range(args.steps):
        px, desc, threads, _ = oracle_sample(seconds=args.ref_seconds)
        vals.append(px)
    elapsed = time.perf_counter() - t_all
    v = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "px/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * QUERY * QUERY / v,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": bench_config(QUERY, args.precision),
        "cpu_baseline": {"value": v, "unit": "px/s", "cores": threads, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "px/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "ms_per_step_kind": "extrapolated: each step times a bounded sample of the query's window "
                            "evaluations and scales it to the whole cone",
        "wall_s": elapsed,
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- idf arm

def traffic_record(precision: str):
    """Per-launch DRAM traffic of the tensor-core conv from a committed ncu
    summary, valid only while the kernel source is unchanged and for the
    precision it was captured at."""
    p = os.path.join(ROOT, "profiles", "conv_tc_traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p))
    if rec.get("precision", "bf16x3") != precision:
        return None
    src = open(os.path.join(ROOT, "paper_2512_08309_gb300", "csrc", "conv_tc.cu"), "rb").read()
    if rec.get("source_sha256") != hashlib.sha256(src).hexdigest():
        return None
    return rec


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def crop_error(idf, W):
    """Error of world W against the stored FP64 oracle values of the full
    20-step configuration on its 256^2 crop: max |model - oracle| in
    sigma_out and max |metres - oracle| in metres, measured now."""
    import numpy as np
    if not os.path.exists(CROP_FIXTURE):
        return {"unavailable": "oracle fixture missing"}
    d = np.load(CROP_FIXTURE)
    x0, y0, w, h = (int(v) for v in d["crop"])
    m = W.query(x0, y0, w, h).astype(np.float64)
    v = W.query(x0, y0, w, h, kind=idf.IDF_OUT_METRES).astype(np.float64)
    em = float(np.max(np.abs(m - d["model"].astype(np.float64))))
    ev = float(np.max(np.abs(v - d["metres"].astype(np.float64))))
    return {"model_max_abs_sigma_out": em / float(d["sigma_model"]), "metres_max_abs_m": ev,
            "metres_abs_max_in_crop": float(np.max(np.abs(d["metres"]))),
            "crop": [x0, y0, w, h], "steps": int(d["steps"]),
            "against": "FP64 oracle (Eq. 1 over the crop's whole cone), tests/golden/config2_crop_k20.npz"}


def tf32_peak(dev, seconds=4.0):
    """cuBLAS TF32 GEMM (float32 8192^3 with TF32 tensor cores) back to back
    for `seconds`: the measured dense TF32 rate of this GPU, TFLOP/s."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        n = 8192
        a = torch.randn((n, n), device=dev)
        b = torch.randn((n, n), device=dev)
        c = torch.empty((n, n), device=dev)
        for _ in range(3):
            torch.matmul(a, b, out=c)
        torch.cuda.synchronize()
        burst = 0.0
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            burst = max(burst, 2.0 * n ** 3 / (e0.elapsed_time(e1) / 1000.0) / 1e12)
        it = 0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record()
        while time.perf_counter() - t0 < seconds:
            for _ in range(10):
                torch.matmul(a, b, out=c)
            it += 10
            torch.cuda.synchronize()
        e1.record()
        torch.cuda.synchronize()
        sustained = 2.0 * n ** 3 * it / (e0.elapsed_time(e1) / 1000.0) / 1e12
        del a, b, c
        return burst, sustained
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def run_idf(args, rank, world, local):
    import numpy as np
    import torch

    import paper_2512_08309_gb300 as idf
    idf.lib()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    st, wts = stack_and_weights()
    q = args.query
    W = idf.World(0, st, wts, precision=args.precision, device=local, profile=True,
                  workspace_bytes=int(args.workspace_gb * (1 << 30)), cache_bytes=int(args.cache_gb * (1 << 30)),
                  autotune=bool(args.autotune), cta_pairs=bool(args.pairs))
    out = torch.empty((q, q), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def loc(i):
        return query_origin(rank, i)

    def step(i):
        W.cache_clear()
        x0, y0 = loc(i)
        W.query_device(x0, y0, q, q, out.data_ptr(), q, kind=idf.IDF_OUT_METRES, stream=stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    s0 = W.stats()
    clocks = Clocks(os.path.join(args.clocks_dir, f"idf_clocks_rank{rank}.csv"))
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop(local)
    ms = e0.elapsed_time(e1)
    s1 = W.stats()
    ms = max_over_ranks(ms, world)
    ms_step = ms / args.steps
    value = world * q * q * args.steps / (ms / 1000.0)
    finite = bool(torch.isfinite(out).all().item())

    prof = {}
    for k in s1["profile"]:
        a, b = s0["profile"][k], s1["profile"][k]
        prof[k] = {f: b[f] - a[f] for f in ("launches", "ms", "flops", "bytes")}
    launches = s1["kernel_launches"] - s0["kernel_launches"]
    wins = [b["windows_evaluated"] - a["windows_evaluated"] for a, b in zip(s0["levels"], s1["levels"])]

    pk, pk_kind = peaks()
    tc = prof["conv_tc"]
    achieved = tc["flops"] / (tc["ms"] / 1000.0) / 1e12 if tc["ms"] > 0 else 0.0
    bf16_sus = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
    # the contraction's own dtype: TF32 is measured here (cuBLAS TF32 GEMM,
    # sustained, as conv_tc runs inside a seconds-long step); the nominal
    # ratio (1.1 / 2.25 PFLOP/s dense) x the measured bf16 peak is given beside it
    tf32_burst, tf32_sus = tf32_peak(dev) if "tf32" in (args.precision, args.also) else (None, None)
    peak = bf16_sus
    peak_kind = f"{pk_kind} bf16 sustained (MEASURED_PEAKS.json)"
    if args.precision == "tf32":
        peak = tf32_sus
        peak_kind = "measured here: cuBLAS TF32 GEMM 8192^3, sustained over 4 s"
    rec = traffic_record(args.precision)
    fpl = tc["flops"] / max(1, tc["launches"])
    # bf16x3 issues three bf16 products per multiply-add of the convolution
    mma_factor = 3.0 if args.precision == "bf16x3" else 1.0
    roofline = {"kernel": "conv_tc (tcgen05 implicit-GEMM conv)", "bound": "tensor",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_kind": peak_kind,
                "mma_work_factor": mma_factor, "achieved_mma": achieved * mma_factor,
                "frac_mma": achieved * mma_factor / peak,
                # DRAM bytes per algorithmic FLOP from the committed ncu capture of the
                # fine UNet's 23 convolutions, scaled to this run's FLOPs per launch
                "traffic": rec["dram_bytes_per_algorithmic_flop"] * fpl if rec else None,
                "algorithmic_bytes_per_launch": tc["bytes"] / max(1, tc["launches"]),
                "flops_per_launch": tc["flops"] / max(1, tc["launches"]),
                "tf32_peak_measured": {"burst": tf32_burst, "sustained": tf32_sus} if tf32_sus else None,
                "frac_vs_nominal_ratio": (achieved / (bf16_sus * 1.1 / 2.25)) if args.precision == "tf32"
                else None,
                "avg_launch_ms": tc["ms"] / max(1, tc["launches"]),
                "share_of_step": tc["ms"] / ms if ms > 0 else None}
    # per-launch roofline of the convolutions: each launch shape's attainable
    # time is max(FLOPs x MMA work factor / tensor peak, algorithmic bytes /
    # HBM peak) (the 64-channel layers at 128^2 move more bytes per FLOP
    # than the machine balance, so the HBM bounds them); the fraction is the
    # attainable time over the measured time, summed over the timed launches
    d0 = {(a, b): (n, t) for a, b, n, t in s0.get("conv_tc_shapes", [])}
    att = meas = hbm_t = 0.0
    for a, b, n, t in s1.get("conv_tc_shapes", []):
        n0, t0 = d0.get((a, b), (0, 0.0))
        if n - n0 <= 0:
            continue
        tt = a * mma_factor / (peak * 1e12)
        tb = b / (pk["hbm_gbs"] * 1e9)
        att += (n - n0) * max(tt, tb)
        hbm_t += (n - n0) * max(tt, tb) if tb > tt else 0.0
        meas += (t - t0) / 1000.0
    if meas > 0:
        roofline["per_launch"] = {
            "frac_of_attainable": att / meas, "attainable_ms": att * 1000.0, "measured_ms": meas * 1000.0,
            "hbm_bound_share_of_attainable": hbm_t / att if att > 0 else None,
            "tensor_peak_tflops": peak, "hbm_peak_gbs": pk["hbm_gbs"],
            "rule": "sum over launches of max(FLOPs x MMA factor / tensor peak, algorithmic bytes / HBM peak) "
                    "/ measured time"}
    hbm = {}
    for k in ("blend", "decode", "groupnorm", "gather"):
        p = prof[k]
        if p["ms"] > 0:
            gbs = p["bytes"] / (p["ms"] / 1000.0) / 1e9
            hbm[k] = {"achieved_gbs": gbs, "frac": gbs / pk["hbm_gbs"], "launches": p["launches"],
                      "share_of_step": p["ms"] / ms}
    # the blend draws one or two normals per pixel (Philox4x32-10 + Box-Muller,
    # bit-exact by definition): its arithmetic, not memory, bounds it, so it is
    # compared with the pure generator (idf_noise_fill over a 8192^2 region)
    if prof["blend"]["ms"] > 0 and prof["blend"]["flops"] > 0:
        nbuf = torch.empty((8192, 8192), dtype=torch.float32, device=dev)
        idf.noise_fill(1, 0, 1, 0, 0, 8192, 8192, nbuf.data_ptr(), 8192, stream=stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(3):
            idf.noise_fill(1, 0, 2 + i, 0, 0, 8192, 8192, nbuf.data_ptr(), 8192, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        gen = 3 * 8192 * 8192 / (a.elapsed_time(b) / 1000.0)
        del nbuf
        rate = prof["blend"]["flops"] / (prof["blend"]["ms"] / 1000.0)
        hbm["blend"].update({"bound": "alu (noise generation)", "normals_per_s": rate,
                             "generator_normals_per_s": gen, "frac_of_generator": rate / gen})

    line = {
        "metric": METRIC, "value": value, "unit": "px/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "tf32": "tf32"}.get(args.precision, "bf16"),
        "data": "synthetic",
        "config": bench_config(q, args.precision, {"coarse": wins[0] / args.steps, "fine": wins[1] / args.steps},
                               world),
        "gpu_launches": launches, "output_finite": finite, "autotune": s1.get("autotune"),
        "roofline": roofline, "hbm_kernels": hbm,
        "kernel_ms": {k: v["ms"] for k, v in prof.items() if v["launches"]},
        "clocks": clk,
    }

    line["error_vs_oracle"] = crop_error(idf, W) if rank == 0 else None
    W.close()

    # end to end through the public host-buffer call (D2H inside the timed
    # region), in the configuration a user runs: no per-kernel profiling, so
    # the UNet forwards repeated across batches and rounds replay as CUDA
    # graphs
    if not args.no_e2e:
        We = idf.World(0, st, wts, precision=args.precision, device=local, cuda_graphs=bool(args.graphs),
                       workspace_bytes=int(args.workspace_gb * (1 << 30)),
                       cache_bytes=int(args.cache_gb * (1 << 30)), autotune=bool(args.autotune), cta_pairs=bool(args.pairs))
        host = np.empty((q, q), dtype=np.float32)
        We.query(*loc(999), q, q, kind=idf.IDF_OUT_METRES, out=host)   # warm-up (tunes, captures)
        torch.cuda.synchronize()
        g0 = We.stats()
        barrier(world)
        t0 = time.perf_counter()
        n_e2e = max(1, args.steps)
        for i in range(n_e2e):
            We.cache_clear()
            x0, y0 = loc(1000 + i)
            We.query(x0, y0, q, q, kind=idf.IDF_OUT_METRES, out=host)
        dt = max_over_ranks(time.perf_counter() - t0, world)
        g1 = We.stats()
        We.close()
        kl = g1["kernel_launches"] - g0["kernel_launches"]
        hc = g1["graphs"]["host_launch_calls"] - g0["graphs"]["host_launch_calls"]
        line["e2e"] = {"value": world * q * q * n_e2e / dt, "unit": "px/s", "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": q * q * 4, "steps": n_e2e, "warmup": 1,
                       "cuda_graphs": bool(args.graphs),
                       "kernels_per_step": kl / n_e2e, "host_launch_calls_per_step": hc / n_e2e,
                       "graph_replays_per_step": (g1["graphs"]["replays"] - g0["graphs"]["replays"]) / n_e2e}

    # a second precision (by default the compensated three-product bf16
    # path) on the same workload, timed the same way, beside the headline
    if args.also and args.also != args.precision:
        W2 = idf.World(0, st, wts, precision=args.also, device=local, profile=True,
                       workspace_bytes=int(args.workspace_gb * (1 << 30)),
                       cache_bytes=int(args.cache_gb * (1 << 30)), autotune=bool(args.autotune), cta_pairs=bool(args.pairs))

        def step2(i):
            W2.cache_clear()
            x0, y0 = loc(2000 + i)
            W2.query_device(x0, y0, q, q, out.data_ptr(), q, kind=idf.IDF_OUT_METRES, stream=stream)

        # the second precision is context beside the headline: at most 3
        # warm-up and 5 timed steps
        w2n, k2n = min(args.warmup, 3), min(args.steps, 5)
        for i in range(w2n):
            step2(i)
        torch.cuda.synchronize()
        t0 = W2.stats()
        barrier(world)
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(k2n):
            step2(w2n + i)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms2 = max_over_ranks(e0.elapsed_time(e1), world)
        t1 = W2.stats()
        err2 = crop_error(idf, W2) if rank == 0 else None
        W2.close()
        c0, c1 = t0["profile"]["conv_tc"], t1["profile"]["conv_tc"]
        tc_ms = c1["ms"] - c0["ms"]
        ach = (c1["flops"] - c0["flops"]) / (tc_ms / 1000.0) / 1e12 if tc_ms > 0 else 0.0
        pk2 = tf32_sus if args.also == "tf32" else bf16_sus
        mf2 = 3.0 if args.also == "bf16x3" else 1.0
        line["also"] = {args.also: {
            "value": world * q * q * k2n / (ms2 / 1000.0), "unit": "px/s", "ms_per_step": ms2 / k2n,
            "steps": k2n, "warmup": w2n, "error_vs_oracle": err2,
            "conv_tc_achieved_tflops": ach, "conv_tc_frac": ach / pk2, "mma_work_factor": mf2,
            "conv_tc_frac_mma": ach * mf2 / pk2, "conv_tc_share_of_step": tc_ms / ms2 if ms2 > 0 else None}}

    # the plain FP32 sampler (float32 SIMT convolutions, same algorithm, one
    # query at a time): one cold q x q metres query at a fresh location,
    # timed the same way, after a small warm-up query
    if args.fp32_steps > 0 and rank == 0:
        Wp = idf.World(0, st, wts, precision="fp32", device=local,
                       workspace_bytes=int(args.workspace_gb * (1 << 30)),
                       cache_bytes=int(args.cache_gb * (1 << 30)))
        wq = torch.empty((256, 256), dtype=torch.float32, device=dev)
        Wp.query_device(*loc(3000), 256, 256, wq.data_ptr(), 256, kind=idf.IDF_OUT_METRES, stream=stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(args.fp32_steps):
            Wp.cache_clear()
            x0, y0 = loc(3001 + i)
            Wp.query_device(x0, y0, q, q, out.data_ptr(), q, kind=idf.IDF_OUT_METRES, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        msp = e0.elapsed_time(e1)
        Wp.close()
        fp32_pxs = q * q * args.fp32_steps / (msp / 1000.0)
        line["plain_fp32"] = {"value": fp32_pxs, "unit": "px/s", "ms_per_step": msp / args.fp32_steps,
                              "steps": args.fp32_steps,
                              "method": "measured: cold metres query of the same size at a fresh location "
                                        "through an IDF_FP32 world (float32 SIMT convolutions)",
                              f"speedup_{args.precision}": value / fp32_pxs}
        if "also" in line:
            line["plain_fp32"][f"speedup_{args.also}"] = line["also"][args.also]["value"] / fp32_pxs
    if not args.no_cpu and rank == 0 and world == 1:
        px, desc, threads, est = oracle_sample(seconds=15.0)
        line["cpu_baseline"] = {"value": px, "unit": "px/s", "cores": threads, "kind": "oracle",
                                "sample": desc}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_profile_unet(args):
    """Small-footprint profiling case: the fine UNet of the 2-level stack on
    N 128x128 windows (about 80 kernel launches per forward)."""
    import torch

    import paper_2512_08309_gb300 as idf
    st, wts = stack_and_weights()
    n = args.profile_unet
    W = idf.World(0, st, wts, precision=args.precision, max_batch=n, cache_bytes=64 << 20, profile=True,
                  cta_pairs=bool(args.pairs))
    x = torch.randn((n, 2, 128, 128), device="cuda")
    y = torch.empty((n, 1, 128, 128), device="cuda")
    W.unet_forward(1, x.data_ptr(), n, y.data_ptr())
    torch.cuda.synchronize()
    s0 = W.stats()
    W.unet_forward(1, x.data_ptr(), n, y.data_ptr())
    torch.cuda.synchronize()
    s1 = W.stats()
    prof = {k: {f: s1["profile"][k][f] - s0["profile"][k][f] for f in ("launches", "ms", "flops")}
            for k in s1["profile"] if s1["profile"][k]["launches"] - s0["profile"][k]["launches"]}
    print(json.dumps({"profile_unet": n, "precision": args.precision, "cta_pairs": bool(args.pairs), "kernels": prof,
                      "finite": bool(torch.isfinite(y).all().item()), "device_status": s1["device_status"],
                      "cta_pair_clusters": s1.get("cta_pair_clusters")}))
    W.close()
    return 0


def run_profile_small(args):
    """Small-footprint profiling case of the fused 16-channel kernel: the
    single-level network on N 32x32 windows, two forwards (one launch each),
    timed with CUDA events."""
    import torch

    import paper_2512_08309_gb300 as idf
    import synth
    st = synth.config1_stack()
    wts = [synth.weights(idf.param_shapes(lv), 0, i) for i, lv in enumerate(st["level"])]
    n = args.profile_small
    W = idf.World(0, st, wts, precision=args.small_precision, max_batch=n, cache_bytes=64 << 20)
    x = torch.randn((n, 1, 32, 32), device="cuda")
    y = torch.empty((n, 1, 32, 32), device="cuda")
    W.unet_forward(0, x.data_ptr(), n, y.data_ptr())
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    W.unet_forward(0, x.data_ptr(), n, y.data_ptr())
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    print(json.dumps({"profile_small": n, "precision": args.small_precision, "ms": ms,
                      "windows_per_s": n / (ms / 1000.0), "finite": bool(torch.isfinite(y).all().item()),
                      "device_status": W.stats()["device_status"]}))
    W.close()
    return 0


def run_student(args):
    """Distil a one-evaluation student from a deterministic teacher.

    Teacher: the plain 16-channel sampler (4 steps, float32) with windows at
    stride = window (independent 32x32 tiles, T = 1, Sec. 6's baseline
    layout), so that each tile's result is a function of its own four noise
    fields N(seed, 0, j, .), j = 0..3, and nothing else.  Pairs: 128x128
    crops of the teacher's output (targets) and the four fields over the crop
    (inputs: sigma_0 N_0 as the noisy state, N_1..N_3 as side channels of
    the student, the re-noise the teacher consumes).  Loss: D(x; 80) vs t,
    AdamW lr 2e-4, batch 64.  Judge: on held-out windows, the rms and max of
    |D - teacher| in sigma_out; a window falls back to the teacher when its
    rms exceeds 5e-2 sigma_out.  Speed: the student's network on the tensor
    cores (TF32, one evaluation per 128x128 window, fed by noise_fill)
    against the teacher on the same query."""
    import numpy as np
    import torch

    import paper_2512_08309_gb300 as idf
    import synth
    dev = torch.device("cuda", 0)
    n_pairs, H = args.student, args.student_window
    c1 = synth.config1_stack()
    tlv = dict(c1["level"][0], stride=int(c1["level"][0]["window"]))
    tst = synth.stack([tlv])
    tw = [synth.weights(idf.param_shapes(tlv), 0, 0)]
    teacher = idf.World(0, tst, tw, precision="fp32")
    sig0 = float(tlv["sigma_max"])
    side, per = 1024, (1024 // H) ** 2
    n_q = (n_pairs + per - 1) // per
    t_gen = time.perf_counter()
    T = torch.empty((n_q * per, H, H), device=dev)
    X = torch.empty((n_q * per, 4, H, H), device=dev)
    big = torch.empty((side, side), device=dev)
    nb = torch.empty((4, side, side), device=dev)
    for q in range(n_q):
        x0, y0 = (q * 7 + 1) * (1 << 20), (q * 13 + 5) * (1 << 19)
        teacher.query_device(x0, y0, side, side, big.data_ptr(), side)
        for j in range(4):
            idf.noise_fill(0, 0, j, x0, y0, side, side, nb[j].data_ptr(), side)
        torch.cuda.synchronize()
        nb[0] *= sig0
        k = side // H
        T[q * per:(q + 1) * per] = big.reshape(k, H, k, H).permute(0, 2, 1, 3).reshape(per, H, H)
        X[q * per:(q + 1) * per] = nb.reshape(4, k, H, k, H).permute(1, 3, 0, 2, 4).reshape(per, 4, H, H)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    T, X = T[:n_pairs], X[:n_pairs]
    n_hold = max(64, n_pairs // 16)
    n_train = n_pairs - n_hold
    sig_out = float(T[n_train:].std())
    lv = dict(synth.student_level(window=H, stride=H // 2), in_ch=4)
    w0 = synth.weights(idf.param_shapes(lv), 0, 0)
    bs = 64
    S = idf.Student(lv, w0, max_batch=bs)

    def held_out_loss():
        tot, cnt = 0.0, 0
        for i in range(n_train, n_pairs, bs):
            j = min(n_pairs, i + bs)
            tot += S.loss_grad(X[i:j].contiguous().data_ptr(), T[i:j].contiguous().data_ptr(), j - i, sig0) * (j - i)
            cnt += j - i
        S.zero_grad()
        return tot / cnt

    loss_before = held_out_loss()
    g = torch.Generator(device="cpu").manual_seed(0)
    t_train = time.perf_counter()
    steps = 0
    curve = []
    for ep in range(args.epochs):
        perm = torch.randperm(n_train, generator=g).to(dev)
        ep_loss = 0.0
        for i in range(0, n_train - bs + 1, bs):
            idx = perm[i:i + bs]
            xb, tb = X[idx].contiguous(), T[idx].contiguous()
            ep_loss += S.loss_grad(xb.data_ptr(), tb.data_ptr(), bs, sig0)
            S.adamw(lr=2e-4, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.01)
            steps += 1
        curve.append(ep_loss / max(1, n_train // bs))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t_train
    loss_after = held_out_loss()
    w_trained = S.weights()
    S.close()

    # the student as a network of the library (TF32 tensor cores): F on the
    # preconditioned input, D = c_skip x_0 + c_out F
    sd = float(lv["sigma_data"])
    c_skip, c_out, c_in = sd * sd / (sig0 ** 2 + sd * sd), sig0 * sd / math.sqrt(sig0 ** 2 + sd * sd), \
        1.0 / math.sqrt(sig0 ** 2 + sd * sd)
    sst = synth.stack([dict(lv, stride=H, steps=1)])
    Ws = idf.World(0, sst, [w_trained], precision="tf32", max_batch=256)
    fb = torch.empty((256, 1, H, H), device=dev)

    def student_d(xin):
        n = xin.shape[0]
        xp = xin.clone()
        xp[:, 0] *= c_in
        out = torch.empty((n, H, H), device=dev)
        for i in range(0, n, 256):
            j = min(n, i + 256)
            Ws.unet_forward(0, xp[i:j].contiguous().data_ptr(), j - i, fb.data_ptr())
            out[i:j] = c_skip * xin[i:j, 0] + c_out * fb[:j - i, 0]
        return out

    D = student_d(X[n_train:])
    torch.cuda.synchronize()
    err = (D - T[n_train:]).abs()
    rms = ((D - T[n_train:]) ** 2).mean(dim=(1, 2)).sqrt() / sig_out
    mx = err.amax(dim=(1, 2)) / sig_out
    judged = {"windows": int(rms.numel()), "rms_median_sigma_out": float(rms.median()),
              "rms_max_sigma_out": float(rms.max()), "max_median_sigma_out": float(mx.median()),
              "fallback_rate_rms_5e-2": float((rms > 5e-2).float().mean()),
              "fallback_rate_max_5e-2": float((mx > 5e-2).float().mean()),
              "rms_overall_sigma_out": float(((D - T[n_train:]) ** 2).mean().sqrt()) / sig_out}
    # untrained student on the same windows (the gain of training)
    Wu = idf.World(0, sst, [w0], precision="tf32", max_batch=256)
    Ws, Wkeep = Wu, Ws
    Du = student_d(X[n_train:])
    Ws = Wkeep
    rms_u = ((Du - T[n_train:]) ** 2).mean(dim=(1, 2)).sqrt() / sig_out
    judged["untrained_rms_median_sigma_out"] = float(rms_u.median())
    Wu.close()

    # speed on a q x q query: the teacher (plain FP32 sampler, independent
    # tiles) against the student's network on the same region's noise fields
    q = args.student_query
    qx, qy = 3 << 24, 5 << 24
    ref = torch.empty((q, q), device=dev)
    teacher.query_device(qx - (1 << 22), qy, 256, 256, ref.data_ptr(), 256)   # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    teacher.query_device(qx, qy, q, q, ref.data_ptr(), q)
    e1.record()
    torch.cuda.synchronize()
    teacher_pxs = q * q / (e0.elapsed_time(e1) / 1000.0)
    teacher.close()
    k = q // H
    fields = torch.empty((4, q, q), device=dev)
    e0.record()
    for j in range(4):
        idf.noise_fill(0, 0, j, qx, qy, q, q, fields[j].data_ptr(), q)
    fields[0] *= sig0
    xin = fields.reshape(4, k, H, k, H).permute(1, 3, 0, 2, 4).reshape(k * k, 4, H, H)
    Dq = student_d(xin)
    e1.record()
    torch.cuda.synchronize()
    student_pxs = q * q / (e0.elapsed_time(e1) / 1000.0)
    Tq = ref.reshape(k, H, k, H).permute(0, 2, 1, 3).reshape(k * k, H, H)
    rq = ((Dq - Tq) ** 2).mean(dim=(1, 2)).sqrt() / sig_out
    Ws.close()
    print(json.dumps({
        "student": {"pairs": n_pairs, "train_pairs": n_train, "held_out": n_hold, "epochs": args.epochs,
                    "steps": steps, "batch": bs, "pair_gen_s": t_gen, "train_s": t_train,
                    "train_loss_per_epoch": curve, "held_out_loss_before": loss_before,
                    "held_out_loss_after": loss_after, "gain_held_out_loss": loss_before / loss_after},
        "teacher": "plain 16-channel sampler, 4 steps, float32, windows at stride = window (independent 32x32 tiles)",
        "sigma_out_teacher": sig_out, "judged_held_out": judged,
        "query": {"side": q, "teacher_px_s": teacher_pxs, "student_px_s": student_pxs,
                  "fallback_rate_rms_5e-2": float((rq > 5e-2).float().mean()),
                  "rms_median_sigma_out": float(rq.median())}}))
    return 0


def run_serve(args):
    """Batched lazy random access: the seeded query workload (sides log-uniform
    in [64, 2048], centres uniform in +-1e6, 30% overlapping an earlier query)
    on the plain 16-channel stack, served closed-loop in groups of at most
    `in_flight` queries through idf_world_query_batch (all windows of a step
    across the group share launches), and the same queries one by one."""
    import numpy as np
    import torch

    import paper_2512_08309_gb300 as idf
    import synth
    dev = torch.device("cuda", 0)
    qs = synth.random_queries(args.serve, seed=0)
    st = synth.config1_stack()
    wts = [synth.weights(idf.param_shapes(lv), 0, i) for i, lv in enumerate(st["level"])]
    maxpx = max(w * h for _, _, w, h in qs)
    bufs = [torch.empty(maxpx, device=dev) for _ in range(args.in_flight)]
    out = {}
    modes = [("batched", args.small_precision), ("single", args.small_precision), ("single_fp32", "fp32")]
    for mode, prec in modes:
        W = idf.World(0, st, wts, precision=prec)
        # warm-up on an unrelated region
        W.query_device(5 << 30, 5 << 30, 256, 256, bufs[0].data_ptr(), 256)
        torch.cuda.synchronize()
        W.cache_clear()
        s0 = W.stats()
        lat = []
        t_all = time.perf_counter()
        if mode == "batched":
            for g0 in range(0, len(qs), args.in_flight):
                grp = qs[g0:g0 + args.in_flight]
                t0 = time.perf_counter()
                W.query_batch([(x0, y0, w, h, bufs[i].data_ptr(), w) for i, (x0, y0, w, h) in enumerate(grp)])
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                lat += [dt] * len(grp)
        else:
            for (x0, y0, w, h) in qs:
                t0 = time.perf_counter()
                W.query_device(x0, y0, w, h, bufs[0].data_ptr(), w)
                torch.cuda.synchronize()
                lat.append(time.perf_counter() - t0)
        total = time.perf_counter() - t_all
        s1 = W.stats()
        W.close()
        px = sum(w * h for _, _, w, h in qs)
        l0, l1 = s0["levels"][0], s1["levels"][0]
        hits, miss = l1["cache_hits"] - l0["cache_hits"], l1["cache_misses"] - l0["cache_misses"]
        out[mode] = {"precision": prec, "px_s": px / total, "total_s": total,
                     "p50_ms": 1000 * float(np.percentile(lat, 50)),
                     "p99_ms": 1000 * float(np.percentile(lat, 99)),
                     "windows": l1["windows_evaluated"] - l0["windows_evaluated"],
                     "cache_hit_rate": hits / max(1, hits + miss),
                     "launches": s1["kernel_launches"] - s0["kernel_launches"]}
    out["speedup_batched_vs_plain_fp32_single"] = out["batched"]["px_s"] / out["single_fp32"]["px_s"]
    print(json.dumps({"serve": {"queries": len(qs), "px": sum(w * h for _, _, w, h in qs), "in_flight": args.in_flight,
                                "stack": "16-channel UNet, 32x32 windows at stride 16, 4 steps",
                                "latency": "per query: submission of its group to completion",
                                **out}}))
    return 0


def run_earth(args):
    """The 16-channel 32x32-window UNet generating the residual band under a
    periodic fBm low band (2048^2 low-resolution px, beta 2.2, signed square
    roots of [-11000, 9000] m): cold N x N metres queries, float32 network
    (its 16 channels are below the tensor-core tile width), with the error
    in metres against the FP64 oracle on a 64 x 48 crop that crosses the
    fixture's period."""
    import numpy as np
    import torch

    import paper_2512_08309_gb300 as idf
    import synth
    from oracle import sampler as OS
    from oracle import unet as OU
    idf.lib()
    dev = torch.device("cuda", 0)
    fx = synth.fbm_lowband(2048, beta=2.2, seed=0)
    st = synth.config4_stack(fx, steps=4)
    wts = [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]
    q = args.earth
    prec = args.small_precision
    W = idf.World(0, st, wts, precision=prec, profile=True)
    out = torch.empty((q, q), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(i):
        W.cache_clear()
        W.query_device(-q // 2 + 65536 * i, -q // 2, q, q, out.data_ptr(), q, kind=idf.IDF_OUT_METRES,
                       stream=stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    s0 = W.stats()
    clocks = Clocks(os.path.join(args.clocks_dir, "idf_clocks_earth.csv"))
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop(0)
    ms = e0.elapsed_time(e1)
    s1 = W.stats()
    m = out.cpu().numpy()
    # errors against the FP64 oracle on four crops (centre, two corners of
    # the timed query's first location, and one across the fixture's period)
    ow = OS.World(0, st, wts)
    errs = []
    for (cx, cy) in ((-32, -32), (-q // 2, -q // 2), (q // 2 - 64, -q // 2), (16384 - 32, 100)):
        crop = (cx, cy, 64, 64)
        got = W.query(*crop, kind=idf.IDF_OUT_METRES).astype(np.float64)
        gm = W.query(*crop).astype(np.float64)
        ref = ow.metres(crop[1], crop[0], crop[3], crop[2])
        rm = ow.model(crop[1], crop[0], crop[3], crop[2])
        errs.append({"crop": list(crop), "max_abs_m": float(np.max(np.abs(got - ref))),
                     "max_abs_metres_in_crop": float(np.max(np.abs(ref))),
                     "model_max_abs_sigma_out": float(np.max(np.abs(gm - rm)) / rm.std())})
    W.close()
    # the plain FP32 sampler on the same query size, one cold query
    fp32 = None
    if prec != "fp32" and args.fp32_steps > 0:
        Wp = idf.World(0, st, wts, precision="fp32")
        Wp.query_device(-q // 2 + 65536 * 99, -q // 2, 256, 256, out.data_ptr(), 256, kind=idf.IDF_OUT_METRES,
                        stream=stream)
        torch.cuda.synchronize()
        e0.record(stream)
        Wp.query_device(-q // 2 + 65536 * 100, -q // 2, q, q, out.data_ptr(), q, kind=idf.IDF_OUT_METRES,
                        stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        Wp.close()
        fp32 = q * q / (e0.elapsed_time(e1) / 1000.0)
    prof = {k: s1["profile"][k]["ms"] - s0["profile"][k]["ms"] for k in s1["profile"]}
    line = {"metric": "final heightmap px/s (metres, Earth-scale low band)", "value": q * q * args.steps / (ms / 1000.0),
            "unit": "px/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "dtype": {"fp8": "e4m3", "bf16": "bf16"}.get(prec, "f32"),
            "data": "synthetic",
            "config": {"workload": f"16-channel 32x32-window UNet (4 steps) residual band + 2048^2 fBm low band "
                                   f"(beta 2.2, period 16384 px), {q}x{q} metres query",
                       "precision": prec},
            "metres_range": [float(m.min()), float(m.max())],
            "error_vs_oracle": errs,
            "plain_fp32": {"value": fp32, "unit": "px/s", "speedup": (q * q * args.steps / (ms / 1000.0)) / fp32}
            if fp32 else None,
            "kernel_ms": {k: v for k, v in prof.items() if v > 0}, "clocks": clk}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.serve:
        return run_serve(args)
    if args.earth:
        return run_earth(args)
    if args.student:
        return run_student(args)
    if args.profile_unet:
        return run_profile_unet(args)
    if args.profile_small:
        return run_profile_small(args)
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
    else:
        rc = run_idf(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
