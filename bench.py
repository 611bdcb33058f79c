#!/usr/bin/env python
"""Benchmark of the R-FSR frame step on GB300 (one JSON line on rank 0).

Workload: the 1920x1080 recipe (8-bit luma, dynamic quarter-sampling mask, 1/f^2 background with
16 moving textured objects, integer velocities |v| <= 8 with sudden changes), K = 3 past frames,
9x9 template, search radius 8, NNC + FRMC checks, D-FSR with 4x4 blocks in a 32x32 support,
100 FSR iterations, FP32 FSR.  Synthetic, seeded inputs (no video data is available).

A step is one frame step of the whole hot path: ingest, motion estimation against 3 past frames,
consistency checks, projection, FSR and the 8-bit reconstruction.  The device-resident arm
(``value``) pushes frames already in HBM through rfsr_push_frame_device and times each step with
CUDA events on the engine's stream; L2 is flushed (a 256 MB write) between timed steps, outside
the events.  ``e2e`` times the same steps through rfsr_push_frame / rfsr_get_frame with host
buffers, host<->device copies included.

``--impl reference`` times the CPU oracle (the plain single-threaded C restatement of the
method) on the host cores: each step is the full oracle frame step on a bounded crop of the same
workload, reported in the same unit.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "HR Mpixel/s of ME+CC+projection at 1080p; p50/p99 frame latency when served"
UNIT = "HR Mpixel/s"
H, W, F = 1080, 1920, 64
T, R, KREF, ITERS = 9, 8, 3, 100
WORKLOAD = ("1920x1080 8-bit luma, dynamic quarter-sampling mask, 1/f^2 texture + 16 moving "
            "objects (|v|<=8, velocity changes every 8-24 frames), 64 frames; K=3, T=9, R=8, "
            "NNC+FRMC, D-FSR 4x4 blocks in 32x32 support, 100 iterations, FP32")

# peaks: measured HBM copy bandwidth; ALU peaks derived from unit counts and the maximum clock
SMS = 152
INT32_LANES_PER_SM = 64       # integer ALU pipe, 32-bit ops per clock per SM
FP32_LANES_PER_SM = 128       # FP32 FMA lanes per SM


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6780.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


# algorithmic work of the kernels (per frame of the workload)
def me_cost_evaluations(h=H, w=W, r=R, k=KREF):
    """Candidates v with p + v inside the frame, summed over all pixels and references."""
    cy = sum(min(y + r, h - 1) - max(y - r, 0) + 1 for y in range(h))
    cx = sum(min(x + r, w - 1) - max(x - r, 0) + 1 for x in range(w))
    return k * cy * cx


ME_OPS_PER_COST = 6        # |a-b|, mask AND, vertical and horizontal running-sum updates (2),
                           # key formation and running minimum (2)


def fsr_flops_per_block(iters=ITERS):
    N, NH = 32, 17
    dft = 2 * (N * NH * N * 2 * 2) + 2 * (N * NH * N * 4 * 2)   # row + column passes, two arrays
    per_iter = 514 * 3 + 544 * 12                                # selection + residual update
    return dft + iters * per_iter


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(",") for r in self.f.read().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "samples": len(sm), "reasons": sorted(reasons)}


def gpu_id_for(dev: int) -> str:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[dev] if vis else str(dev)


def crop_history(seq, t, y0, x0, size):
    ys, xs = slice(y0, y0 + size[0]), slice(x0, x0 + size[1])
    smp, msk = seq.samples[t][ys, xs], seq.masks[t][ys, xs]
    hist = [(seq.frames[t - k][ys, xs], seq.samples[t - k][ys, xs], seq.masks[t - k][ys, xs])
            for k in range(1, KREF + 1)]
    return smp, msk, hist


def oracle_crop_rate(seq, steps, size=(96, 96), seed=0):
    """Mpixel/s of the CPU oracle's full frame step on crops of the workload."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    tot = 0.0
    px = 0
    for i in range(steps):
        t = 3 + (i % (len(seq) - 3))
        y0 = int(rng.integers(0, H - size[0] + 1)) & ~1
        x0 = int(rng.integers(0, W - size[1] + 1)) & ~1
        smp, msk, hist = crop_history(seq, t, y0, x0, size)
        t0 = time.perf_counter()
        oracle.frame_step(smp, msk, hist, cc_mode=oracle.CC_NNC_FRMC, T=T, R=R)
        tot += time.perf_counter() - t0
        px += size[0] * size[1]
    return px / tot / 1e6, tot


def run_reference(args, rank, world):
    if rank != 0:
        return
    seq = synth.config3(F=16)
    size = (48, 48)
    oracle_crop_rate(seq, args.warmup, size, seed=1)
    rate, tot = oracle_crop_rate(seq, args.steps, size, seed=2)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(rate, 6), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * tot / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{size[0]}x{size[1]} crop per step"},
        "cpu_baseline": {"value": round(rate, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"full oracle frame step on one {size[0]}x{size[1]} crop "
                                   "of the 1080p workload per step, single thread"},
        "e2e": {"value": round(rate, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2203_09200_gb300 import build as pbuild
    from paper_2203_09200_gb300 import rfsr

    torch.cuda.set_device(local_rank)
    pbuild.build()
    seq = synth.config3(seed=3 + rank, F=F)
    HW = H * W
    d_smp = torch.from_numpy(seq.samples).cuda()
    d_msk = torch.from_numpy(seq.masks).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    eng = rfsr.Engine(device=local_rank, cuda_stream=stream.cuda_stream, profile=True)
    st = eng.create_stream(height=H, width=W, cc_mode="nnc_frmc", template_size=T,
                           search_radius=R, num_refs=KREF, fsr_iterations=ITERS)

    def step(f):
        st.push_frame_device(d_smp[f], d_msk[f])

    # warm-up: fills the 3-frame history, so every timed step uses K = 3
    nwarm = max(args.warmup, KREF)
    for i in range(nwarm):
        step(i % F)
        st.get_frame_device(timeout_ms=120000)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(gpu_id_for(local_rank)) if rank == 0 else None
    launches0 = rfsr.kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    phases = []
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()                       # evict L2 between timed steps (not timed)
        ev[i][0].record(stream)
        step((nwarm + i) % F)
        ev[i][1].record(stream)
        st.get_frame_device(timeout_ms=120000)
        phases.append(st.phase_ms())
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = rfsr.kernel_launches() - launches0
    clocks = sampler.stop() if sampler else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_s = sum(step_ms) / 1e3
    if world > 1:
        t = torch.tensor([tot_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_s = float(t.item())
        dist.barrier()
    ph = np.array(phases)                       # (steps, 4): ingest, ME, checks+PR, FSR
    ph_mean = ph.mean(axis=0)
    frames_total = args.steps * world
    value = frames_total * HW / tot_s / 1e6

    # e2e: host buffers through the public API, copies inside the timed region
    st2 = eng.create_stream(height=H, width=W, cc_mode="nnc_frmc", template_size=T,
                            search_radius=R, num_refs=KREF, fsr_iterations=ITERS)
    host_s = [np.ascontiguousarray(seq.samples[f]) for f in range(F)]
    host_m = [np.ascontiguousarray(seq.masks[f]) for f in range(F)]
    for i in range(nwarm):
        st2.push_frame(host_s[i % F], host_m[i % F])
        st2.get_frame(timeout_ms=120000)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0 = time.perf_counter()
    for i in range(args.steps):
        f = (nwarm + i) % F
        st2.push_frame(host_s[f], host_m[f])
        st2.get_frame(timeout_ms=120000)
    torch.cuda.synchronize()
    e_s = time.perf_counter() - e0
    if world > 1:
        t = torch.tensor([e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e_s = float(t.item())
    e2e = frames_total * HW / e_s / 1e6
    eng.destroy()

    if rank != 0:
        return
    hbm, mhz, src = load_peaks()
    nb = (H // 4) * (W // 4)
    me_ops = ME_OPS_PER_COST * me_cost_evaluations()
    fsr_flops = fsr_flops_per_block() * nb
    int_peak = SMS * INT32_LANES_PER_SM * mhz * 1e6
    fp32_peak = SMS * FP32_LANES_PER_SM * 2 * mhz * 1e6
    me_s, cc_s, fsr_s = ph_mean[1] / 1e3, ph_mean[2] / 1e3, ph_mean[3] / 1e3
    kern = {"me": (me_ops / me_s / 1e12, int_peak / 1e12, "Tops/s (int32)"),
            "fsr": (fsr_flops / fsr_s / 1e12, fp32_peak / 1e12, "TFLOP/s (fp32)")}
    dom = "me" if me_s >= fsr_s else "fsr"
    ach, peak, unit = kern[dom]
    roof = {"kernel": {"me": "me_kernel", "fsr": "fsr_kernel"}[dom], "bound": "alu",
            "achieved": round(ach, 3), "peak": round(peak, 3), "unit": unit,
            "frac": round(ach / peak, 4), "traffic": None,
            "peak_source": f"derived: {SMS} SMs x "
                           f"{INT32_LANES_PER_SM if dom == 'me' else FP32_LANES_PER_SM * 2} "
                           f"ops/clk x {mhz:.0f} MHz ({src} max clock)",
            "other": {k: {"achieved": round(v[0], 3), "peak": round(v[1], 3), "unit": v[2],
                          "frac": round(v[0] / v[1], 4)} for k, v in kern.items() if k != dom}}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        rate, tot = oracle_crop_rate(seq, 1, (96, 96), seed=5)
        cpu = {"value": round(rate, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"full oracle frame step (ME+CC+PR+FSR, NNC+FRMC) on one 96x96 crop of "
                         f"frame 3 of the 1080p workload with 3 past frames, {tot:.1f} s"}
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * tot_s / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "value_scope": "full frame step (ingest, ME, checks, "
                   "projection, FSR, 8-bit reconstruction) per HR pixel",
                   "l2": "flushed between timed steps (256 MB write, outside the events)",
                   "parallelism": f"replicas x{world}"},
        "breakdown": {"ingest_ms": round(ph_mean[0], 4), "me_ms": round(ph_mean[1], 4),
                      "cc_pr_ms": round(ph_mean[2], 4), "fsr_ms": round(ph_mean[3], 4),
                      "me_cc_pr_mpix_s": round(HW / ((ph_mean[0] + ph_mean[1] + ph_mean[2]) / 1e3)
                                               / 1e6, 3),
                      "wall_ms_per_step": round(1e3 * wall / args.steps, 4)},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e, 3), "unit": UNIT, "h2d_bytes_per_step": 2 * HW,
                "d2h_bytes_per_step": HW},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
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
