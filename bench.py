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


# Algorithmic work of the metric's path, counted as the method states it: a template cost
# C(p, v) is a sum of |s_t - rec| over the measured pixels of the T x T template (Sec. 2.2), so one
# cost evaluation is n(p) masked byte absolute differences, n(p) the measured pixels in the
# template around p (about T^2 / 4 under quarter sampling).  ME evaluates every candidate v with
# p + v inside the frame; FRMC evaluates the 49 reverse costs C(p + d, v - d) with p + d inside
# for every pixel it checks (Sec. 3.1.1), whatever the outcome.
FRMC_OFFSETS = (-7, -3, -1, 0, 1, 3, 7)


def template_counts(msk, t=T):
    """n(p): measured pixels of the t x t template around every pixel (0 outside the frame)."""
    h = t // 2
    m = np.pad(np.asarray(msk, np.int64) != 0, h).astype(np.int64)
    c = np.pad(m.cumsum(0).cumsum(1), ((1, 0), (1, 0)))
    Hh, Ww = np.asarray(msk).shape
    return c[t:t + Hh, t:t + Ww] - c[:Hh, t:t + Ww] - c[t:t + Hh, :Ww] + c[:Hh, :Ww]


def me_byteops(msk, t=T, r=R):
    """Masked byte |a-b| of forward ME against one past frame: sum over p of n(p) |V(p)|."""
    n = template_counts(msk, t)
    Hh, Ww = n.shape
    cy = np.array([min(y + r, Hh - 1) - max(y - r, 0) + 1 for y in range(Hh)], np.int64)
    cx = np.array([min(x + r, Ww - 1) - max(x - r, 0) + 1 for x in range(Ww)], np.int64)
    return int((n * cy[:, None] * cx[None, :]).sum())


def me_cost_evaluations(h, w, r=R):
    """Template costs forward ME evaluates against one past frame: the (p, v) pairs with v in
    [-R, R]^2 and p + v inside the frame."""
    cy = np.array([min(y + r, h - 1) - max(y - r, 0) + 1 for y in range(h)], np.int64)
    cx = np.array([min(x + r, w - 1) - max(x - r, 0) + 1 for x in range(w)], np.int64)
    return int(cy.sum() * cx.sum())


def frmc_source_work(msk, t=T):
    """S(p) = sum over the FRMC offsets d with p + d inside of n(p + d): the masked byte |a-b| of
    one pixel's FRMC check."""
    n = template_counts(msk, t)
    Hh, Ww = n.shape
    pad = np.pad(n, 7)
    S = np.zeros_like(n)
    for dy in FRMC_OFFSETS:
        for dx in FRMC_OFFSETS:
            S += pad[7 + dy:7 + dy + Hh, 7 + dx:7 + dx + Ww]
    return S


def fsr_flops_per_block(iters=ITERS):
    N, NH = 32, 17
    dft = 2 * (N * NH * N * 2 * 2) + 2 * (N * NH * N * 4 * 2)   # row + column passes, two arrays
    per_iter = 514 * 3 + 544 * 12                                # selection + residual update
    return dft + iters * per_iter


# committed ncu summaries: DRAM bytes per launch of a kernel, valid while its sources are unchanged
CSRC = os.path.join(ROOT, "paper_2203_09200_gb300", "csrc")
KERNEL_PROFILES = {"fsr_kernel": ("fsr_kernel_1080p.md", ["fsr.cu", "rfsr_internal.h"]),
                   "me9_kernel": ("me9_kernel_1080p.md", ["me.cu", "me9_tile.cuh", "rfsr_internal.h"]),
                   "cc_project_kernel": ("cc_project_kernel_1080p.md", ["cc.cu", "rfsr_internal.h"]),
                   "rme9_kernel": ("rme9_kernel_1080p.md", ["me.cu", "me9_tile.cuh", "rfsr_internal.h"])}


def kernel_source_sha(kernel):
    """Hash of the kernel's source code without comments and whitespace (an edit to a comment
    does not change the kernel the counters were taken on)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in KERNEL_PROFILES[kernel][1]:
        src = open(os.path.join(CSRC, f), encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(re.sub(r"\s+", "", src).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel):
    """dram__bytes_read.sum + dram__bytes_write.sum of one launch from the kernel's ncu summary in
    profiles/, or None when there is none or it was taken on other kernel sources."""
    import re
    path = os.path.join(ROOT, "profiles", KERNEL_PROFILES[kernel][0])
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    sha = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    tb = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", txt)
    if not sha or not tb or sha.group(1) != kernel_source_sha(kernel):
        return None
    return int(tb.group(1))


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def wait_first(self, timeout_s: float = 5.0):
        """Block until nvidia-smi has written its first sample (or timeout_s passed), so that
        the samples cover the timed region from its start."""
        t0 = time.perf_counter()
        while self.p is not None and time.perf_counter() - t0 < timeout_s:
            if os.path.getsize(self.f.name) > 0 or self.p.poll() is not None:
                return
            time.sleep(0.02)

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


def oracle_crop_rate(seq, steps, size=(96, 96), seed=0, threads=1):
    """CPU oracle on crops of the workload: (ME+CC+PR Mpixel/s, full-step Mpixel/s, seconds).
    Each crop runs the oracle's frame step without FSR (the metric's scope) and then in full;
    threads > 1 uses the oracle's OpenMP build (same results)."""
    import oracle
    oracle.build(omp=threads > 1)
    oracle.set_threads(threads)
    try:
        return _oracle_crops(oracle, seq, steps, size, seed)
    finally:
        oracle.set_threads(1)


def _oracle_crops(oracle, seq, steps, size, seed):
    rng = np.random.default_rng(seed)
    t_mecc = t_full = 0.0
    px = 0
    for i in range(steps):
        t = 3 + (i % (len(seq) - 3))
        y0 = int(rng.integers(0, H - size[0] + 1)) & ~1
        x0 = int(rng.integers(0, W - size[1] + 1)) & ~1
        smp, msk, hist = crop_history(seq, t, y0, x0, size)
        t0 = time.perf_counter()
        oracle.frame_step(smp, msk, hist, cc_mode=oracle.CC_NNC_FRMC, T=T, R=R, run_fsr=False)
        t1 = time.perf_counter()
        oracle.frame_step(smp, msk, hist, cc_mode=oracle.CC_NNC_FRMC, T=T, R=R)
        t2 = time.perf_counter()
        t_mecc += t1 - t0
        t_full += t2 - t1
        px += size[0] * size[1]
    return px / t_mecc / 1e6, px / t_full / 1e6, t_mecc + t_full


def run_reference(args, rank, world):
    if rank != 0:
        return
    seq = synth.config3(F=16)
    size = (48, 48)
    oracle_crop_rate(seq, args.warmup, size, seed=1)
    rate, full, tot = oracle_crop_rate(seq, args.steps, size, seed=2)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(rate, 6), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * tot / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{size[0]}x{size[1]} crop per step",
                   "value_scope": "oracle ME + checks + projection (frame step without FSR)"},
        "full_step": {"value": round(full, 6), "unit": UNIT},
        "cpu_baseline": {"value": round(rate, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"oracle frame step on one {size[0]}x{size[1]} crop of the "
                                   "1080p workload per step (3 past frames), single thread: "
                                   "without FSR (value), then with FSR (full_step)"},
        "e2e": {"value": round(rate, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


SIZES4 = [(240, 320), (480, 640), (720, 1280), (1080, 1920)]
SIZES5 = [(240, 320), (480, 640), (720, 1280), (1080, 1920), (1440, 2560), (2160, 3840)]


def crop_streams(base: "synth.VideoSequence", specs, frames):
    """Per stream: crops of a shared content sequence at a seeded offset, with the stream's own
    fixed or dynamic quarter-sampling mask (the content recipe of the source sequence)."""
    out = []
    Hb, Wb = base.shape
    for i, sp in enumerate(specs):
        rng = np.random.default_rng(sp.seed)
        y0 = int(rng.integers(0, Hb - sp.H + 1)) & ~1
        x0 = int(rng.integers(0, Wb - sp.W + 1)) & ~1
        t0 = int(rng.integers(0, len(base)))
        if sp.mask_type == synth.MASK_FIXED:
            m = synth.positions_to_mask(synth.fixed_positions(sp.H, sp.W, rng))
            masks = [m]
        else:
            perm = synth.dynamic_permutations(sp.H, sp.W, rng)
            masks = [synth.positions_to_mask(synth.dynamic_positions(perm, t)) for t in range(4)]
        fr = [base.frames[(t0 + t) % len(base), y0:y0 + sp.H, x0:x0 + sp.W] for t in range(frames)]
        smp = [np.ascontiguousarray(fr[t] * masks[t % len(masks)]) for t in range(frames)]
        msk = [masks[t % len(masks)] for t in range(frames)]
        out.append((sp, smp, msk))
    return out


def small_streams(n_streams=256, frames=16, seed=6):
    """n streams of 320x240 (the smallest size of the 64-stream mix), half fixed / half dynamic."""
    rng = np.random.default_rng(seed)
    return [synth.StreamSpec(240, 320, synth.MASK_FIXED if i < n_streams // 2 else synth.MASK_DYNAMIC,
                             frames, int(rng.integers(0, 2 ** 31 - 1))) for i in range(n_streams)]


def run_batching(rfsr, torch, specs=None, frames=16, what=None):
    """Many streams: one batched step per round against a per-stream launch loop (both with
    device-resident inputs, the same frames, bit-identical outputs).  The batched engine's
    autotuner settles on a calibration pass over the same streams first; the timed pass then
    runs with the shape it chose (new streams, same engine)."""
    if specs is None:
        specs = synth.config4_streams(n_streams=64, frames=frames)
        what = ("64 streams, sizes from 320x240/640x480/1280x720/1920x1080, half fixed / half "
                "dynamic masks")
    n_streams = len(specs)
    base = synth.config2(seed=44, H=1080, W=1920, F=frames)
    streams = crop_streams(base, specs, frames)
    d_in = [[(torch.from_numpy(s).cuda(), torch.from_numpy(m).cuda()) for s, m in zip(smp, msk)]
            for _, smp, msk in streams]
    pix = sum(sp.H * sp.W for sp, _, _ in streams)
    res = {}

    def rounds(eng, cs, batched):
        sts = [eng.create_stream(height=sp.H, width=sp.W, mask_type=sp.mask_type)
               for sp, _, _ in streams]
        ev = []
        for t in range(frames):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(cs)
            for i, st in enumerate(sts):
                st.push_frame_device(*d_in[i][t])
            if batched:
                eng.step()
            e1.record(cs)
            for st in sts:
                st.get_frame_device(timeout_ms=120000)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        for st in sts:
            st.destroy()
        return [a.elapsed_time(b) for a, b in ev[3:]]            # rounds with 3 past frames

    for mode in ("loop", "batched"):
        cs = torch.cuda.Stream()
        eng = rfsr.Engine(device=torch.cuda.current_device(), cuda_stream=cs.cuda_stream,
                          batched=(mode == "batched"), max_inflight=2)
        if mode == "batched":
            rounds(eng, cs, True)                                # autotuner calibration pass
            res["autotune"] = eng.tuning()
        launches0 = rfsr.kernel_launches()
        steady = rounds(eng, cs, mode == "batched")
        res[mode] = {"mpix_s": round(pix * len(steady) / (sum(steady) / 1e3) / 1e6, 3),
                     "ms_per_round": round(float(np.mean(steady)), 3),
                     "launches_per_round": round((rfsr.kernel_launches() - launches0) / frames, 1)}
        eng.destroy()
    res["speedup"] = round(res["batched"]["mpix_s"] / res["loop"]["mpix_s"], 3)
    res["workload"] = (f"{what}, {frames} frames each, band-limited panned texture + moving "
                       f"rectangles (crops of one 1080p sequence), device-resident inputs; timed "
                       f"rounds 3..{frames - 1} (3 past frames)")
    return res


MODES = ("rme", "rmc", "frmc", "nnc", "nnc_frmc", "none")


def run_check_modes(rfsr, torch, steps=8):
    """The 1280x720 dynamic-mask recipe under each consistency-check mode: device time of ME and
    of checks + projection (with the RME reverse field), the ME+CC+PR throughput and the fraction
    of missing pixels that receive a projection, over frames with 3 past frames."""
    seq = synth.config2(seed=2, F=3 + steps)
    h, w = seq.shape
    d_smp, d_msk = torch.from_numpy(seq.samples).cuda(), torch.from_numpy(seq.masks).cuda()
    out = {}
    for mode in MODES:
        with rfsr.Engine(device=torch.cuda.current_device(), profile=True) as eng:
            st = eng.create_stream(height=h, width=w, cc_mode=mode, template_size=T,
                                   search_radius=R, num_refs=KREF)
            ph, proj = [], []
            for f in range(3 + steps):
                st.push_frame_device(d_smp[f], d_msk[f])
                st.get_frame_device(timeout_ms=120000)
                if f >= 3:
                    ph.append(st.phase_ms())
                    miss = seq.masks[f] == 0
                    proj.append(float((st.debug_get(rfsr.DBG_PCNT)[miss] > 0).mean()))
            a = np.array(ph).mean(axis=0)
            out[mode] = {"me_ms": round(float(a[1]), 4), "cc_pr_ms": round(float(a[2]), 4),
                         "me_cc_pr_mpix_s": round(h * w / ((a[0] + a[1] + a[2]) / 1e3) / 1e6, 3),
                         "projected_frac": round(float(np.mean(proj)), 4)}
    out["workload"] = (f"1280x720 dynamic-mask recipe (band-limited pan + 4 rectangles), K=3, "
                       f"T=9, R=Rc=8, frames 3..{2 + steps}, device-resident inputs, one stream")
    return out


def run_me_predictive(rfsr, torch, radii=(0, 2, 4), steps=8):
    """The opt-in predictive-centre ME (past frames t-2, t-3 searched within radius Rp of k v_1;
    not the paper's method) on the 1080p workload: device time of ME and of checks + projection,
    the ME+CC+PR rate and the projected fraction over frames with 3 past frames (free-running),
    and, on one teacher-forced frame, the share of t-2 / t-3 vectors that differ from the full
    search.  Rp = 0 is the full search (the metric's configuration)."""
    seq = synth.config3(seed=1, F=3 + steps)
    h, w = seq.shape
    d_smp, d_msk = torch.from_numpy(seq.samples).cuda(), torch.from_numpy(seq.masks).cuda()
    t = 3 + steps - 1
    hist = [(seq.frames[t - k], seq.samples[t - k], seq.masks[t - k]) for k in (1, 2, 3)]
    out, exact = {}, None
    for rp in radii:
        with rfsr.Engine(device=torch.cuda.current_device(), profile=True) as eng:
            st = eng.create_stream(height=h, width=w, cc_mode="nnc_frmc", template_size=T,
                                   search_radius=R, num_refs=KREF, me_predict_radius=rp)
            ph, proj = [], []
            for f in range(3 + steps):
                st.push_frame_device(d_smp[f], d_msk[f])
                st.get_frame_device(timeout_ms=120000)
                if f >= 3:
                    ph.append(st.phase_ms())
                    miss = seq.masks[f] == 0
                    proj.append(float((st.debug_get(rfsr.DBG_PCNT)[miss] > 0).mean()))
            st.set_history(hist)
            st.push_frame(seq.samples[t], seq.masks[t])
            st.get_frame(timeout_ms=120000)
            mv = [st.debug_get(rfsr.DBG_MV, k) for k in (2, 3)]
        a = np.array(ph).mean(axis=0)
        if exact is None:
            exact = mv
        out[f"rp_{rp}"] = {
            "me_ms": round(float(a[1]), 4), "cc_pr_ms": round(float(a[2]), 4),
            "me_cc_pr_mpix_s": round(h * w / ((a[0] + a[1] + a[2]) / 1e3) / 1e6, 3),
            "projected_frac": round(float(np.mean(proj)), 4),
            "vectors_changed_frac": [round(float((m != e).any(axis=-1).mean()), 4)
                                     for m, e in zip(mv, exact)]}
    out["workload"] = (f"1920x1080 workload, NNC+FRMC, K=3, T=9, R=8, frames 3..{2 + steps} "
                       f"free-running; changed vectors of t-2 / t-3 on frame {t} with the "
                       f"generator's frames as history; rp_0 = the full search")
    return out


def run_fused_me_cc(rfsr, torch, steps=12):
    """The 1080p workload with ME and the checks as separate launches (the default) and as one
    fused persistent launch per frame (engine option fuse_me_cc): device time of ME + checks +
    projection per frame over frames with 3 past frames, L2 not flushed."""
    seq = synth.config3(seed=1, F=3 + steps)
    h, w = seq.shape
    d_smp, d_msk = torch.from_numpy(seq.samples).cuda(), torch.from_numpy(seq.masks).cuda()
    out = {}
    for name, fuse in (("separate", False), ("fused", True)):
        with rfsr.Engine(device=torch.cuda.current_device(), profile=True, fuse_me_cc=fuse) as eng:
            st = eng.create_stream(height=h, width=w, cc_mode="nnc_frmc", template_size=T,
                                   search_radius=R, num_refs=KREF)
            ph = []
            for f in range(3 + steps):
                st.push_frame_device(d_smp[f], d_msk[f])
                st.get_frame_device(timeout_ms=120000)
                if f >= 3:
                    ph.append(st.phase_ms())
            a = np.array(ph).mean(axis=0)
            out[name] = {"me_cc_pr_ms": round(float(a[1] + a[2]), 4),
                         "launches_per_frame": 3 if fuse else 4}
    out["fused_over_separate"] = round(out["fused"]["me_cc_pr_ms"] / out["separate"]["me_cc_pr_ms"], 3)
    out["workload"] = (f"1920x1080 workload, NNC+FRMC, K=3, T=9, R=8, frames 3..{2 + steps}, "
                       f"device-resident inputs, one unbatched stream (launches: ingest, ME, "
                       f"checks, FSR; fused: ingest, ME + checks, FSR)")
    return out


def run_concealed(rfsr, torch, delta=0.5, frames=3):
    """Stand-alone FSR (rfsr_fsr_device) of one 1080p frame of the workload with concealed weighting
    delta > 0 (wavefronts, one launch per wave) against delta = 0 (all blocks in one launch):
    device time per frame, with the projections of the generator's ground truth."""
    seq = synth.config3(seed=3, F=1)
    H, W = seq.shape
    smp, msk = seq.samples[0], seq.masks[0]
    rng = np.random.default_rng(3)
    pcnt = np.where((msk == 0) & (rng.random((H, W)) < 0.4), 1, 0).astype(np.uint8)
    psum = (pcnt.astype(np.uint16) * seq.frames[0]).astype(np.uint16)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d = [dev(smp), dev(msk), dev(psum), dev(pcnt)]
    out32 = torch.zeros((H, W), dtype=torch.float32, device="cuda")
    out8 = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    res = {}
    for dl in (0.0, delta):
        call = lambda: rfsr.fsr_device(*d, out32, out8, H, W, cuda_stream=s.cuda_stream,
                                       fsr_concealed_weight=dl)
        call()
        n0 = rfsr.kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(frames):
            call()
        e1.record(s)
        torch.cuda.synchronize()
        res[f"delta_{dl:g}"] = {"ms_per_frame": round(e0.elapsed_time(e1) / frames, 3),
                                "launches_per_frame": (rfsr.kernel_launches() - n0) // frames}
    res["workload"] = ("FSR alone, 1920x1080 frame 0 of the workload, 40 % of missing pixels "
                       "projected, 100 iterations; L2 not flushed (FSR reads 12 MB per frame)")
    return res


def run_serving_all(rfsr, torch, frame_scale=0.1):
    """The serving report: paced cameras first (the latency a stream sees below saturation), then
    the saturated closed loop with the whole memory and under a 2 GB budget, then the unloaded
    service time per size."""
    return {"paced_30fps": run_serving(rfsr, torch, n_streams=64, rate_hz=5.0, pace_fps=30.0,
                                       frame_scale=frame_scale),
            "closed_loop": run_serving(rfsr, torch, frame_scale=frame_scale),
            "budget_2gb": run_serving(rfsr, torch, memory_budget=2 << 30, frame_scale=frame_scale),
            "unloaded": run_unloaded_latency(rfsr, torch)}


def run_unloaded_latency(rfsr, torch, frames=12):
    """Per-frame latency of the serving engine with one stream alone and one frame in flight
    (host buffers, push -> collected), per size of the arrival mix: the service time that the
    loaded runs add queueing to."""
    import time as _t
    base = synth.config3(seed=56, H=2160, W=3840, F=4)
    out = {}
    for (H, W) in SIZES5:
        rng = np.random.default_rng(H + W)
        perm = synth.dynamic_permutations(H, W, rng)
        ms = [synth.positions_to_mask(synth.dynamic_positions(perm, t)) for t in range(4)]
        sm = [np.ascontiguousarray(base.frames[t, :H, :W] * ms[t]) for t in range(4)]
        with rfsr.Engine(device=torch.cuda.current_device(), serve=True, max_inflight=2) as eng:
            st = eng.create_stream(height=H, width=W)
            lat = []
            for t in range(frames):
                t0 = _t.perf_counter()
                st.push_frame(sm[t % 4], ms[t % 4])
                st.get_frame(timeout_ms=120000)
                if t >= 3:
                    lat.append(1e3 * (_t.perf_counter() - t0))
        out[f"{W}x{H}"] = {"p50_ms": round(float(np.percentile(lat, 50)), 3),
                           "p99_ms": round(float(np.percentile(lat, 99)), 3)}
    return out


def run_serving(rfsr, torch, n_streams=256, rate_hz=20.0, frame_scale=0.1, seed=5, memory_budget=0,
                pace_fps=0.0):
    """Poisson arrivals on a serving engine, closed loop with <= 2 frames in flight per stream:
    per-frame latency (push returned -> result collected) and aggregate throughput.  pace_fps > 0
    paces every stream: frame n is pushed no earlier than n / pace_fps after the stream's
    arrival (a camera), still with <= 2 frames in flight."""
    import time as _t
    arr = synth.config5_arrivals(seed=seed, n_streams=n_streams, rate_hz=rate_hz)
    nf = [max(2, int(round(a.spec.frames * frame_scale))) for a in arr]
    # content: the 1/f^2 + moving objects recipe at the largest size; every stream is a crop at
    # its own seeded offset, starting at its own seeded frame, with its own seeded mask(s).  The
    # frame is pushed whole as the sample plane (the library ignores unmeasured bytes).
    nbase = 16
    base = synth.config3(seed=55, H=2160, W=3840, F=nbase)
    crops, masks = {}, {}
    for i, a in enumerate(arr):
        sp = a.spec
        rng = np.random.default_rng(sp.seed)
        y0 = int(rng.integers(0, 2160 - sp.H + 1)) & ~1
        x0 = int(rng.integers(0, 3840 - sp.W + 1)) & ~1
        crops[i] = (y0, x0, int(rng.integers(0, nbase)))
        if sp.mask_type == synth.MASK_FIXED:
            masks[i] = [synth.positions_to_mask(synth.fixed_positions(sp.H, sp.W, rng))]
        else:
            perm = synth.dynamic_permutations(sp.H, sp.W, rng)
            masks[i] = [synth.positions_to_mask(synth.dynamic_positions(perm, t)) for t in range(4)]

    def frame_of(i, n):
        y0, x0, t0 = crops[i]
        sp = arr[i].spec
        return base.frames[(t0 + n) % nbase, y0:y0 + sp.H, x0:x0 + sp.W]
    eng = rfsr.Engine(device=torch.cuda.current_device(), serve=True, max_inflight=2,
                      memory_budget=memory_budget)
    n_queued, max_queue = 0, 0
    active, lat, done_px = {}, [], 0
    nxt = 0
    t_start = _t.perf_counter()
    queued = []
    while nxt < len(arr) or active or queued:
        now = _t.perf_counter() - t_start
        while nxt < len(arr) and arr[nxt].time_s <= now:
            sp = arr[nxt].spec
            st = eng.create_stream(allow_queued=True, height=sp.H, width=sp.W,
                                   mask_type=sp.mask_type)
            if st.live:
                active[nxt] = [st, 0, [], _t.perf_counter()]
            else:
                queued.append((nxt, st))
                n_queued += 1
                max_queue = max(max_queue, len(queued))
            nxt += 1
        for q in list(queued):
            if q[1].live:
                active[q[0]] = [q[1], 0, [], _t.perf_counter()]
                queued.remove(q)
        for i in list(active):
            st, sent, inflight, t0 = active[i]
            due = pace_fps <= 0 or _t.perf_counter() - t0 >= sent / pace_fps
            if sent < nf[i] and len(inflight) < 2 and due:
                st.push_frame(frame_of(i, sent), masks[i][sent % len(masks[i])])
                inflight.append(_t.perf_counter())
                active[i][1] = sent + 1
            if inflight:
                try:
                    st.get_frame(timeout_ms=0)
                except rfsr.RfsrError as e:
                    if e.code != rfsr.RFSR_ETIMEDOUT:
                        raise
                else:
                    lat.append(_t.perf_counter() - inflight.pop(0))
                    done_px += st.H * st.W
            if active[i][1] >= nf[i] and not inflight:
                st.destroy()
                del active[i]
    wall = _t.perf_counter() - t_start
    eng.destroy()
    lat_ms = np.array(lat) * 1e3
    loop = (f"each stream paced at {pace_fps:g} fps" if pace_fps > 0 else "closed loop") + \
        " with <= 2 frames in flight per stream"
    return {"p50_ms": round(float(np.percentile(lat_ms, 50)), 3),
            "p99_ms": round(float(np.percentile(lat_ms, 99)), 3),
            "mpix_s": round(done_px / wall / 1e6, 3), "frames": int(len(lat)),
            "wall_s": round(wall, 2),
            "memory_budget": memory_budget or "80% of free device memory",
            "streams_queued": n_queued, "max_queue": max_queue,
            "workload": (f"{n_streams} streams arriving Poisson at {rate_hz:g}/s, sizes "
                         "320x240..3840x2160, fixed or dynamic mask 50/50 (seeded per stream), "
                         "1/f^2 texture + moving objects (each stream its own seeded crop and "
                         f"start frame of a 16-frame 4K sequence), frames U{{30..300}} x "
                         f"{frame_scale:g}, {loop}, host buffers, serving engine (continuous "
                         "batching, memory admission)")}


# ---------------------------------------------------------------------------------------------
# reconstruction quality (frame-wise PSNR / SSIM against the ground-truth frames)
# ---------------------------------------------------------------------------------------------
def border_px(h, w):
    """The paper omits a 40-pixel border at 1280x720; scaled to the frame size (at least 2)."""
    return max(2, int(round(40 * min(h / 720.0, w / 1280.0))))


def psnr(a, b, border):
    d = a[border:-border, border:-border].astype(np.float64) - b[border:-border, border:-border]
    mse = float(np.mean(d * d))
    return 99.0 if mse == 0 else 10.0 * np.log10(255.0 ** 2 / mse)


def ssim(a, b, border):
    """Mean SSIM (Wang et al. 2004: 11x11 Gaussian window, sigma 1.5, K1 0.01, K2 0.03, L 255)."""
    import scipy.ndimage as nd
    x, y = a.astype(np.float64), b.astype(np.float64)
    f = lambda z: nd.gaussian_filter(z, 1.5, truncate=3.5)
    mx, my = f(x), f(y)
    sxx, syy, sxy = f(x * x) - mx * mx, f(y * y) - my * my, f(x * y) - mx * my
    c1, c2 = (0.01 * 255) ** 2, (0.03 * 255) ** 2
    m = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return float(m[border:-border, border:-border].mean())


QUALITY_METHODS = [
    ("fsr_single_frame", dict(num_refs=0, cc_mode="none")),
    ("rfsr_rme", dict(cc_mode="rme", fsr_overwrite_projected=1)),
    ("dfsr_rme", dict(cc_mode="rme")),
    ("dfsr_rmc", dict(cc_mode="rmc")),
    ("dfsr_frmc", dict(cc_mode="frmc")),
    ("dfsr_nnc", dict(cc_mode="nnc")),
    ("dfsr_nnc_frmc", dict(cc_mode="nnc_frmc")),
    ("dfsr_no_check", dict(cc_mode="none")),
]


def quality_run(rfsr, seq, method_kw, with_ssim=True):
    """Free-running recursion through the stream API; per frame (PSNR, SSIM) of the 8-bit output."""
    h, w = seq.shape
    b = border_px(h, w)
    out = []
    with rfsr.Engine(device=0) as eng:
        st = eng.create_stream(height=h, width=w, mask_type=seq.mask_type, **method_kw)
        for t in range(len(seq)):
            st.push_frame(seq.samples[t], seq.masks[t])
            rec = st.get_frame(timeout_ms=120000)
            out.append((psnr(rec, seq.frames[t], b), ssim(rec, seq.frames[t], b) if with_ssim else None))
    return out


def run_quality(rfsr, torch):
    seqs = [("1280x720 dynamic", synth.config2(seed=2, F=32)),
            ("1280x720 fixed", synth.config2(seed=2, F=32, mask_type=synth.MASK_FIXED)),
            ("1920x1080 dynamic", synth.config3(seed=3, F=24)),
            ("64x64 fixed translation", synth.config1(seed=1))]
    res = {}
    for name, seq in seqs:
        r = {}
        for m, kw in QUALITY_METHODS:
            q = quality_run(rfsr, seq, kw)
            p = np.array([a for a, _ in q])
            s_ = np.array([b for _, b in q])
            r[m] = {"psnr_db": round(float(p.mean()), 3), "ssim": round(float(s_.mean()), 4),
                    "psnr_db_frames_10_on": round(float(p[10:].mean()), 3) if len(p) > 10 else None}
        base = r["fsr_single_frame"]["psnr_db"]
        for m in r:
            r[m]["gain_vs_single_frame_db"] = round(r[m]["psnr_db"] - base, 3)
        res[name] = r
    res["protocol"] = ("free-running recursion through rfsr_push_frame / rfsr_get_frame, K=3, T=9, "
                       "R=Rc=8, FSR 100 iterations; frame-wise PSNR and mean SSIM of the 8-bit "
                       "output against the generator's ground truth with the paper's 40-pixel "
                       "border (scaled to the frame size) omitted, averaged over all frames")
    return res


# ---------------------------------------------------------------------------------------------
# N > 1: one independent replica per rank (weak scaling), times reduced by maximum
# ---------------------------------------------------------------------------------------------
def replica_seed(rank: int) -> int:
    """Each rank runs the 1080p recipe with its own content seed (independent replicas)."""
    return 3 + rank


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The whole job's time is the slowest rank's (all_reduce MAX; identity for one rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(frames_per_rank: int, world: int, pixels: int, seconds: float) -> float:
    """HR Mpixel/s of the whole job: every rank's frames over the slowest rank's time."""
    return frames_per_rank * world * pixels / seconds / 1e6


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2203_09200_gb300 import build as pbuild
    from paper_2203_09200_gb300 import rfsr

    torch.cuda.set_device(local_rank)
    pbuild.build()
    seq = synth.config3(seed=replica_seed(rank), F=F)
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
    if sampler:
        sampler.wait_first()
    launches0 = rfsr.kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    phases = []
    frames_run = []
    checked = []                                # pixels FRMC checked, per timed frame
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
        frames_run.append((nwarm + i) % F)
        # the work count of this frame (outside the events): NNC+FRMC decides ACCEPT or
        # CHECK_REJECT exactly for the pixels its FRMC checked
        dec = np.stack([st.debug_get(rfsr.DBG_DECISION, k) for k in range(1, KREF + 1)])
        checked.append(((dec == rfsr.DEC_ACCEPT) | (dec == rfsr.DEC_CHECK_REJECT)).sum(axis=0))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = rfsr.kernel_launches() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_s = max_over_ranks(sum(step_ms) / 1e3, world)
    if world > 1:
        dist.barrier()
    ph = np.array(phases)                       # (steps, 4): ingest, ME, checks+PR, FSR
    ph_mean = ph.mean(axis=0)
    # ingest + ME + checks + projection over all steps
    mecc_s = max_over_ranks(float(ph[:, :3].sum()) / 1e3, world)
    value = job_rate(args.steps, world, HW, mecc_s)     # the metric: ME+CC+projection
    full_value = job_rate(args.steps, world, HW, tot_s)

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
    # two frames in flight: frame i+1 is pushed (validated, staged, copied) while frame i runs;
    # every step's host->device copy and device->host read stay inside the timed region
    st2.push_frame(host_s[nwarm % F], host_m[nwarm % F])
    for i in range(args.steps):
        if i + 1 < args.steps:
            f = (nwarm + i + 1) % F
            st2.push_frame(host_s[f], host_m[f])
        st2.get_frame(timeout_ms=120000)
    torch.cuda.synchronize()
    e_s = max_over_ranks(time.perf_counter() - e0, world)
    clocks = sampler.stop() if sampler else None    # sampled over both timed regions
    e2e = job_rate(args.steps, world, HW, e_s)
    eng.destroy()
    del d_smp, d_msk, flush
    batching = serving = check_modes = concealed = me_predictive = fused = None
    if not args.no_serving:
        batching = run_batching(rfsr, torch)
        batching["small_frames"] = run_batching(
            rfsr, torch, small_streams(), what="256 streams of 320x240, half fixed / half dynamic masks")
        serving = run_serving_all(rfsr, torch)
        check_modes = run_check_modes(rfsr, torch)
        concealed = run_concealed(rfsr, torch)
        me_predictive = run_me_predictive(rfsr, torch)
        fused = run_fused_me_cc(rfsr, torch)

    if rank != 0:
        return
    hbm, mhz, src = load_peaks()
    nb = (H // 4) * (W // 4)
    fsr_flops = fsr_flops_per_block() * nb
    fp32_peak = SMS * FP32_LANES_PER_SM * 2 * mhz * 1e6
    # the metric's path as one unit: ME (me9_kernel) + checks and projection (cc_project_kernel),
    # algorithmic masked byte |a-b| per frame over their summed CUDA-event time per frame
    me_w, cc_w = {}, []
    for f, chk in zip(frames_run, checked):
        key = seq.masks[f].tobytes()
        if key not in me_w:
            me_w[key] = (KREF * me_byteops(seq.masks[f]), frmc_source_work(seq.masks[f]))
        cc_w.append(int((me_w[key][1] * chk).sum()))
    me_ops = float(np.mean([me_w[seq.masks[f].tobytes()][0] for f in frames_run]))
    cc_ops = float(np.mean(cc_w))
    _, vabs_clk = rfsr.alu_peak("vabsdiffu4", device=local_rank)
    byte_peak = vabs_clk * 4 * SMS * mhz * 1e6
    me_s, cc_s, fsr_s = ph_mean[1] / 1e3, ph_mean[2] / 1e3, ph_mean[3] / 1e3
    ach = (me_ops + cc_ops) / (me_s + cc_s)
    tr_me, tr_cc = profiled_traffic("me9_kernel"), profiled_traffic("cc_project_kernel")
    roof = {"kernel": "me9_kernel + cc_project_kernel<9> (ME + checks + projection, one launch "
                      "each per frame: the metric's path)",
            "bound": "alu", "achieved": round(ach / 1e12, 3), "peak": round(byte_peak / 1e12, 3),
            "unit": "T masked byte |a-b| per s", "frac": round(ach / byte_peak, 4),
            "traffic": (tr_me + tr_cc) if tr_me and tr_cc else None,
            "work_per_frame": {"me_byteops": me_ops, "frmc_byteops": cc_ops,
                               "frmc_checked_pixels": float(np.mean([c.sum() for c in checked])),
                               "me_cost_evaluations": KREF * me_cost_evaluations(H, W)},
            "me_cost_evaluations_per_s": round(KREF * me_cost_evaluations(H, W) / me_s, 1),
            "dram_gbs": (round((tr_me + tr_cc) / (me_s + cc_s) / 1e9, 2) if tr_me and tr_cc
                         else None),
            "peak_source": f"__vabsdiffu4 (4 byte |a-b| per instruction) measured by rfsr_alu_peak: "
                           f"{vabs_clk:.1f} per clock per SM x 4 bytes x {SMS} SMs x {mhz:.0f} MHz "
                           f"({src} max clock)",
            "other": {"me9_kernel": {"achieved": round(me_ops / me_s / 1e12, 3),
                                     "peak": round(byte_peak / 1e12, 3),
                                     "unit": "T masked byte |a-b| per s",
                                     "frac": round(me_ops / me_s / byte_peak, 4)},
                      "fsr_kernel": {"achieved": round(fsr_flops / fsr_s / 1e12, 3),
                                     "peak": round(fp32_peak / 1e12, 3), "unit": "TFLOP/s (fp32)",
                                     "frac": round(fsr_flops / fsr_s / fp32_peak, 4),
                                     "traffic": profiled_traffic("fsr_kernel"),
                                     "peak_source": f"derived: {SMS} SMs x "
                                                    f"{FP32_LANES_PER_SM * 2} flop/clk x {mhz:.0f} MHz"}}}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        rate, full, tot = oracle_crop_rate(seq, 8, (96, 96), seed=5)
        ncpu = os.cpu_count() or 1
        orate, ofull, otot = oracle_crop_rate(seq, 16, (128, 128), seed=6, threads=ncpu)
        cpu = {"value": round(rate, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
               "full_step_value": round(full, 6),
               "sample": f"oracle frame step (NNC+FRMC) on eight 96x96 crops of frames 3..10 of "
                         f"the 1080p workload with 3 past frames each: ME+CC+PR alone (value), "
                         f"then with FSR (full_step_value); {tot:.1f} s on one host core",
               "openmp": {"value": round(orate, 6), "full_step_value": round(ofull, 6),
                          "cores": ncpu, "sample": f"the oracle's OpenMP build (same results) on "
                          f"sixteen 128x128 crops, {otot:.1f} s on {ncpu} host threads"}}
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * tot_s / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "value_scope": "ingest + ME + checks + projection: device "
                   "time between the phase events of each timed full frame step (same stream); "
                   "ms_per_step and full_step cover the whole step with FSR",
                   "l2": "flushed between timed steps (256 MB write, outside the events)",
                   "parallelism": f"replicas x{world}"},
        "breakdown": {"ingest_ms": round(ph_mean[0], 4), "me_ms": round(ph_mean[1], 4),
                      "cc_pr_ms": round(ph_mean[2], 4), "fsr_ms": round(ph_mean[3], 4),
                      "wall_ms_per_step": round(1e3 * wall / args.steps, 4)},
        "full_step": {"value": round(full_value, 3), "unit": UNIT,
                      "scope": "ingest, ME, checks, projection, FSR, 8-bit reconstruction"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e, 3), "unit": UNIT, "h2d_bytes_per_step": 2 * HW,
                "d2h_bytes_per_step": HW,
                "scope": "full frame step through rfsr_push_frame / rfsr_get_frame with host "
                         "buffers, two frames in flight (every copy inside the timed region); the "
                         "public stream API always runs the whole step, so this is the full-step "
                         "metric"},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "batching": batching,
        "serving": serving,
        "check_modes": check_modes,
        "concealed_fsr": concealed,
        "me_predictive": me_predictive,
        "fused_me_cc": fused,
    }
    print(json.dumps(line), flush=True)


def summarize_launches(path):
    """Markdown table of an ncu launch list (--metrics gpu__time_duration.sum --csv): launches,
    total and mean device time and share of each kernel."""
    import collections
    import csv
    rows = list(csv.reader(open(path)))
    hdr = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hdr]
    ki, vi, ui = h.index("Kernel Name"), h.index("Metric Value"), h.index("Metric Unit")
    scale = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0}
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows[hdr + 1:]:
        if len(r) <= vi:
            continue
        name = r[ki].split("(")[0]
        for pre in ("rfsr::<unnamed>::", "<unnamed>::", "unnamed>::", "rfsr::", "void "):
            name = name.replace(pre, "")
        agg[name][0] += 1
        agg[name][1] += float(r[vi].replace(",", "")) * scale[r[ui]]
    tot = sum(v[1] for v in agg.values())
    out = ["| kernel | launches | total ms | mean ms | share |", "|---|---|---|---|---|"]
    for n, (c, t) in sorted(agg.items(), key=lambda x: -x[1][1]):
        out.append(f"| {n[:70]} | {c} | {t:.3f} | {t / c:.3f} | {100 * t / tot:.1f}% |")
    return "\n".join(out)


def run_ncu_case(args):
    """A short, untimed kernel sequence for an ncu capture: 'frame_step' runs `frames` frames of
    the 1080p workload on one unbatched stream (device-resident inputs, check mode --cc-mode,
    predictive-centre ME radius --me-predict-radius, fused ME + checks with --fuse-me-cc);
    'batched' runs `frames` batched steps of --streams streams of the uneven-size mix (default
    tile shape, no autotuning)."""
    import torch
    from paper_2203_09200_gb300 import build as pbuild
    from paper_2203_09200_gb300 import rfsr
    torch.cuda.set_device(0)
    pbuild.build()
    nf = args.frames
    if args.ncu_case == "frame_step":
        seq = synth.config3(seed=3, F=nf)
        d_smp, d_msk = torch.from_numpy(seq.samples).cuda(), torch.from_numpy(seq.masks).cuda()
        with rfsr.Engine(device=0, fuse_me_cc=args.fuse_me_cc) as eng:
            st = eng.create_stream(height=H, width=W, cc_mode=args.cc_mode, template_size=T,
                                   search_radius=R, num_refs=KREF, fsr_iterations=ITERS,
                                   me_predict_radius=args.me_predict_radius)
            for f in range(nf):
                st.push_frame_device(d_smp[f], d_msk[f])
                st.get_frame_device(timeout_ms=120000)
    else:
        specs = synth.config4_streams(n_streams=args.streams, frames=nf)
        streams = crop_streams(synth.config2(seed=44, H=1080, W=1920, F=nf), specs, nf)
        d_in = [[(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in zip(sm, mk)]
                for _, sm, mk in streams]
        with rfsr.Engine(device=0, batched=True, autotune=False) as eng:
            sts = [eng.create_stream(height=sp.H, width=sp.W, mask_type=sp.mask_type)
                   for sp, _, _ in streams]
            for f in range(nf):
                for i, st in enumerate(sts):
                    st.push_frame_device(*d_in[i][f])
                eng.step()
                for st in sts:
                    st.get_frame_device(timeout_ms=120000)
    torch.cuda.synchronize()
    print(f"ncu case {args.ncu_case}: {nf} frames done", flush=True)


def build_parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the batching and serving measurements")
    ap.add_argument("--ncu-case", choices=["frame_step", "batched"],
                    help="run only a short untimed kernel sequence (for ncu captures)")
    ap.add_argument("--frames", type=int, default=6, help="frames of --ncu-case")
    ap.add_argument("--streams", type=int, default=64, help="streams of --ncu-case batched")
    ap.add_argument("--cc-mode", default="nnc_frmc", choices=list(MODES),
                    help="consistency-check mode of --ncu-case frame_step")
    ap.add_argument("--fuse-me-cc", action="store_true",
                    help="--ncu-case frame_step with the fused ME + checks launch")
    ap.add_argument("--me-predict-radius", type=int, default=0,
                    help="predictive-centre ME radius of --ncu-case frame_step (0: full search)")
    ap.add_argument("--serving-full", action="store_true",
                    help="print the serving report with every stream's full U{30..300} frames and "
                         "exit (the default run plays a tenth of each stream's frames)")
    ap.add_argument("--quality", action="store_true",
                    help="print the reconstruction-quality table (PSNR / SSIM per method) and exit")
    ap.add_argument("--summarize-launches", metavar="CSV",
                    help="print the per-kernel table of an ncu launch list and exit")
    return ap


def main():
    ap = build_parser()
    args = ap.parse_args()
    if args.summarize_launches:
        print(summarize_launches(args.summarize_launches))
        return
    if args.ncu_case:
        run_ncu_case(args)
        return
    if args.serving_full:
        import torch
        from paper_2203_09200_gb300 import build as pbuild
        from paper_2203_09200_gb300 import rfsr
        torch.cuda.set_device(0)
        pbuild.build()
        print(json.dumps({"serving_full": run_serving_all(rfsr, torch, frame_scale=1.0)}),
              flush=True)
        return
    if args.quality:
        import torch
        from paper_2203_09200_gb300 import build as pbuild
        from paper_2203_09200_gb300 import rfsr
        torch.cuda.set_device(0)
        pbuild.build()
        print(json.dumps({"quality": run_quality(rfsr, torch)}), flush=True)
        return
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
