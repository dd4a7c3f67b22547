#!/usr/bin/env python
"""Benchmark of the w-projection gridding path on GB300 (one JSON line on stdout).

A step is one imaging pass over one batch with all inputs resident in HBM: grid_zero,
vis_compress (placement, compression, compaction, normaliser), grid_vis (the gridder) and
grid_correct (inverse FFT, normalisation, taper and sinc correction, Stokes I).  The table
build is one-off and outside the timed region, as in the thesis (Sec. 5.3.1 times the
gridder only).  Inputs (6.2 GB for the default workload) are larger than L2.

value  = real grid-point updates per second of the whole step, summed over ranks: the updates
         the gridder performs, gridded records x S^2 x polarisations (the thesis's "real rate",
         Sec. 5.3.1).  The "total" rate, which also counts the compressed records as if they
         were gridded, is reported beside it under `rates`.
e2e    = the same metric with pinned host inputs copied to the device and the Stokes-I image
         copied back inside the timed region of every step (double-buffered: the copies of the
         next step overlap the current step's compute).
roofline = the gridder kernel against the FP32 FMA pipe (8 flops per update, Sec. 5.4.4).

`--impl reference` times the FP64 CPU oracle on the host cores on bounded samples of the
same workload (only rank 0 runs it under torchrun).
"""
import argparse
import datetime
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
sys.path.insert(0, ROOT)

WORKLOADS = {
    "wproj_2k": "64 stations (3 km Gaussian), 2016 baselines x 3600 steps at 1 s, 16 channels 120-180 MHz, "
                "4 pols, complex64; grid 2048^2 x 16 ch; 32 sqrt(w)-spaced w-planes, supports 9..65; "
                "beta=8; FP32 table; compression on",
    "w0_small": "32 stations (2 km disk), 496 baselines x 256 steps at 10 s, 1 channel 150 MHz, 1 pol; "
                "grid 512^2; w=0, support 7, beta=8; compression off",
    "mfs_2k": "channel interleaving onto one grid (multi-frequency synthesis): the wproj_2k geometry (2016 "
              "baselines x 3600 steps at 1 s, 4 pols) with 16 channels 12.2 kHz apart from 150 MHz; grid 2048^2 x 1; "
              "32 sqrt(w)-spaced w-planes, supports 9..65; beta=8; FP32 table; compression over the natural "
              "record order",
    "wstack_2k": "w-stacking: the wproj_2k geometry (2016 baselines x 3600 steps at 1 s, 4 pols) with 4 channels "
                 "120-124 MHz; 32 sqrt(w)-spaced planes each holding the w = 0 kernel (support 9) on 2048^2 x 4 x 32 "
                 "grids; the finaliser sums the plane images times exp(+j2pi w_k (n-1)); beta=8; FP32 table; "
                 "compression on",
    "degrid_1k": "differentiable sky model: 1024^2 FP32 sky (4 channels x 4 pols; seeded point sources plus a "
                 "Gaussian blob) -> degridding forward, chi^2 against noisy complex64 visibilities, hand-written "
                 "adjoint gridding backward; 64 stations (3 km Gaussian), 2016 baselines x 600 steps at 6 s, "
                 "4 channels 120-180 MHz, 16 sqrt(w)-spaced w-planes, supports 9..33, beta=8, compression on",
    "batch_8k": "256 stations (10 km log-radial), 32640 baselines x 1800 steps at 2 s, 64 channels 50-350 MHz, "
                "1 pol, complex64; grid 8192^2 x 64 ch; 64 sqrt(w)-spaced w-planes, supports 9..129; beta=8; "
                "FP32 table; compression on; 8 groups of 8 channels prepared one after another into one work "
                "list (WG_PREP_APPEND), one persistent gridder launch over all 64 channels, the whole step "
                "captured in one CUDA graph, gridder plan autotuned on the appended batch",
}
# the unit of `value` and `e2e` in both arms (the driver divides one arm's value by the other's)
UNIT = "G grid-point updates/s (real rate: updates the gridder performs, whole step)"
# precision variants timed beside the plain FP32 path: (name, table store, half vis, compensated)
VARIANTS = (("fp32+compensated", "f32", False, True), ("f16 table", "f16", False, False),
            ("bf16 table", "bf16", False, False), ("f16 vis", "f32", True, False),
            ("f16 table+f16 vis+compensated", "f16", True, True))
# bounded CPU samples of the same geometry (channels, time steps)
CPU_SAMPLE = {"wproj_2k": (16, 1200), "w0_small": (1, 256), "batch_8k": (2, 720), "degrid_1k": (1, 300),
              "mfs_2k": (4, 1200), "wstack_2k": (2, 1200)}
# worker processes of the CPU baseline (one channel each) where the oracle's table build is cheap
CPU_PROCS = {"wproj_2k": 16}
REF_SAMPLE = {"wproj_2k": (2, 360), "w0_small": (1, 256), "batch_8k": (1, 40), "degrid_1k": (1, 60)}
COMPRESS = {"wproj_2k": True, "w0_small": False, "batch_8k": True, "degrid_1k": True, "mfs_2k": True,
            "wstack_2k": True}
# channel interleaving: every channel onto one grid, compression in natural record order
INTERLEAVE = {"mfs_2k": True}
# w-stacking: planes of the w = 0 kernel (support WSTACK_SUPPORT), one grid channel per plane
WSTACK = {"wstack_2k": 32}
WSTACK_SUPPORT = 9
# workloads that are a slice of another geometry
SYNTH_NAME = {"wstack_2k": ("wproj_2k", {"n_chan": 4})}
CHAN_GROUP = {"batch_8k": 8}
# gridder plans the autotuner tries (seg_len, slots, fixed R): on the batch for the single-grid
# workloads, per channel group for the batched one
STEP_PLANS = [(128, 256, False), (128, 256, True), (256, 256, True), (64, 256, True), (128, 128, True),
              (128, 128, False)]
BATCH_PLANS = [(256, 256, True), (256, 256, False), (128, 256, True), (256, 128, True)]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms.  Started (and waited for) before the
    warm-up so that its start-up never falls inside the timed region; only samples time-stamped
    inside the timed region are kept."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.t0 = self.t1 = None
        self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self, wait_s=20.0):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        t = time.time()
        while time.time() - t < wait_s:
            if os.path.getsize(self.tmp.name) > 0:
                break
            time.sleep(0.1)

    def begin(self):
        self.t0 = datetime.datetime.now()

    def end(self):
        self.t1 = datetime.datetime.now()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                except ValueError:
                    continue
                rows.append((ts, parts))
        os.unlink(self.tmp.name)
        inside = [p for ts, p in rows if self.t0 and self.t1 and
                  self.t0 - datetime.timedelta(seconds=0.25) <= ts <= self.t1 + datetime.timedelta(seconds=0.25)]
        if not inside and rows and self.t1:
            inside = [min(rows, key=lambda r: abs((r[0] - self.t1).total_seconds()))[1]]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [v for v in (num(r[1]) for r in inside) if v is not None]
        mx = [v for v in (num(r[2]) for r in inside) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside)}


def barrier(world):
    """All ranks meet (no-op on one rank)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value, world, device="cpu"):
    """The largest of every rank's value (the slowest rank's time), on every rank."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ms, world):
    """Replicas: every rank processes the same units; the job's rate is all ranks' units over
    the slowest rank's time, in 1e9 units per second."""
    return world * units_per_rank / (ms * 1e-3) / 1e9


def measured_ceilings(real_rate: float, P: int) -> dict:
    """The two ceilings of the gridder's roofline, measured on this device by the library's
    microbenchmarks (ceiling_measure): the FP32 FMA rate (8 flops per update) and the kernel-
    sample fetch bandwidth (one 8-byte sample per point and record, shared by P polarisations),
    with the gridder's real update rate against each and against the lower of the two."""
    import paper_1403_4209_gb300 as wg
    c = {k: wg.ceiling(k) for k in ("fp32_fma2", "fp32_fma", "fetch_l1", "fetch_l2", "shared")}
    fma = max(c["fp32_fma2"], c["fp32_fma"]) / 8.0
    l1, l2 = c["fetch_l1"] * P / 8.0, c["fetch_l2"] * P / 8.0
    low = min(fma, l2)
    return {"fp32_fma2_tflops": round(c["fp32_fma2"] / 1e12, 2), "fp32_fma_tflops": round(c["fp32_fma"] / 1e12, 2),
            "fetch_l1_tbs": round(c["fetch_l1"] / 1e12, 2), "fetch_l2_tbs": round(c["fetch_l2"] / 1e12, 2),
            "shared_tbs": round(c["shared"] / 1e12, 2),
            "updates_ceiling_fma_G": round(fma / 1e9, 1), "updates_ceiling_fetch_l2_G": round(l2 / 1e9, 1),
            "updates_ceiling_fetch_l1_G": round(l1 / 1e9, 1), "bound": "fma" if fma <= l2 else "fetch_l2",
            "frac_of_fma": round(real_rate / fma, 4), "frac_of_fetch_l2": round(real_rate / l2, 4),
            "frac_of_min": round(real_rate / low, 4),
            "note": "real gridder updates/s against measured ceilings; kernel samples stream mostly from L2 "
                    "(ncu l1tex hit rate about 16 %), so the fetch ceiling is the L2 one"}


def _gridder_traffic(per_launch_units):
    """DRAM bytes per k_grid launch from the committed ncu summary, scaled to this launch's
    gridded updates; None if the gridder source changed since the counters were taken."""
    prof = os.path.join(ROOT, "profiles", "k_grid_wproj_2k.md")
    src = os.path.join(ROOT, "paper_1403_4209_gb300", "csrc", "grid.cu")
    if not os.path.exists(prof):
        return None
    kv = {}
    with open(prof) as f:
        for line in f:
            if ":" in line and line.startswith("- "):
                k, v = line[2:].rsplit(":", 1)
                kv[k.strip()] = v.strip().strip("`")
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if kv.get("grid.cu sha256[:16]") != h:
            return None
        return float(kv["dram bytes per update"]) * per_launch_units
    except (KeyError, ValueError):
        return None


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_1403_4209_gb300 as wg
    import synth

    torch.cuda.set_device(local_rank)
    dev = "cuda:%d" % local_rank
    base, kw = SYNTH_NAME.get(args.workload, (args.workload, {}))
    kw = dict(kw)
    if args.n_chan is not None:
        kw["n_chan"] = args.n_chan
    wl = synth.make(base, device=dev, n_times=args.n_times, chan0=args.chan0, **kw)
    stack_k = WSTACK.get(args.workload, 0)                 # w-stacking planes (0: w-projection)
    if stack_k:
        tab = wg.ConvTable.build(wl.du, stack_k, wl.w_max, wl.oversample, wl.taper_support,
                                 supports=[WSTACK_SUPPORT] * stack_k, stacking=True)
    else:
        tab = wg.ConvTable.build(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    inter = INTERLEAVE.get(args.workload, False)
    gc = 1 if inter else wl.n_chan * max(1, stack_k)       # grid channels
    g = wg.Grid(wl.n_grid, wl.du, wl.n_pol, gc, device=dev)
    uvw_d = torch.as_tensor(wl.uvw, device=dev)
    freq_d = torch.as_tensor(wl.freq, device=dev)
    batch = wg.VisBatch(uvw_d, freq_d, wl.vis, wl.weight, wl.flag)
    wlst = wg.WorkList(wl.rows * wl.n_chan, wl.n_chan, wl.n_pol)
    img_mode = wg.IMAGE_WSTACK if stack_k else wg.IMAGE_STOKES_I
    img_shape = (wl.n_chan, wl.n_pol, wl.n_grid, wl.n_grid) if stack_k else (gc, wl.n_grid, wl.n_grid)
    img = torch.empty(img_shape, dtype=torch.float32, device=dev)
    compress = COMPRESS[args.workload]
    stream = torch.cuda.current_stream()
    ev_g = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]

    ev_p = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]

    def step(k=None):
        g.zero()
        if k is not None:
            ev_p[k][0].record(stream)
        wg.vis_compress(g, tab, batch, wlst, compress=compress, interleave=inter, wstack=bool(stack_k))
        if k is not None:
            ev_p[k][1].record(stream)
            ev_g[k][0].record(stream)
        wg.grid_vis(g, tab, wlst)
        if k is not None:
            ev_g[k][1].record(stream)
        wg.grid_correct(g, tab, mode=img_mode, out=img)

    # one-off, outside the timed region: pick the gridder plan on this batch
    g.zero()
    wg.vis_compress(g, tab, batch, wlst, compress=compress, interleave=inter, wstack=bool(stack_k))
    plan = wg.grid_autotune(g, tab, wlst, candidates=STEP_PLANS, repeats=2)[:3]

    clocks = ClockSampler(local_rank)
    clocks.start()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = wlst.stats()
    barrier(world)
    torch.cuda.synchronize()
    clocks.begin()
    n0 = wg.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = wg.launch_count() - n0
    clocks.end()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    t_grid = sum(a.elapsed_time(b) for a, b in ev_g) / args.steps
    t_prep = sum(a.elapsed_time(b) for a, b in ev_p) / args.steps
    ms = max_over_ranks(ms, world, dev)
    barrier(world)
    real = st["updates"]
    total = st["updates"] + st["updates_saved"]
    value = whole_job_rate(real, ms, world)

    # end to end: every step copies its inputs from pinned host memory and reads its Stokes-I
    # image back.  The copies of step k+1 run on a copy stream into the other of two device
    # input buffers while step k computes (double buffering).  Measured right after the
    # device-timed steps, over as many steps.
    h_uvw = torch.as_tensor(wl.uvw).pin_memory()
    h_vis = wl.vis.cpu().pin_memory()
    h_w = wl.weight.cpu().pin_memory()
    h_f = wl.flag.cpu().pin_memory()
    h_img = torch.empty(img.shape, dtype=img.dtype).pin_memory()
    h2d = h_uvw.numel() * 8 + h_vis.numel() * 8 + h_w.numel() * 4 + h_f.numel() + freq_d.numel() * 8
    d2h = h_img.numel() * 4
    slots = []
    for _ in range(2):
        u = torch.empty_like(uvw_d)
        slots.append((u, wg.VisBatch(u, freq_d, torch.empty_like(wl.vis), torch.empty_like(wl.weight),
                                     torch.empty_like(wl.flag))))
    cstream = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    ne = max(3, args.steps)
    # per-step copy and compute intervals, for the share of the copies hidden under compute
    tl_c = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ne)]
    tl_s = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ne)]

    def issue_copy(k, tl):
        u, b = slots[k % 2]
        with torch.cuda.stream(cstream):
            cstream.wait_event(consumed[k % 2])
            if tl:
                tl_c[k][0].record(cstream)
            u.copy_(h_uvw, non_blocking=True)
            b.vis.copy_(h_vis, non_blocking=True)
            b.weight.copy_(h_w, non_blocking=True)
            b.flag.copy_(h_f, non_blocking=True)
            if tl:
                tl_c[k][1].record(cstream)
            copied[k % 2].record(cstream)

    def e2e_run(n, tl=False):
        for k in range(2):
            consumed[k].record(stream)
        issue_copy(0, tl)
        for k in range(n):
            if k + 1 < n:
                issue_copy(k + 1, tl)
            stream.wait_event(copied[k % 2])
            if tl:
                tl_s[k][0].record(stream)
            b = slots[k % 2][1]
            g.zero()
            wg.vis_compress(g, tab, b, wlst, compress=compress, interleave=inter, wstack=bool(stack_k))
            wg.grid_vis(g, tab, wlst)
            wg.grid_correct(g, tab, mode=img_mode, out=img)
            # the slot is released after the image read-back is queued, so the next
            # host-to-device copy cannot take the link ahead of it and hold up step k+1
            h_img.copy_(img, non_blocking=True)
            consumed[k % 2].record(stream)
            if tl:
                tl_s[k][1].record(stream)

    e2e_run(2)
    torch.cuda.synchronize()
    barrier(world)
    x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x0.record(stream)
    e2e_run(ne, tl=True)
    x1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = x0.elapsed_time(x1) / ne
    ms_e2e = max_over_ranks(ms_e2e, world, dev)
    # copy k+1 against step k: the share of the copy time that ran under compute
    hid = tot = 0.0
    for k in range(ne - 1):
        c0, c1 = x0.elapsed_time(tl_c[k + 1][0]), x0.elapsed_time(tl_c[k + 1][1])
        s0, s1 = x0.elapsed_time(tl_s[k][0]), x0.elapsed_time(tl_s[k][1])
        tot += c1 - c0
        hid += max(0.0, min(c1, s1) - max(c0, s0))
    copy_hidden = hid / tot if tot > 0 else None
    # mean durations of a copy and of a step while both streams run
    copy_ms_ov = statistics.mean(a.elapsed_time(b) for a, b in tl_c[1:])
    step_ms_ov = statistics.mean(a.elapsed_time(b) for a, b in tl_s)
    # the host-to-device copies alone (the link's share of the end-to-end step)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(cstream)
    for k in range(3):
        u, b = slots[k % 2]
        with torch.cuda.stream(cstream):
            u.copy_(h_uvw, non_blocking=True)
            b.vis.copy_(h_vis, non_blocking=True)
            b.weight.copy_(h_w, non_blocking=True)
            b.flag.copy_(h_f, non_blocking=True)
    c1.record(cstream)
    torch.cuda.synchronize()
    ms_h2d = c0.elapsed_time(c1) / 3
    e2e = {"value": round(whole_job_rate(real, ms_e2e, world), 3), "unit": UNIT,
           "total_rate_G": round(whole_job_rate(total, ms_e2e, world), 3), "ms_per_step": round(ms_e2e, 3), "steps": ne, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "h2d_alone_ms": round(ms_h2d, 3),
           "h2d_gbs": round(h2d / (ms_h2d * 1e-3) / 1e9, 1),
           "copy_hidden_frac": None if copy_hidden is None else round(copy_hidden, 3),
           "copy_ms_overlapped": round(copy_ms_ov, 3), "step_ms_overlapped": round(step_ms_ov, 3),
           "pipelining": "inputs double-buffered on a copy stream"}
    del slots, h_uvw, h_vis, h_w, h_f, h_img
    torch.cuda.synchronize()

    # precision variants (reduced-precision tables, half visibilities, compensated flushes)
    variants = {}
    if not args.no_variants and not inter and not stack_k:
        vis_h, scale_h = synth.to_half_vis(wl.vis)
        batch_h = wg.VisBatch(uvw_d, freq_d, vis_h, wl.weight, wl.flag, vis_scale=scale_h)
        for name, store, half, comp in VARIANTS:
            tv = wg.ConvTable.build(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support,
                                    supports=wl.supports, store=store)
            gv = wg.Grid(wl.n_grid, wl.du, wl.n_pol, wl.n_chan, device=dev, compensated=comp)
            bv = batch_h if half else batch
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            nv = 5
            for it in range(3 + nv):
                if it == 3:
                    evs[0].record(stream)
                gv.zero()
                wg.vis_compress(gv, tv, bv, wlst, compress=compress)
                if it == 3 + nv - 1:
                    evs[2].record(stream)
                wg.grid_vis(gv, tv, wlst)
                if it == 3 + nv - 1:
                    evs[3].record(stream)
                wg.grid_correct(gv, tv, mode=wg.IMAGE_STOKES_I, out=img)
            evs[1].record(stream)
            torch.cuda.synchronize()
            ms_v = evs[0].elapsed_time(evs[1]) / nv
            variants[name] = {"ms_per_step": round(ms_v, 3), "gridder_ms": round(evs[2].elapsed_time(evs[3]), 3),
                              "value": round(real / (ms_v * 1e-3) / 1e9, 1),
                              "total_rate_G": round(total / (ms_v * 1e-3) / 1e9, 1)}
            del tv, gv
        del batch_h, vis_h

    # uniform and robust re-weighting of the same batch (a pre-pass, outside the step)
    w_out = torch.empty_like(batch.weight)
    t_weight = {}
    for scheme in ("uniform", "robust"):
        wg.vis_weight(g, tab, batch, scheme=scheme, interleave=inter, wstack=bool(stack_k), out=w_out)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(3):
            wg.vis_weight(g, tab, batch, scheme=scheme, interleave=inter, wstack=bool(stack_k), out=w_out)
        a1.record(stream)
        torch.cuda.synchronize()
        t_weight[scheme] = a0.elapsed_time(a1) / 3
    del w_out

    # the full-Stokes finaliser on the same grid (quad-pol only), timed separately
    t_stokes = None
    if wl.n_pol == 4 and not stack_k:
        img4 = torch.empty((gc, 4, wl.n_grid, wl.n_grid), dtype=torch.float32, device=dev)
        wg.grid_correct(g, tab, mode=wg.IMAGE_STOKES_LINEAR, out=img4)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(3):
            wg.grid_correct(g, tab, mode=wg.IMAGE_STOKES_LINEAR, out=img4)
        a1.record(stream)
        torch.cuda.synchronize()
        t_stokes = a0.elapsed_time(a1) / 3
        del img4

    # degridding of the same batch (predict mode), timed separately
    out_v = torch.empty_like(wl.vis)
    for _ in range(2):
        wg.degrid_vis(g, tab, batch, wlst, out=out_v)
    torch.cuda.synchronize()
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    nd = max(3, args.steps // 2)
    for _ in range(nd):
        wg.degrid_vis(g, tab, batch, wlst, out=out_v)
    d1.record(stream)
    torch.cuda.synchronize()
    t_degrid = d0.elapsed_time(d1) / nd

    peaks, src = _peaks()
    props = torch.cuda.get_device_properties(local_rank)
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
    achieved = 8.0 * real / (t_grid * 1e-3) / 1e12
    traffic = _gridder_traffic(real)

    line = {
        "metric": "gridding/degridding G grid-point updates/s and % roofline at stated grid error",
        "value": round(value, 3),
        "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "%s: %s%s" % (args.workload, WORKLOADS[args.workload],
                                              "" if args.n_chan is None and args.n_times is None else
                                              " (slice: %s channels, %s steps)" % (args.n_chan, args.n_times)),
                   "records_per_step": wl.rows * wl.n_chan, "l2": "inputs larger than L2 (no flush needed)",
                   "plan_seg_len_slots_fixed_r": plan,
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "rates": {"real_step_G": round(value, 3),
                  "total_step_G": round(whole_job_rate(total, ms, world), 3),
                  "real_gridder_G": round(real / (t_grid * 1e-3) / 1e9, 3),
                  "total_gridder_G": round(total / (t_grid * 1e-3) / 1e9, 3),
                  "degrid_real_G": round(real / (t_degrid * 1e-3) / 1e9, 3),
                  "degrid_total_G": round(total / (t_degrid * 1e-3) / 1e9, 3),
                  "gridder_ms": round(t_grid, 4), "degrid_ms": round(t_degrid, 4),
                  "records_gridded": st["gridded"], "records_compressed": st["compressed"],
                  "record_rate_real_M": round(st["gridded"] / (t_grid * 1e-3) / 1e6, 1),
                  "record_rate_total_M": round(st["griddable"] / (t_grid * 1e-3) / 1e6, 1),
                  "compression_ratio_records": round(st["compressed"] / max(1, st["gridded"]), 3),
                  "compression_ratio_updates": round(st["updates_saved"] / max(1, st["updates"]), 3),
                  "prep_ms": round(t_prep, 4),
                  "weighting_uniform_ms": round(t_weight["uniform"], 3),
                  "weighting_robust_ms": round(t_weight["robust"], 3),
                  "correct_stokes_iquv_ms": None if t_stokes is None else round(t_stokes, 3),
                  "prep_record_rate_M": round(st["records"] / (t_prep * 1e-3) / 1e6, 1),
                  "updates_real": real, "updates_total": total},
        "roofline": {"kernel": "k_grid", "bound": "alu", "achieved": round(achieved, 3),
                     "peak": round(peak_tflops, 2), "unit": "TFLOP/s",
                     "frac": round(achieved / peak_tflops, 4),
                     "peak_source": "FP32 FMA pipe: %d SMs x 128 lanes x 2 flops x %.0f MHz (%s sm_max_mhz)"
                                    % (props.multi_processor_count, sm_mhz, src),
                     "traffic": traffic},
        "ceilings": measured_ceilings(real / (t_grid * 1e-3), wl.n_pol),
        "variants": variants,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        nc, nt = CPU_SAMPLE[args.workload]
        procs = min(CPU_PROCS.get(args.workload, 1), os.cpu_count() or 1, nc)
        line["cpu_baseline"] = cpu_sample(args.workload, nc if procs > 1 else min(nc, 4), nt, procs)
        if args.workload == "wproj_2k" and args.n_chan is None and args.n_times is None:
            errs = variant_errors(dev, plan)
            line["grid_error"] = errs.pop("fp32")
            for name, e in errs.items():
                if name in variants:
                    variants[name]["grid_error"] = e
        else:
            line["grid_error"] = grid_error_sample(args.workload, dev, plan, inter, stack_k)
    return line


def _table_worker(args):
    """One worker of oracle_table_parallel: the kernels of a few planes, as {plane: (samples, zeta)}."""
    du, K, w_max, beta, taper, supports, planes = args
    import oracle
    t = oracle.build_table(du, K, w_max, beta, taper, supports=supports, planes=planes)
    b2 = beta * beta
    return {k: (t.data[t.offsets[k]:t.offsets[k] + b2 * int(t.supports[k]) ** 2].copy(),
                t.zeta[k * b2:(k + 1) * b2].copy()) for k in planes}


def oracle_table_parallel(wl, planes=None, procs=None):
    """The oracle's table (Algorithm "convgen", prescribed supports), its planes built in spawned
    worker processes (every plane is computed independently of the others); `planes` limits
    it to the planes a sample uses.  Host-side set-up of the CPU legs, never timed."""
    import multiprocessing as mp

    import oracle
    K = wl.n_wplanes
    todo = list(range(K)) if planes is None else sorted(int(k) for k in planes)
    t = oracle.build_table(wl.du, K, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports, planes=())
    procs = max(1, min(procs or (os.cpu_count() or 1), len(todo), 16))
    chunks = [todo[i::procs] for i in range(procs)]
    jobs = [(wl.du, K, wl.w_max, wl.oversample, wl.taper_support, list(wl.supports), c) for c in chunks if c]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        parts = pool.map(_table_worker, jobs)
    b2 = wl.oversample ** 2
    for part in parts:
        for k, (d, z) in part.items():
            t.data[t.offsets[k]:t.offsets[k] + d.shape[0]] = d
            t.zeta[k * b2:(k + 1) * b2] = z
    return t


# gridded entries one gridder launch may index (32-bit entry indices, with a margin)
ENTRY_LIMIT = (1 << 31) - 1 - 1024


def split_launches(counts, limit=ENTRY_LIMIT):
    """Consecutive channel groups packed into gridder launches of at most `limit` gridded
    entries each, a group's entries never split; raises ValueError if one group alone has more."""
    launches, cur = [], 0
    for gi, n in enumerate(counts):
        if n > limit:
            raise ValueError("channel group %d has %d gridded entries, more than one launch takes (%d)"
                             % (gi, n, limit))
        if not launches or cur + n > limit:
            launches.append([])
            cur = 0
        launches[-1].append(gi)
        cur += n
    return launches


def batch_grid_error(dev, plan, ot, stores=("f32",)):
    """Grid error of the batched configuration (8192^2, 64 planes, one polarisation) against the
    FP64 oracle's plain gridding on its outer-w slice: 4 channels (331-350 MHz) x 24 steps x 300
    baselines, reaching support 129 (the -m gpu parity test's slice), for each table store."""
    import numpy as np
    import torch

    import oracle
    import paper_1403_4209_gb300 as wg
    import synth
    bl, t0 = synth.outer_w_slice("batch_8k", n_times=24, n_top=100, n_spread=200)
    wl = synth.make("batch_8k", baselines=bl, n_times=24, t_start=t0, n_chan=4, chan0=60)
    b = wg.VisBatch(torch.as_tensor(wl.uvw, device=dev), torch.as_tensor(wl.freq, device=dev), wl.vis.to(dev),
                    wl.weight.to(dev), wl.flag.to(dev))
    got = {}
    for store in stores:
        tab = wg.ConvTable.build(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support,
                                 supports=wl.supports, store=store)
        g = wg.Grid(wl.n_grid, wl.du, wl.n_pol, wl.n_chan, device=dev)
        w = wg.WorkList(wl.rows * wl.n_chan, wl.n_chan, wl.n_pol)
        wg.vis_compress(g, tab, b, w)
        w.plan(tab, *plan)
        wg.grid_vis(g, tab, w)
        got[store] = g.data.cpu().numpy()
        del g, w, tab
        torch.cuda.empty_cache()
    del b
    f = wl.flag.numpy()
    pl = oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, ot, flag=f)
    ref = oracle.grid_plain(pl, ot, wl.vis.numpy(), wl.weight.numpy(), f, wl.n_grid)
    S = pl.S[pl.griddable]
    sample = ("batch_8k geometry, 4 channels (331-350 MHz) x 24 steps around the largest |w| x 300 baselines "
              "(100 with the largest |w|), %d records, supports %d..%d" % (wl.rows * wl.n_chan, int(S.min()), int(S.max())))
    return {store: {"rel_l2": float(np.linalg.norm(v - ref) / np.linalg.norm(ref)),
                    "max_abs_over_max": float(np.max(np.abs(v - ref)) / np.max(np.abs(ref))),
                    "reference": "FP64 oracle, plain gridding definition", "sample": sample}
            for store, v in got.items()}


def run_batch(args, rank, world, local_rank):
    """Batching at scale: every channel group is prepared into one work list (WG_PREP_APPEND)
    onto its channel slice of one grid, then one persistent gridder launch grids every
    channel and one finaliser call makes the Stokes-I images.  The whole step is captured once
    in a CUDA graph and replayed."""
    import torch

    import paper_1403_4209_gb300 as wg
    import synth

    torch.cuda.set_device(local_rank)
    dev = "cuda:%d" % local_rank
    G = CHAN_GROUP[args.workload] if args.n_chan is None else min(CHAN_GROUP[args.workload], args.n_chan)
    wl = synth.make(args.workload, device=dev, n_chan=args.n_chan, n_times=args.n_times, chan_group=G,
                    chan0=args.chan0)
    tab = wg.ConvTable.build(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    N, P, C = wl.n_grid, wl.n_pol, wl.n_chan
    full = torch.zeros((C, N, N, P), dtype=torch.complex64, device=dev)
    img = torch.empty((C, N, N), dtype=torch.float32, device=dev)
    uvw_d = torch.as_tensor(wl.uvw, device=dev)
    grid = wg.Grid(N, wl.du, P, C, storage=full)
    c0s = [c0 for c0, _ in wl.chan_groups]
    freqs = [torch.as_tensor(wl.freq[c0:c1], device=dev) for c0, c1 in wl.chan_groups]
    batches = [(c0, wg.VisBatch(uvw_d, fq, v, w, f))
               for (c0, _), fq, v, w, f in zip(wl.chan_groups, freqs, wl.vis, wl.weight, wl.flag)]
    stream = torch.cuda.current_stream()
    in_bytes = wl.uvw.nbytes + sum(v.numel() * 8 + f.numel() for v, f in zip(wl.vis, wl.flag)) + \
        wl.weight[0].numel() * 4

    # sizing pass: each group prepared on its own gives the statistics and the number of
    # gridded entries, so the appended work list is created with room for all of them.  Groups
    # are split over launches only if the entries of one launch would pass 2^31 - 1.
    wtmp = wg.WorkList(wl.rows * G, G, P)
    real, total, counts = 0, 0, []
    for (c0, c1), (_, b) in zip(wl.chan_groups, batches):
        view = wg.Grid(N, wl.du, P, c1 - c0, storage=full[c0:c1])
        wg.vis_compress(view, tab, b, wtmp)
        st = wtmp.stats()
        real += st["updates"]
        total += st["updates"] + st["updates_saved"]
        counts.append(st["gridded"])
    del wtmp, view
    torch.cuda.empty_cache()
    launches = split_launches(counts)
    wlst = wg.WorkList(wl.rows * G, G, P, max_entries=max(sum(counts[i] for i in ls) for ls in launches) + 1024)

    def prepare(ls, table):
        wlst.clear()
        for gi in ls:
            c0, b = batches[gi]
            wg.vis_compress(grid, table, b, wlst, append=True, chan0=c0)

    # the gridder plan, autotuned on the appended batches of the first launch, and the gridder's
    # own time under it (summed over launches)
    grid.zero()
    prepare(launches[0], tab)
    seg, slots, fixed_r, _ = wg.grid_autotune(grid, tab, wlst, candidates=BATCH_PLANS, repeats=1)
    plan = (seg, slots, fixed_r)
    t_grid = 0.0
    for ls in launches:
        grid.zero()
        prepare(ls, tab)
        wlst.plan(tab, *plan)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        wg.grid_vis(grid, tab, wlst)
        e1.record(stream)
        torch.cuda.synchronize()
        t_grid += e0.elapsed_time(e1)

    def step():
        grid.zero()
        for ls in launches:
            prepare(ls, tab)
            wg.grid_vis(grid, tab, wlst)        # plans the appended entries, then one gridder launch
        wg.grid_correct(grid, tab, mode=wg.IMAGE_STOKES_I, out=img)

    step()                      # eager once: FFT plans and scratch are allocated outside the capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    n0 = wg.launch_count()
    with torch.cuda.graph(graph):
        step()
    captured = wg.launch_count() - n0
    clocks = ClockSampler(local_rank)
    clocks.start()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks.begin()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.end()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, world, dev)
    value = whole_job_rate(real, ms, world)
    del graph

    # the FP16 table at one polarisation: 4-byte samples halve the sample bytes the gridder
    # fetches per update (eager, the gridder's time under the same plan)
    variants = {}
    if not args.no_variants:
        tab16 = wg.ConvTable.build(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support,
                                   supports=wl.supports, store="f16")
        t16 = 0.0
        for ls in launches:
            for rep in range(2):                 # a warm-up launch, then the timed one
                grid.zero()
                prepare(ls, tab16)
                wlst.plan(tab16, *plan)
                v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                v0.record(stream)
                wg.grid_vis(grid, tab16, wlst)
                v1.record(stream)
                torch.cuda.synchronize()
            t16 += v0.elapsed_time(v1)
        variants["f16 table"] = {"gridder_ms": round(t16, 3), "real_gridder_G": round(real / (t16 * 1e-3) / 1e9, 3),
                                 "total_gridder_G": round(total / (t16 * 1e-3) / 1e9, 3)}
        del tab16
        torch.cuda.empty_cache()

    # end to end through the public API (eager calls): every step copies uvw and every group's
    # visibilities, weights and flags from pinned host memory into one set of device buffers
    # and reads the Stokes-I images back.  The buffers are released once the groups are
    # prepared, so the next step's copies run on a copy stream while this step's gridder runs;
    # the images are read back on the copy stream while the next step prepares.
    e2e = None
    if args.e2e_steps > 0:
        h_uvw = torch.empty(uvw_d.shape, dtype=uvw_d.dtype, pin_memory=True)
        h_uvw.copy_(uvw_d)
        h_vis = [torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for v in wl.vis]
        h_flag = [torch.empty(f.shape, dtype=f.dtype, pin_memory=True) for f in wl.flag]
        for hv, hf, v, f in zip(h_vis, h_flag, wl.vis, wl.flag):
            hv.copy_(v)
            hf.copy_(f)
        h_w = torch.empty(wl.weight[0].shape, dtype=torch.float32, pin_memory=True)
        h_w.copy_(wl.weight[0])
        # the device-resident inputs of the graph-timed steps are released for the copies' buffers
        del batches
        wl.vis.clear()
        wl.flag.clear()
        torch.cuda.empty_cache()
        h_img = torch.empty(img.shape, dtype=img.dtype, pin_memory=True)
        u_d = torch.empty_like(uvw_d)
        ins = [(torch.empty(hv.shape, dtype=hv.dtype, device=dev), torch.empty(h_w.shape, dtype=h_w.dtype, device=dev),
                torch.empty(hf.shape, dtype=hf.dtype, device=dev)) for hv, hf in zip(h_vis, h_flag)]
        cstream = torch.cuda.Stream()
        copied, released, imaged, read = (torch.cuda.Event() for _ in range(4))
        h2d = h_uvw.numel() * 8 + sum(hv.numel() * 8 + hf.numel() + h_w.numel() * 4 for hv, hf in zip(h_vis, h_flag))
        d2h = img.numel() * 4

        def issue_copies():
            with torch.cuda.stream(cstream):
                cstream.wait_event(released)
                u_d.copy_(h_uvw, non_blocking=True)
                for (v, w_, f_), hv, hf in zip(ins, h_vis, h_flag):
                    v.copy_(hv, non_blocking=True)
                    w_.copy_(h_w, non_blocking=True)
                    f_.copy_(hf, non_blocking=True)
                copied.record(cstream)

        def e2e_steps(n):
            released.record(stream)
            read.record(stream)
            issue_copies()
            for k in range(n):
                stream.wait_event(copied)
                grid.zero()
                for ls in launches:
                    wlst.clear()
                    for gi in ls:
                        v, w_, f_ = ins[gi]
                        wg.vis_compress(grid, tab, wg.VisBatch(u_d, freqs[gi], v, w_, f_), wlst, append=True,
                                        chan0=c0s[gi])
                    if ls is launches[-1]:
                        released.record(stream)
                        if k + 1 < n:
                            issue_copies()
                    wg.grid_vis(grid, tab, wlst)
                stream.wait_event(read)          # the previous step's images have been read back
                wg.grid_correct(grid, tab, mode=wg.IMAGE_STOKES_I, out=img)
                imaged.record(stream)
                with torch.cuda.stream(cstream):
                    cstream.wait_event(imaged)
                    h_img.copy_(img, non_blocking=True)
                    read.record(cstream)
            stream.wait_event(read)

        e2e_steps(1)
        torch.cuda.synchronize()
        barrier(world)
        x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        x0.record(stream)
        e2e_steps(args.e2e_steps)
        x1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = max_over_ranks(x0.elapsed_time(x1) / args.e2e_steps, world, dev)
        e2e = {"value": round(whole_job_rate(real, ms_e2e, world), 3), "unit": UNIT,
               "total_rate_G": round(whole_job_rate(total, ms_e2e, world), 3), "ms_per_step": round(ms_e2e, 3),
               "steps": args.e2e_steps, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "pipelining": "one set of device input buffers, released after the groups are prepared: the next "
                             "step's copies run on a copy stream under this step's gridder, and the images are read "
                             "back on it under the next step's preparation; eager calls (no graph)"}
        del h_uvw, h_vis, h_flag, h_w, h_img, u_d, ins
        torch.cuda.synchronize()
    peaks, src = _peaks()
    props = torch.cuda.get_device_properties(local_rank)
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
    achieved = 8.0 * real / (t_grid * 1e-3) / 1e12
    line = {
        "metric": "gridding/degridding G grid-point updates/s and % roofline at stated grid error",
        "value": round(value, 3),
        "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "%s: %s%s" % (args.workload, WORKLOADS[args.workload],
                                              "" if args.n_chan is None and args.n_times is None else
                                              " (slice: %s channels from %d, %s steps)" % (args.n_chan, args.chan0, args.n_times)),
                   "records_per_step": wl.rows * C, "input_bytes": int(in_bytes),
                   "l2": "inputs larger than L2 (no flush needed)", "chan_group": G,
                   "gridder_launches_per_step": len(launches), "entries_per_launch": [sum(counts[i] for i in ls) for ls in launches],
                   "plan_seg_len_slots_fixed_r": list(plan), "parallelism": "replicas" if world > 1 else "1 GPU"},
        "rates": {"real_step_G": round(value, 3),
                  "total_step_G": round(whole_job_rate(total, ms, world), 3),
                  "real_gridder_G": round(real / (t_grid * 1e-3) / 1e9, 3),
                  "total_gridder_G": round(total / (t_grid * 1e-3) / 1e9, 3),
                  "gridder_ms": round(t_grid, 3), "updates_real": real, "updates_total": total},
        "roofline": {"kernel": "k_grid (one persistent launch over all %d channels)" % C if len(launches) == 1
                               else "k_grid (sum over %d launches)" % len(launches),
                     "bound": "alu", "achieved": round(achieved, 3),
                     "peak": round(peak_tflops, 2), "unit": "TFLOP/s",
                     "frac": round(achieved / peak_tflops, 4),
                     "peak_source": "FP32 FMA pipe: %d SMs x 128 lanes x 2 flops x %.0f MHz (%s sm_max_mhz)"
                                    % (props.multi_processor_count, sm_mhz, src),
                     "traffic": None},
        "ceilings": measured_ceilings(real / (t_grid * 1e-3), P),
        "e2e": e2e,
        "variants": variants,
        "gpu_launches": int(captured * args.steps),
        "graph": {"captured_launches_per_step": int(captured), "replays": args.steps},
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        ot = oracle_table_parallel(wl)
        line["cpu_baseline"] = cpu_sample(args.workload, *CPU_SAMPLE[args.workload], ot=ot)
        errs = batch_grid_error(dev, plan, ot, stores=("f32",) + (("f16",) if variants else ()))
        line["grid_error"] = errs["f32"]
        if "f16" in errs:
            variants["f16 table"]["grid_error"] = errs["f16"]
    return line


def _sky(C, P, N, seed):
    """Seeded sky image [C][P][N][N]: point sources in the parallel hands plus a Gaussian blob."""
    import numpy as np
    rng = np.random.default_rng(seed)
    img = np.zeros((C, P, N, N), np.float32)
    for _ in range(8):
        y, x = rng.integers(N // 4, 3 * N // 4, 2)
        img[:, [0, P - 1], y, x] += rng.uniform(0.1, 1.0)
    yy, xx = np.mgrid[0:N, 0:N]
    img[:, 0] += 0.3 * np.exp(-((xx - 0.55 * N) ** 2 + (yy - 0.45 * N) ** 2) / (N / 16.0) ** 2)
    return img


def run_autograd(args, rank, world, local_rank):
    """Differentiation: one step = forward (degridding of the sky), chi^2, backward (adjoint
    gridding), all through the autograd Function."""
    import torch

    import paper_1403_4209_gb300 as wg
    import synth

    torch.cuda.set_device(local_rank)
    dev = "cuda:%d" % local_rank
    wl = synth.make(args.workload, device=dev, n_chan=args.n_chan, n_times=args.n_times, chan0=args.chan0)
    tab = wg.ConvTable.build(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    uvw_d = torch.as_tensor(wl.uvw, device=dev)
    freq_d = torch.as_tensor(wl.freq, device=dev)
    sm = wg.SkyModel(tab, uvw_d, freq_d, wl.weight, wl.flag, wl.n_grid, wl.du)
    x = torch.as_tensor(_sky(wl.n_chan, wl.n_pol, wl.n_grid, 77), device=dev).requires_grad_(True)
    v_obs = wl.vis
    stream = torch.cuda.current_stream()

    def step():
        x.grad = None
        loss = (sm(x) - v_obs).abs().pow(2).sum()
        loss.backward()
        return loss

    clocks = ClockSampler(local_rank)
    clocks.start()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st_f = sm.wl_fwd.stats()
    st_a = sm.wl_adj.stats()
    barrier(world)
    torch.cuda.synchronize()
    clocks.begin()
    n0 = wg.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = wg.launch_count() - n0
    clocks.end()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, world, dev)
    # kernel times of the forward and backward halves
    f0, f1, b1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    x.grad = None
    f0.record(stream)
    pred = sm(x)
    f1.record(stream)
    loss = (pred - v_obs).abs().pow(2).sum()
    b0 = torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    loss.backward()
    b1.record(stream)
    torch.cuda.synchronize()
    t_fwd, t_bwd = f0.elapsed_time(f1), b0.elapsed_time(b1)
    tot_f = st_f["updates"] + st_f["updates_saved"]
    tot_a = st_a["updates"] + st_a["updates_saved"]
    value = whole_job_rate(st_f["updates"] + st_a["updates"], ms, world)
    line = {
        "metric": "gridding/degridding G grid-point updates/s and % roofline at stated grid error",
        "value": round(value, 3),
        "unit": "G grid-point updates/s (real rate: forward degridding + backward gridding, whole step)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "%s: %s" % (args.workload, WORKLOADS[args.workload]),
                   "records_per_step": wl.rows * wl.n_chan, "l2": "inputs larger than L2 (no flush needed)",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "rates": {"forward_ms": round(t_fwd, 3), "backward_ms": round(t_bwd, 3),
                  "total_step_G": round(whole_job_rate(tot_f + tot_a, ms, world), 3),
                  "forward_total_G": round(tot_f / (t_fwd * 1e-3) / 1e9, 3),
                  "backward_total_G": round(tot_a / (t_bwd * 1e-3) / 1e9, 3),
                  "updates_total_forward": tot_f, "updates_total_backward": tot_a,
                  "updates_real_forward": st_f["updates"], "updates_real_backward": st_a["updates"]},
        "roofline": None,
        "e2e": None,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_sample_autograd(args.workload, *CPU_SAMPLE[args.workload])
    return line


def cpu_sample_autograd(workload, n_chan, n_times):
    """The FP64 oracle's chi^2 and gradient (forward model and adjoint) on a bounded sample."""
    import numpy as np

    import oracle
    import synth
    from oracle import model

    wl = synth.make(workload, n_chan=n_chan, n_times=n_times)
    ot = oracle.build_table(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    img = _sky(wl.n_chan, wl.n_pol, wl.n_grid, 77).astype(np.float64)
    t0 = time.perf_counter()
    pl = oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, ot, flag=wl.flag.numpy())
    model.chi2_grad(pl, ot, img, wl.vis.numpy(), wl.taper_support)
    dt = time.perf_counter() - t0
    upd = 2 * int(np.sum(pl.S[pl.griddable].astype(np.int64) ** 2)) * wl.n_pol
    return {"value": round(upd / dt / 1e9, 4), "unit": "G grid-point updates/s (total rate)", "cores": 1,
            "kind": "oracle", "seconds": round(dt, 2),
            "sample": "%s geometry, %d channel x %d time steps x %d baselines (%d records), FP64 oracle: "
                      "placement, forward model and adjoint (chi^2 gradient), single thread" % (
                          workload, n_chan, n_times, wl.n_baselines, wl.rows * wl.n_chan)}


def _oracle_setup(workload, chans, n_times, ot=None):
    """Inputs (one channel each) and the oracle's table for the CPU sample (untimed)."""
    import oracle
    import synth
    base, _ = SYNTH_NAME.get(workload, (workload, {}))
    sets = [synth.make(base, n_chan=1, chan0=c, n_times=n_times) for c in chans]
    wl = sets[0]
    if ot is not None:
        return sets, ot
    if WSTACK.get(workload):
        from oracle.wstack import stacking_table
        K = WSTACK[workload]
        ot = stacking_table(wl.du, K, wl.w_max, wl.oversample, wl.taper_support, supports=[WSTACK_SUPPORT] * K)
    else:
        ot = oracle.build_table(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    return sets, ot


def _oracle_run(workload, wl, ot):
    """The FP64 oracle (placement, compression, gridding) on a workload slice; returns (real
    updates, total updates, start, end) on the host's monotonic clock."""
    import numpy as np

    import oracle
    from oracle.grid import compress
    vis, w, f = wl.vis.numpy(), wl.weight.numpy(), wl.flag.numpy()
    inter = INTERLEAVE.get(workload, False)
    t0 = time.perf_counter()
    pl = oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, ot, flag=f)
    if WSTACK.get(workload):
        from oracle.wstack import grid_stacked
        g, c = oracle.classify(pl)
        grid_stacked(pl, ot, vis, w, f, wl.n_grid)
    elif COMPRESS[workload] and inter:
        g, c, *_ = compress(pl, vis, w, f, interleave=True)
        oracle.grid_compressed(pl, ot, vis, w, f, wl.n_grid, interleave=True)
    elif COMPRESS[workload]:
        g, c = oracle.classify(pl)
        oracle.grid_compressed(pl, ot, vis, w, f, wl.n_grid)
    else:
        g, c = pl.griddable, np.zeros_like(pl.griddable)
        oracle.grid_plain(pl, ot, vis, w, f, wl.n_grid)
    t1 = time.perf_counter()
    st = oracle.stats(pl, g, c)
    return st["updates"] * wl.n_pol, (st["updates"] + st["updates_saved"]) * wl.n_pol, t0, t1


def _oracle_proc(workload, chans, n_times, start, q):
    """One worker of the all-core CPU baseline: set up its channels, wait for the others, run."""
    import threading
    sets, ot = _oracle_setup(workload, chans, n_times)
    try:
        start.wait(timeout=600)
    except threading.BrokenBarrierError:
        pass
    for wl in sets:
        q.put(_oracle_run(workload, wl, ot) + (wl.n_baselines, wl.rows))


def cpu_sample(workload, n_chan, n_times, procs=1, ot=None):
    """The FP64 oracle on a bounded sample of the same geometry: n_chan channels x n_times steps.
    procs > 1 spreads the channels over worker processes (spawned, so no CUDA state is
    inherited) that start their timed sections together; the all-core rate is all updates over
    the span of the timed sections, the single-core rate the mean over channels."""
    if procs <= 1 and INTERLEAVE.get(workload, False):
        import oracle
        import synth
        wl = synth.make(workload, n_chan=n_chan, n_times=n_times)
        ot = oracle.build_table(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
        upd, tot, t0, t1 = _oracle_run(workload, wl, ot)
        return {"value": round(upd / (t1 - t0) / 1e9, 4), "unit": UNIT,
                "total_rate_G": round(tot / (t1 - t0) / 1e9, 4),
                "cores": 1, "kind": "oracle", "seconds": round(t1 - t0, 2),
                "sample": "%s geometry, %d interleaved channels x %d time steps x %d baselines (%d records), FP64 "
                          "oracle: placement + compression + gridding onto one grid, single thread" % (
                              workload, n_chan, n_times, wl.n_baselines, wl.rows * wl.n_chan)}
    if procs <= 1:
        sets, ot = _oracle_setup(workload, range(n_chan), n_times, ot)
        res = [_oracle_run(workload, wl, ot) for wl in sets]
        upd = sum(r[0] for r in res)
        tot = sum(r[1] for r in res)
        dt = sum(r[3] - r[2] for r in res)
        return {"value": round(upd / dt / 1e9, 4), "unit": UNIT, "total_rate_G": round(tot / dt / 1e9, 4),
                "cores": 1, "kind": "oracle", "seconds": round(dt, 2),
                "sample": "%s geometry, %d channels x %d time steps x %d baselines (%d records), FP64 oracle: "
                          "placement + compression + gridding, single thread" % (
                              workload, n_chan, n_times, sets[0].n_baselines, sets[0].rows * n_chan)}
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    start = ctx.Barrier(procs)
    ps = [ctx.Process(target=_oracle_proc, args=(workload, list(range(i, n_chan, procs)), n_times, start, q))
          for i in range(procs)]
    for p in ps:
        p.start()
    res = [q.get(timeout=900) for _ in range(n_chan)]
    for p in ps:
        p.join(60)
    upd = sum(r[0] for r in res)
    tot = sum(r[1] for r in res)
    span = max(r[3] for r in res) - min(r[2] for r in res)
    single = sum(r[0] / (r[3] - r[2]) for r in res) / len(res)
    return {"value": round(upd / span / 1e9, 4), "unit": UNIT, "total_rate_G": round(tot / span / 1e9, 4),
            "cores": procs, "kind": "oracle", "seconds": round(span, 2), "single_core_value": round(single / 1e9, 4),
            "sample": "%s geometry, %d channels x %d time steps x %d baselines (%d records), FP64 oracle: "
                      "placement + compression + gridding, channels spread over %d processes" % (
                          workload, n_chan, n_times, res[0][4], sum(r[5] for r in res), procs)}


def grid_error_sample(workload, dev, plan, interleave=False, stack_k=0):
    """Grid error of the CUDA path against the FP64 oracle (plain definition, eq. "gridding") on a
    seeded slice of the workload (300 baselines x 24 steps x 2 channels), with the bench's plan."""
    import numpy as np
    import torch

    import oracle
    import paper_1403_4209_gb300 as wg
    import synth
    base, kw = SYNTH_NAME.get(workload, (workload, {}))
    wl = synth.make(base, n_chan=2, n_times=24, n_baselines=300)
    if stack_k:
        sup = [WSTACK_SUPPORT] * stack_k
        tab = wg.ConvTable.build(wl.du, stack_k, wl.w_max, wl.oversample, wl.taper_support, supports=sup, stacking=True)
    else:
        tab = wg.ConvTable.build(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    g = wg.Grid(wl.n_grid, wl.du, wl.n_pol, 1 if interleave else wl.n_chan * max(1, stack_k), device=dev)
    b = wg.VisBatch(torch.as_tensor(wl.uvw, device=dev), torch.as_tensor(wl.freq, device=dev), wl.vis.to(dev),
                    wl.weight.to(dev), wl.flag.to(dev))
    w = wg.WorkList(wl.rows * wl.n_chan, wl.n_chan, wl.n_pol)
    wg.vis_compress(g, tab, b, w, compress=COMPRESS[workload], interleave=interleave, wstack=bool(stack_k))
    w.plan(tab, *plan)
    wg.grid_vis(g, tab, w)
    got = g.data.cpu().numpy()
    f = wl.flag.numpy()
    if stack_k:
        from oracle.wstack import grid_stacked, stacking_table
        ot = stacking_table(wl.du, stack_k, wl.w_max, wl.oversample, wl.taper_support, supports=sup)
        pl = oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, ot, flag=f)
        ref = grid_stacked(pl, ot, wl.vis.numpy(), wl.weight.numpy(), f, wl.n_grid)
    else:
        ot = oracle.build_table(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
        pl = oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, ot, flag=f)
        ref = oracle.grid_plain(pl, ot, wl.vis.numpy(), wl.weight.numpy(), f, wl.n_grid, interleave=interleave)
    return {"rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "max_abs_over_max": float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))),
            "reference": "FP64 oracle, plain gridding definition",
            "sample": "%s geometry, 300 baselines x 24 steps x 2 channels (%d records)" % (workload,
                                                                                      wl.rows * wl.n_chan)}


def variant_errors(dev, plan):
    """Grid error against the FP64 oracle (the plain definition, eq. "gridding"; the whole
    channel through the oracle's compressed gridding, equal to it up to rounding) of the plain
    FP32 path and of every precision variant, on two inputs of the wproj_2k geometry: the
    300-baseline x 24-step x 2-channel slice, and the whole of channel 15 (180 MHz: 2016
    baselines x 3600 steps, 7.26 M records), where a pixel takes many flushes.  The gridder
    runs under the benchmark's plan."""
    import numpy as np
    import torch

    import oracle
    import paper_1403_4209_gb300 as wg
    import synth
    out = {}
    ot = None
    for cname, kw in (("slice", dict(n_chan=2, n_times=24, n_baselines=300)), ("channel15", dict(n_chan=1, chan0=15))):
        wl = synth.make("wproj_2k", **kw)
        if ot is None:      # slices share the full workload's cell size and w_max, hence the table
            ot = oracle.build_table(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support,
                                    supports=wl.supports)
        vis, w, f = wl.vis.numpy(), wl.weight.numpy(), wl.flag.numpy()
        pl = oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, ot, flag=f)
        ref = (oracle.grid_plain if cname == "slice" else oracle.grid_compressed)(pl, ot, vis, w, f, wl.n_grid)
        nref, mref = np.linalg.norm(ref), np.max(np.abs(ref))
        uvw_d, freq_d = torch.as_tensor(wl.uvw, device=dev), torch.as_tensor(wl.freq, device=dev)
        vis_d = wl.vis.to(dev)
        vis_h, scale_h = synth.to_half_vis(vis_d)
        b32 = wg.VisBatch(uvw_d, freq_d, vis_d, wl.weight.to(dev), wl.flag.to(dev))
        b16 = wg.VisBatch(uvw_d, freq_d, vis_h, b32.weight, b32.flag, vis_scale=scale_h)
        wlst = wg.WorkList(wl.rows * wl.n_chan, wl.n_chan, wl.n_pol)
        for name, store, half, comp in (("fp32", "f32", False, False),) + VARIANTS:
            tab = wg.ConvTable.build(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support,
                                     supports=wl.supports, store=store)
            g = wg.Grid(wl.n_grid, wl.du, wl.n_pol, wl.n_chan, device=dev, compensated=comp)
            wg.vis_compress(g, tab, b16 if half else b32, wlst)
            wlst.plan(tab, *plan)
            wg.grid_vis(g, tab, wlst)
            d = g.data.cpu().numpy() - ref
            out.setdefault(name, {})[cname] = {"rel_l2": float(np.linalg.norm(d) / nref),
                                               "max_abs_over_max": float(np.max(np.abs(d)) / mref)}
            del tab, g, d
        del wlst, b32, b16, vis_d, vis_h
        torch.cuda.empty_cache()
    samples = {"slice": "wproj_2k geometry, 300 baselines x 24 steps x 2 channels (14400 records)",
               "channel15": "wproj_2k geometry, channel 15 (180 MHz), 2016 baselines x 3600 steps (7257600 records)"}
    for v in out.values():
        v["reference"] = "FP64 oracle"
        v["samples"] = samples
    return out


def run_reference(args):
    """The oracle as the reference arm: each step one bounded sample on the host cores."""
    import numpy as np

    import oracle
    import synth

    n_chan, n_times = REF_SAMPLE[args.workload]
    wl = synth.make(args.workload, n_chan=n_chan, n_times=n_times)
    ot = oracle.build_table(wl.du, wl.n_wplanes, wl.w_max, wl.oversample, wl.taper_support, supports=wl.supports)
    vis, w, f = wl.vis.numpy(), wl.weight.numpy(), wl.flag.numpy()

    def step():
        pl = oracle.place(wl.uvw, wl.freq, wl.du, wl.n_grid, ot, flag=f)
        if COMPRESS[args.workload]:
            g, c = oracle.classify(pl)
            oracle.grid_compressed(pl, ot, vis, w, f, wl.n_grid)
        else:
            g, c = pl.griddable, np.zeros_like(pl.griddable)
            oracle.grid_plain(pl, ot, vis, w, f, wl.n_grid)
        return oracle.stats(pl, g, c)

    for _ in range(args.warmup):
        st = step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = step()
    dt = (time.perf_counter() - t0) / args.steps
    real = st["updates"] * wl.n_pol
    total = (st["updates"] + st["updates_saved"]) * wl.n_pol
    value = real / dt / 1e9
    unit = UNIT
    sample = ("%s geometry, %d channels x %d time steps x %d baselines (%d records) per step" %
              (args.workload, n_chan, n_times, wl.n_baselines, wl.rows * wl.n_chan))
    return {
        "impl": "reference",
        "metric": "gridding/degridding G grid-point updates/s and % roofline at stated grid error",
        "value": round(value, 4), "unit": unit, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "%s: %s%s" % (args.workload, WORKLOADS[args.workload],
                                              "" if args.n_chan is None and args.n_times is None else
                                              " (slice: %s channels, %s steps)" % (args.n_chan, args.n_times)), "sample": sample},
        "rates": {"total_rate_G": round(total / dt / 1e9, 4), "updates_real": real, "updates_total": total},
        "cpu_baseline": {"value": round(value, 4), "unit": unit, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# The thesis's experiment batches 2-4 (Sec. 5.4, tables "batch2" / "batch3" / "batch4"):
# the real gridding rate per convolution-function size as the uv cell (grid side N at a fixed
# uv extent), the oversampling factor and the number of polarisations vary.  One plane (K = 1)
# with a prescribed support S isolates the support; the geometry is the 2-channel slice of the
# w-projection workload (2016 baselines x 3600 steps, 120 and 124 MHz).
SWEEPS = {
    "support": [dict(N=2048, beta=8, pols=4, S=S) for S in (7, 15, 31, 63, 127)],
    "oversample": [dict(N=2048, beta=b, pols=4, S=S) for S in (15, 63) for b in (2, 4, 8)],
    "grid": [dict(N=n, beta=8, pols=4, S=S) for S in (15, 63) for n in (1024, 2048, 4096)],
    "pols": [dict(N=2048, beta=8, pols=p, S=S) for S in (15, 63) for p in (1, 2, 4)],
}
SWEEP_POLS = {1: [0], 2: [0, 3], 4: [0, 1, 2, 3]}


def run_sweep(args):
    """One JSON line per sweep point: records, compression, plan, real and total gridder rates
    (CUDA events over 5 launches after grid_autotune), preparation time."""
    import dataclasses

    import torch

    import paper_1403_4209_gb300 as wg
    import synth
    dev = "cuda"
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    base = synth.make("wproj_2k", device=dev, n_chan=2, n_times=args.n_times)
    du0 = base.du                     # cell at N = 2048: the uv extent stays fixed as N varies
    uvw_d, freq_d = torch.as_tensor(base.uvw, device=dev), torch.as_tensor(base.freq, device=dev)
    names = list(SWEEPS) if args.sweep == "all" else [args.sweep]
    for name in names:
        for pt in SWEEPS[name]:
            N, beta, S, pols = pt["N"], pt["beta"], pt["S"], SWEEP_POLS[pt["pols"]]
            du = du0 * 2048 / N
            wl = dataclasses.replace(base, vis=base.vis[..., pols].contiguous(),
                                     weight=base.weight[..., pols].contiguous(),
                                     flag=base.flag[..., pols].contiguous())
            P = len(pols)
            tab = wg.ConvTable.build(du, 1, wl.w_max, beta, wl.taper_support, supports=[S])
            g = wg.Grid(N, du, P, wl.n_chan, device=dev)
            batch = wg.VisBatch(uvw_d, freq_d, wl.vis, wl.weight, wl.flag)
            wlst = wg.WorkList(wl.rows * wl.n_chan, wl.n_chan, P)
            wg.vis_compress(g, tab, batch, wlst)
            plan = wg.grid_autotune(g, tab, wlst, repeats=2)
            st = wlst.stats()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            for _ in range(2):
                wg.vis_compress(g, tab, batch, wlst)
            ev[0].record(stream)
            for _ in range(5):
                wg.vis_compress(g, tab, batch, wlst)
            ev[1].record(stream)
            ev[2].record(stream)
            for _ in range(5):
                wg.grid_vis(g, tab, wlst)
            ev[3].record(stream)
            torch.cuda.synchronize()
            t_prep, t_grid = ev[0].elapsed_time(ev[1]) / 5, ev[2].elapsed_time(ev[3]) / 5
            real, total = st["updates"], st["updates"] + st["updates_saved"]
            print(json.dumps({
                "sweep": name, "N": N, "beta": beta, "n_pol": P, "support": S, "du": round(du, 4),
                "records": st["records"], "griddable": st["griddable"], "gridded": st["gridded"],
                "compression_ratio_records": round(st["compressed"] / max(1, st["gridded"]), 3),
                "plan_seg_len_slots_fixed_r": list(plan[:3]), "prep_ms": round(t_prep, 3),
                "gridder_ms": round(t_grid, 3), "real_gridder_G": round(real / (t_grid * 1e-3) / 1e9, 1),
                "total_gridder_G": round(total / (t_grid * 1e-3) / 1e9, 1),
                "record_rate_real_M": round(st["gridded"] / (t_grid * 1e-3) / 1e6, 1)}), flush=True)
            del tab, g, wlst, wl, batch
            torch.cuda.empty_cache()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="wproj_2k")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip timing the precision variants")
    ap.add_argument("--n-chan", type=int, default=None, help="run a slice: first n channels (profiling)")
    ap.add_argument("--n-times", type=int, default=None, help="run a slice: n time steps (profiling)")
    ap.add_argument("--chan0", type=int, default=0, help="first channel of an --n-chan slice")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched 8192^2 section that the default wproj_2k run adds under 'batch_8k'")
    ap.add_argument("--batch-steps", type=int, default=5,
                    help="timed steps of that section (at most --steps; about 2.4 s each)")
    ap.add_argument("--e2e-steps", type=int, default=3,
                    help="end-to-end steps of the batched workload (0: skip)")
    ap.add_argument("--sweep", choices=sorted(SWEEPS) + ["all"], default=None,
                    help="instead of the benchmark line, the rate sweeps of the thesis's experiment batches 2-4 "
                         "(one JSON line per point)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if args.sweep:
        if rank == 0:
            run_sweep(args)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    runner = run_batch if args.workload in CHAN_GROUP else run_autograd if args.workload == "degrid_1k" else run_ours
    line = runner(args, rank, world, local_rank)
    if args.workload == "wproj_2k" and args.n_chan is None and args.n_times is None and not args.no_batch:
        # the batched configuration (8192^2 grids, 64 channels, 64 planes, one graph per step) at
        # full size, reported beside the headline under its own key with its own measurements
        import copy

        import torch
        torch.cuda.empty_cache()
        b_args = copy.copy(args)
        b_args.workload = "batch_8k"
        b_args.steps = max(1, min(args.steps, args.batch_steps))
        b_args.warmup = 3
        line["batch_8k"] = run_batch(b_args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
