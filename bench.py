"""Benchmark of the B300 3DGS rasterizer; prints ONE JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload 1m|6m|fwdbwd|small|batch|multi] [--no-legs]

A step is one pass of the whole hot path over one frame: preprocess, depth sort of
the surviving splats, emission of their tile copies, tile sort, and compositing of
one view (fwdbwd: plus the adjoint). The default workload is 1M Gaussians with SH
degree 3 seen from a 32-camera orbit at 1920x1080 (steps cycle through the views);
the attribute arrays (236 MB) exceed the 126 MB L2, so no flush is needed between
steps.

value      frame time in ms (whole job: max-over-ranks time / frames of all ranks),
           inputs resident in HBM, CUDA events on the launching stream.
e2e        the same through the C ABI with host buffers: every step copies the
           scene from pinned host memory, renders, and reads the image back.
roofline   the stage that dominates the frame: against the measured HBM copy
           bandwidth (MEASURED_PEAKS.json) for the HBM-bound stages, algorithmic
           bytes per launch over the CUDA-event launch time; against the FP32 issue
           rate for the compositor (15 instructions per (pixel, splat) test).
hbm_stages every HBM-bound stage (preprocess, depth sort, emission, tile sort)
           against the copy peak.
legs       (default run) the metric's other legs, each with its own clocks: the 6M
           dynamic frame, the 500k forward + backward step, and the 128-image batch
           (fused pipeline, autotuned) against the 8-lane graph and 128 sequential
           renders.
cpu_baseline  the FP64 oracle on the host cores, a bounded sample of the same
           frame (a stride of its tiles), scaled to a frame.
--impl reference   times that oracle alone as the reference arm.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

# per-stage times of vis_profile_end (8 stages), by sort mode
STAGES_DF = ["clear", "preprocess", "depth_sort", "emission", "tile_counts", "tile_sort_passes", "ranges",
             "composite"]
STAGES_TD = ["clear", "preprocess", "duplicate", "sort_histogram", "none", "sort_passes", "ranges", "composite"]
METRIC = "1080p frame ms at 1M/6M Gaussians SH3; fwd+bwd ms; sort keys/s vs HBM peak"


def _peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return dict(hbm_gbs=float(d["hbm_gbs"]), source="measured", sm_max_mhz=float(d.get("sm_max_mhz", 2032.0)))
    return dict(hbm_gbs=6400.0, source="fallback", sm_max_mhz=2032.0)


def replica_first_view(rank, steps):
    """Replicas shard by view: replica `rank` renders `steps` consecutive views starting at
    rank * steps (modulo the orbit), so no two replicas render the same frames."""
    return rank * steps


def max_over_ranks(value, dist, device):
    """The job's time: the slowest replica's (all_reduce MAX; the value itself on one rank)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------------------------------
# workloads
# ------------------------------------------------------------------------------------------

def load_workload(name):
    from paper_2512_08478_b300 import synth
    if name == "1m":
        sc, cams = synth.workload_1m(views=32)
        desc = dict(workload="1M Gaussians SH3, 64-component mixture, 32-view orbit r=15, 1920x1080, 50 deg vfov",
                    n_gaussians=1_000_000, sh_degree=3, width=1920, height=1080, views=32, tile=16)
        return sc, cams, desc, None
    if name == "6m":
        sc, extras, cams = synth.workload_dynamic()
        desc = dict(workload="6M Gaussians SH3, dynamic (moving means, pulsing opacity), 1920x1080 slow orbit",
                    n_gaussians=6_000_000, sh_degree=3, width=1920, height=1080, frames=120, tile=16)
        return sc, cams, desc, extras
    if name == "fwdbwd":
        sc, target, cams = synth.workload_fwdbwd()
        desc = dict(workload="500k Gaussians SH3, 800x800, L2 loss vs perturbed target, forward + backward",
                    n_gaussians=500_000, sh_degree=3, width=800, height=800, views=len(cams), tile=16)
        return sc, cams, desc, target
    if name == "small":
        sc, cams = synth.workload_small()
        desc = dict(workload="10k Gaussians SH0, 256x256, one camera", n_gaussians=10_000, sh_degree=0,
                    width=256, height=256, views=1, tile=16)
        return sc, cams, desc, None
    raise SystemExit(f"unknown workload {name}")


# ------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        # The garbage collector is held off while the timed work is enqueued: a full
        # collection in the middle of the launch loop stalls the host for milliseconds, long
        # enough for the GPU to run out of queued frames.
        gc.collect()
        self.gc_was_enabled = gc.isenabled()
        gc.disable()
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None
        time.sleep(0.25)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.gc_was_enabled:
            gc.enable()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["unavailable"], samples=0)
        return dict(sm_mhz=float(np.median(sm)), sm_max_mhz=mx, reasons=sorted(reasons), samples=len(sm))


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------

def _kernel_sha(files):
    """Hash of the kernel sources a committed ncu capture was taken on."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        h.update((ROOT / "paper_2512_08478_b300" / "csrc" / f).read_bytes())
    return h.hexdigest()[:16]


def _committed_traffic(stage, M, n, tile=None):
    """DRAM bytes (read + write) per launch of the stage's kernel from a committed ncu capture
    (profiles/traffic.json), scaled to this launch by keys or Gaussians; None if absent, if
    the kernel's source changed since the capture (the entry records the sources' hash), or
    if the capture's tile size (when it records one) is not this launch's."""
    p = ROOT / "profiles" / "traffic.json"
    if not p.exists():
        return None
    d = json.loads(p.read_text()).get(stage)
    if not d or "sources" not in d or d.get("source_sha") != _kernel_sha(d["sources"]):
        return None
    if tile is not None and d.get("tile") is not None and int(d["tile"]) != int(tile):
        return None
    if "bytes_per_key" in d:
        return int(d["bytes_per_key"] * M)
    if "bytes_per_gaussian" in d:
        return int(d["bytes_per_gaussian"] * n)
    return None


def measure(args, workload, with_e2e=True, with_cpu=True, dist=None):
    """Times `args.steps` frames of `workload` (after `args.warmup`), with per-stage times from
    a second pass, the dominant stage's roofline and the HBM-bound stages against the copy
    peak; returns the result line (dict)."""
    import torch
    import paper_2512_08478_b300 as vis

    world, rank, local = _dist()
    sc_np, cams, desc, extra = load_workload(workload)
    W, H = desc["width"], desc["height"]
    sc = vis.Scene.from_numpy(sc_np)
    n = sc.n
    cap = 16 * n + (1 << 20)
    sort_mode = args.sort_mode if args.sort_mode is not None else vis.make_opts().sort_mode
    ppt = args.ppt if args.ppt is not None else 1
    tile = args.tile if args.tile is not None else 16

    def make(t, p):
        return vis.make_opts(sort_mode=sort_mode, tile=t, pixels_per_thread=p, digit_bits=args.digit_bits)
    opts = make(tile, ppt)
    # sized for the smallest tile tried: its layout is the largest (per-tile arrays), so every
    # candidate fits
    ws = vis.Workspace(n, W, H, key_capacity=cap, opts=make(min(16, tile), ppt))
    rgb = torch.empty((3, H, W), device="cuda")
    alpha = torch.empty((H, W), device="cuda")
    stream = torch.cuda.current_stream()
    fwdbwd = workload == "fwdbwd"
    if fwdbwd:
        tgt = vis.Scene.from_numpy(extra)
        tgt_rgb = torch.empty_like(rgb)
        tgt_a = torch.empty_like(alpha)
        grads = {k: torch.empty_like(sc.tensors[k]) for k in vis.FIELDS}
        d_alpha = torch.zeros_like(alpha)
        d_rgb = torch.empty_like(rgb)
    cam_objs = [vis.make_camera(c) for c in cams]
    view0 = replica_first_view(rank, args.steps)
    # pre-packed fp16 scene (Algorithm 1's pre-pack, once, outside the timing); a packed frame
    # is static (a dynamic scene would have to be re-packed every frame)
    packed = bool(args.packed) and not fwdbwd
    if packed:
        psc = vis.PackedScene.pack(sc)
        torch.cuda.synchronize()
    handle = psc.handle if packed else sc.handle
    # depth-buffer-aware compositing against a wall of constant view depth (section 3.4's depth
    # test without writes; the buffer stands in for an opaque mesh's depth prepass)
    dbuf = (torch.full((H, W), float(args.depth_plane), dtype=torch.float32, device="cuda")
            if args.depth_plane is not None else None)
    dynamic = workload == "6m" and not packed
    if dynamic:
        # the scene keeps frame 0; a frame renders with the update applied inside the
        # preprocess (vis_render_dynamic); the update kernel on its own is timed in the stage
        # pass, into scratch arrays
        dyn = {k: torch.from_numpy(v).cuda() for k, v in extra.items()}
        means0 = sc.tensors["means"]
        logits0 = sc.tensors["opacity_logits"]
        upd_means, upd_logits = torch.empty_like(means0), torch.empty_like(logits0)
        n_frames = desc["frames"]
        upd_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]

    def frame(i, timed=False):
        k = (view0 + i) % len(cam_objs)
        c = cam_objs[k]
        if dynamic:
            if timed:
                upd_ev[i][0].record(stream)
                vis.vis_dynamic_update(means0, dyn["velocity"], logits0, dyn["amp"], dyn["freq"], dyn["phase"],
                                       k / n_frames, upd_means, upd_logits)
                upd_ev[i][1].record(stream)
            vis.vis_render_dynamic(handle, dyn["velocity"], dyn["amp"], dyn["freq"], dyn["phase"], k / n_frames, c,
                                   W, H, (0.0, 0.0, 0.0), rgb, alpha, ws.buf, opts)
        else:
            vis.vis_render(handle, c, W, H, (0.0, 0.0, 0.0), rgb, alpha, ws.buf, opts, depth=dbuf)
        if fwdbwd:
            torch.sub(rgb, tgt_rgb, out=d_rgb)
            d_rgb.mul_(2.0 / rgb.numel())
            vis.vis_render_backward(sc.handle, c, W, H, (0.0, 0.0, 0.0), d_rgb, d_alpha, ws.buf, grads, opts)

    if fwdbwd:   # target image of view 0 (fixed), rendered once outside the timing
        vis.vis_render(tgt.handle, cam_objs[0], W, H, (0.0, 0.0, 0.0), tgt_rgb, tgt_a, ws.buf, opts)
        vis.vis_check(ws.buf)

    tuned_ms = None
    if args.ppt is None or args.tile is None:
        # tile size (16 or 32 px) and compositor block shape (1 or 2 pixels per thread; the
        # image depends on neither): the fastest on this workload's first views, outside the
        # timed region
        from paper_2512_08478_b300 import tuning
        cands = [(t, p) for t in ((16, 32) if args.tile is None else (tile,))
                 for p in ((1, 2) if args.ppt is None else (ppt,))]

        def tune_step(c, _i=[0]):
            nonlocal opts
            opts = make(*c)
            frame(_i[0] % 4)
            _i[0] += 1
        (tile, ppt), tuned_ms = tuning.pick_fastest(cands, tune_step, reps=4, warmup=2)
        opts = make(tile, ppt)
    ws.opts = opts   # the layout of the chosen options (the buffer holds every candidate's)
    desc["tile"] = tile
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        # the warm-up runs after the sampler's start-up pause, right before the timed frames,
        # so that the GPU is not left idle just before the first of them
        for i in range(args.warmup):
            frame(i)
        vis.vis_check(ws.buf)
        # ---- device-timed region ----
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for i in range(args.steps):
            frame(i)
        ev1.record(stream)
        torch.cuda.synchronize()
    vis.vis_check(ws.buf)
    t_ms = ev0.elapsed_time(ev1)
    clk_summary = clk.summary()
    # per-stage times: the same frames once more with events between the stages, outside the
    # timed region (an event between two kernels stops the second one's early launch)
    import ctypes as C
    vis.lib().vis_profile_begin()
    for i in range(args.steps):
        frame(i, timed=True)
    torch.cuda.synchronize()
    stage = (C.c_double * 8)()
    ns, nr, npass = C.c_int(), C.c_int(), C.c_int()
    vis._ok(vis.lib().vis_profile_end(stage, 8, C.byref(ns), C.byref(nr), C.byref(npass)))
    vis.vis_check(ws.buf)
    t_ms = max_over_ranks(t_ms, dist, "cuda")
    frames_total = args.steps * world
    value = t_ms / frames_total
    names = STAGES_DF if sort_mode == 1 else STAGES_TD
    stage_ms = {names[k]: stage[k] / max(nr.value, 1) for k in range(8)}
    update_ms = (sum(a.elapsed_time(b) for a, b in upd_ev) / args.steps) if dynamic else None
    lay = ws.layout()
    fused = lay.key_bytes == 2
    passes = npass.value

    # keys per frame averaged over the views used, and the preprocess traffic each view needs:
    # every Gaussian is read for the depth and cull test, only those in front (z > near,
    # opacity >= alpha_min) for the covariance, and only the survivors (tiles touched > 0) for
    # their SH coefficients and splat record
    mlist, nvis, nok = [], [], []
    opac = torch.sigmoid(sc.tensors["opacity_logits"].reshape(-1))
    a_min = float(np.float32(vis.make_opts().alpha_min))
    for i in range(min(args.steps, len(cam_objs))):
        k = (view0 + i) % len(cam_objs)
        if dynamic:   # the frame's own attributes
            vis.vis_dynamic_update(means0, dyn["velocity"], logits0, dyn["amp"], dyn["freq"], dyn["phase"],
                                   k / n_frames, upd_means, upd_logits)
            opac = torch.sigmoid(upd_logits.reshape(-1))
        frame(i)
        mlist.append(vis.vis_check(ws.buf))
        touched = ws.buf[lay.off_touched: lay.off_touched + 4 * n].view(torch.int32)
        zview = ws.buf[lay.off_depth: lay.off_depth + 4 * n].view(torch.float32)
        nvis.append(int((touched != 0).sum()))
        nok.append(int(((zview > cams[k].near) & (opac >= a_min)).sum()))
    M = float(np.mean(mlist))
    n_vis, n_ok = float(np.mean(nvis)), float(np.mean(nok))

    # ---- algorithmic bytes of the HBM-bound stages ----
    peaks = _peaks()
    sh_k = (desc["sh_degree"] + 1) ** 2
    # means + logit read, depth + rect + count written: 40 B; quaternion + log-scales: 28 B for the
    # Gaussians in front; SH (12 B per coefficient) read and 48 B record written per survivor
    bytes_pre = n * 40 + n_ok * 28 + n_vis * (12 * sh_k + 48)
    pre_note = "40 B per Gaussian + 28 B per Gaussian in front + SH and 48 B record per survivor"
    if packed:   # fp16 planes: pos 8 B for all, cov 12 B in front, colour words per survivor
        bytes_pre = n * 32 + n_ok * 12 + n_vis * (vis.vis_packed_size(1, desc["sh_degree"])[2] + 48)
    if dynamic:   # the update's arrays: velocity, amplitude, frequency and phase per Gaussian
        bytes_pre += n * 24
        pre_note = "64 B per Gaussian (with the update's 24) + 28 B per Gaussian in front + SH and 48 B record " \
                   "per survivor"
    hbm = {"preprocess": (bytes_pre, stage_ms["preprocess"], pre_note)}
    if sort_mode == 1:
        dp = {8: 4, 10: 4, 11: 3}[args.digit_bits]   # digit passes of the depth sort
        # compaction: count + depth read per Gaussian, (depth, index) written per survivor; the
        # depth histogram reads 4 B per survivor; each pass reads and writes 8 B per survivor
        hbm["depth_sort"] = (8 * n + 8 * n_vis + 4 * n_vis + 16 * dp * n_vis, stage_ms["depth_sort"],
                             f"compaction 8 B per Gaussian + 8 B per survivor, histogram 4 B and {dp} passes of "
                             "16 B per survivor")
        # touch sums and emission: index + count, then index + footprint per survivor; 2 B tile id
        # + 4 B index written per copy
        hbm["emission"] = (28 * n_vis + 6 * M, stage_ms["emission"],
                           "28 B per survivor (indices, counts, footprints) + 6 B per copy written")
        # per-tile counts: footprint read per Gaussian; passes: 2 + 4 B read and written per copy,
        # the last writes the 4 B value only
        tile_b = 16 * n + M * (12 * passes - 2) if fused else 16 * n + M * 16 * passes
        hbm["tile_sort"] = (tile_b, stage_ms["tile_counts"] + stage_ms["tile_sort_passes"],
                            "16 B footprint per Gaussian + 12 B per copy per pass (the last pass 10 B)")
        sort_ms = stage_ms["depth_sort"] + stage_ms["emission"] + stage_ms["tile_counts"] + \
            stage_ms["tile_sort_passes"] + stage_ms["ranges"]
    else:
        hbm["sort"] = (M * (8 + 24 * passes), stage_ms["sort_histogram"] + stage_ms["sort_passes"],
                       "8 B key read by the histogram + 24 B per key per pass")
        sort_ms = stage_ms["duplicate"] + stage_ms["sort_histogram"] + stage_ms["sort_passes"] + stage_ms["ranges"]
    hbm_stages = {}
    for k, (b, ms, note) in hbm.items():
        a = b / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        hbm_stages[k] = dict(bytes=int(b), ms=round(ms, 4), achieved_gbs=round(a, 1),
                             frac=round(a / peaks["hbm_gbs"], 4), bytes_model=note)

    # ---- roofline of the dominant stage ----
    cands = ["preprocess", "composite"] + (["tile_sort", "depth_sort"] if sort_mode == 1 else ["sort"])
    dom_ms = {c: (hbm_stages[c]["ms"] if c in hbm_stages else stage_ms[c]) for c in cands}
    dom = max(cands, key=lambda c: dom_ms[c])
    if dom == "composite":
        # the compositor is bound by FP32 issue (~15 FP32 instructions per (pixel, splat) test,
        # one ex2 per composited pair): count its tests on the first view (one extra render with
        # statistics, outside the timed region), as the one-pixel compositor (8 x 4 warp blocks)
        # counts them whichever block shape is timed, so that the algorithmic count does not
        # depend on the implementation's choice
        st_opts = vis.make_opts(sort_mode=sort_mode, tile=tile, pixels_per_thread=1,
                                digit_bits=args.digit_bits, collect_stats=1)
        vis.vis_render(handle, cam_objs[view0 % len(cam_objs)], W, H, (0.0, 0.0, 0.0), rgb, alpha, ws.buf,
                       st_opts, depth=dbuf)
        vis.vis_check(ws.buf)
        ctrl = vis.read_ctrl(ws.buf)
        inst = 15.0 * ctrl["pair_tests"]
        mhz = clk_summary.get("sm_mhz") or peaks.get("sm_max_mhz", 2032.0)
        n_sm = torch.cuda.get_device_properties(local).multi_processor_count
        peak_t = n_sm * 128 * mhz * 1e6 / 1e12
        ach_t = inst / (stage_ms["composite"] * 1e-3) / 1e12
        hb = M * (4 + 48) + W * H * (16 + 8)
        roof = dict(kernel="composite", bound="alu", achieved=round(ach_t, 3), peak=round(peak_t, 2),
                    unit="T FP32 lane-instructions/s", frac=round(ach_t / peak_t, 4),
                    traffic=_committed_traffic("composite", M, n, tile),
                    peak_source=f"{n_sm} SMs x 128 FP32 lanes x {mhz:.0f} MHz (sampled clock)",
                    algorithmic_instructions_per_launch=int(inst), pair_tests=ctrl["pair_tests"],
                    hits=ctrl["hits"], launch_ms=round(stage_ms["composite"], 4),
                    instruction_model="15 FP32 instructions per (pixel, splat) test (offset, two whitened "
                                      "projections, squared norm, threshold, and the composited pair's share); "
                                      "tests as the one-pixel compositor's 8x4 warp blocks count them",
                    hbm_view=dict(achieved=round(hb / (stage_ms["composite"] * 1e-3) / 1e9, 1),
                                  peak=peaks["hbm_gbs"], unit="GB/s",
                                  frac=round(hb / (stage_ms["composite"] * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)))
    else:
        h = hbm_stages[dom]
        roof = dict(kernel=dom, bound="hbm", achieved=h["achieved_gbs"], peak=peaks["hbm_gbs"], unit="GB/s",
                    frac=h["frac"],
                    traffic=_committed_traffic("preprocess_dynamic" if (dom == "preprocess" and dynamic) else dom, M, n,
                                               tile),
                    peak_source=peaks["source"],
                    algorithmic_bytes_per_launch=h["bytes"], launch_ms=h["ms"], bytes_model=h["bytes_model"])

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if with_e2e:
        e2e = (run_e2e(args, vis, torch, sc_np, cam_objs, W, H, cap, dist, opts) if not (packed or dbuf is not None)
               else dict(value=None, note="not measured for a pre-packed scene or a depth buffer"))

    # kernels per frame: preprocess, (mode 1) block-sum scan, compaction, depth histogram,
    # depth passes, touch sums, scan, emission, tile counts, tile scan, tile look-back clear,
    # tile passes / (mode 0) scan, duplication, histogram, passes, ranges; the compositor; the
    # backward adds the compositor's adjoint and the preprocess adjoint; a depth buffer its
    # per-tile maximum
    depth_passes = {8: 4, 10: 4, 11: 3}[args.digit_bits]
    fused_tiles = lay.key_bytes == 2
    launches = {0: 6 + passes, 1: 8 + depth_passes + passes + (3 if fused_tiles else 2)}[sort_mode] + \
        (2 if fwdbwd else 0) + (1 if dbuf is not None else 0)
    line = dict(metric=METRIC, value=round(value, 4), unit="ms/frame", n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=round(t_ms / args.steps, 4), higher_is_better=False,
                scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(desc, sort_mode=sort_mode, packed=packed, pixels_per_thread=ppt,
                            tuned_ms=({f"tile{k[0]}_ppt{k[1]}": round(v, 4) for k, v in tuned_ms.items()}
                                      if tuned_ms else None),
                            digit_bits=args.digit_bits,
                            depth_buffer=(f"wall at view depth {args.depth_plane}" if dbuf is not None else None),
                            l2="inputs larger than L2 (attributes exceed 126 MB); no flush",
                            parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
                clocks=clk_summary, e2e=e2e, gpu_launches=int(args.steps * launches),
                roofline=roof, hbm_stages=hbm_stages,
                stage_ms={k: round(v, 4) for k, v in stage_ms.items() if k != "none"},
                keys_per_frame=int(M), visible_per_frame=int(n_vis), sort_passes=passes,
                dynamic_update_ms=(round(update_ms, 4) if update_ms is not None else None),
                sort_ms=round(sort_ms, 4), sort_keys_per_s=round(M / sort_ms * 1e3, 1),
                gaussians_per_s=round(n / value * 1e3, 1))
    if fwdbwd:
        fwd = sum(stage_ms.values())
        line["forward_ms"] = round(fwd, 4)
        line["backward_ms"] = round(value - fwd, 4)
    if rank == 0 and world == 1 and with_cpu and not packed:
        line["cpu_baseline"] = cpu_baseline(workload, sc_np, cams, desc, budget_s=args.cpu_seconds)
    return line


def run_ours(args):
    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    line = measure(args, args.workload, with_e2e=True, with_cpu=not args.no_cpu, dist=dist)
    if args.workload == "1m" and world == 1 and not args.no_legs and not args.packed and args.depth_plane is None:
        # the metric's other legs, each timed on its own: the 6M dynamic frame, the 500k
        # fwd+bwd step and the 128-image batch
        line["legs"] = legs(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def legs(args):
    import copy
    import torch
    out = {}
    keep = ("value", "unit", "steps", "warmup", "clocks", "config", "stage_ms", "hbm_stages", "roofline",
            "keys_per_frame", "visible_per_frame", "sort_ms", "sort_keys_per_s", "gaussians_per_s",
            "dynamic_update_ms", "forward_ms", "backward_ms", "gpu_launches")
    for name, wl in (("dynamic_6m", "6m"), ("fwdbwd_500k", "fwdbwd")):
        a = copy.copy(args)
        a.steps = min(args.steps, 20)
        r = measure(a, wl, with_e2e=False, with_cpu=False)
        out[name] = {k: r[k] for k in keep if k in r and r[k] is not None}
        torch.cuda.empty_cache()
    out["batch_128"] = batch_leg(args)
    torch.cuda.empty_cache()
    return out


def batch_leg(args):
    """16 assets x 8 cameras = 128 images, the autotuned fused pipeline (one graph-captured
    vis_render_batch) against the 8-lane graph and against 128 sequential vis_render calls of
    the plain path, all with the tuned options (images compared bit for bit)."""
    import torch
    import paper_2512_08478_b300 as vis
    from paper_2512_08478_b300 import synth, tuning
    world, rank, local = _dist()
    scenes_np, cams, cam_scene = synth.workload_batch()
    scenes = [vis.Scene.from_numpy(s) for s in scenes_np]
    tried = []
    if args.no_autotune:
        opts_d, tuned_ms = dict(tile=16, digit_bits=8, pixels_per_thread=1), None
    else:
        opts_d, tuned_ms = tuning.autotune(scenes, cams, cam_scene, cache=None, log=tried.append)
    opts = vis.make_opts(**opts_d)
    stream = torch.cuda.current_stream()
    steps = max(3, min(args.steps, 10))

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            for _ in range(max(3, args.warmup // 2)):   # warm-up right before the timed steps
                fn()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, clk.summary()

    fused = vis.Batch(scenes, cams, cam_scene, lanes=0, opts=opts)
    fused.render()
    t_fused, clk_fused = timed(fused.launch)
    keys = fused.check()
    ref = [(r.clone(), a.clone()) for r, a in zip(fused.rgb, fused.alpha)]
    del fused
    torch.cuda.empty_cache()
    lanes = vis.Batch(scenes, cams, cam_scene, lanes=8, opts=opts)
    lanes.render()
    t_lanes, clk_lanes = timed(lanes.launch)
    lanes.check()
    same_lanes = all(torch.equal(lanes.rgb[i], ref[i][0]) and torch.equal(lanes.alpha[i], ref[i][1])
                     for i in range(len(cams)))
    del lanes
    torch.cuda.empty_cache()
    nmax = max(s.n for s in scenes)
    ws = vis.Workspace(nmax, max(int(c.W) for c in cams), max(int(c.H) for c in cams),
                       key_capacity=16 * nmax + (1 << 20), opts=opts)
    outs = [(torch.empty((3, c.H, c.W), device="cuda"), torch.empty((c.H, c.W), device="cuda")) for c in cams]
    cam_objs = [vis.make_camera(c) for c in cams]

    def sequential():
        for i, c in enumerate(cam_objs):
            vis.vis_render(scenes[cam_scene[i]].handle, c, cams[i].W, cams[i].H, (0.0, 0.0, 0.0), outs[i][0],
                           outs[i][1], ws.buf, opts)

    t_seq, clk_seq = timed(sequential)
    vis.vis_check(ws.buf)
    same_seq = all(torch.equal(outs[i][0], ref[i][0]) and torch.equal(outs[i][1], ref[i][1]) for i in range(len(cams)))
    n_g = sum(scenes[a].n for a in cam_scene)
    return dict(value=round(t_fused, 4), unit="ms/batch", steps=steps,
                config=dict(workload="16 assets (N log-uniform 2e4..2e6, SH 0..3) x 8 orbit cameras at "
                                     "{512^2, 1280x720, 1920x1080}", images=len(cams),
                            gaussians=[s.n for s in scenes], opts=opts_d, pipeline="fused (lanes = 0)"),
                lanes8_ms=round(t_lanes, 4), sequential_ms=round(t_seq, 4),
                speedup_vs_sequential=round(t_seq / t_fused, 3), speedup_vs_lanes=round(t_lanes / t_fused, 3),
                images_identical_to_sequential=bool(same_seq), images_identical_to_lanes=bool(same_lanes),
                keys_largest_group=int(keys), gaussian_views_per_s=round(n_g / t_fused * 1e3, 1),
                autotune=dict(best_ms=tuned_ms, tried=tried), clocks=clk_fused,
                clocks_lanes=clk_lanes, clocks_sequential=clk_seq)


def run_batch(args):
    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    leg = batch_leg(args)
    line = dict(metric="ms per 128-image heterogeneous batch (16 assets x 8 cameras)", n_gpus=1, warmup=args.warmup,
                ms_per_step=leg["value"], higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f32",
                data="synthetic", **leg)
    print(json.dumps(line), flush=True)


def _merged_rigid(scenes_np, models):
    """One plain scene of the models' Gaussians under rigid + uniform-scale transforms
    (means A mu + b, log-scales + log s, rotations composed), SH zero-padded to the highest
    degree: the same splats drawn through the single-scene path."""
    from scipy.spatial.transform import Rotation
    deg = max(s["sh_degree"] for s in scenes_np)
    K = (deg + 1) ** 2
    parts = {k: [] for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    for sc, M in zip(scenes_np, models):
        A, b = M[:, :3].astype(np.float64), M[:, 3].astype(np.float64)
        s = float(np.cbrt(np.linalg.det(A)))
        q = sc["quats"].astype(np.float64)
        rot = Rotation.from_matrix(A / s) * Rotation.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], 1))
        xyzw = rot.as_quat()
        parts["means"].append(sc["means"] @ A.T + b)
        parts["log_scales"].append(sc["log_scales"] + math.log(s))
        parts["quats"].append(np.stack([xyzw[:, 3], xyzw[:, 0], xyzw[:, 1], xyzw[:, 2]], 1))
        parts["opacity_logits"].append(sc["opacity_logits"])
        sh = np.zeros((sc["means"].shape[0], K, 3), np.float32)
        sh[:, : sc["sh"].shape[1]] = sc["sh"]
        parts["sh"].append(sh)
    out = {k: np.ascontiguousarray(np.concatenate(v), np.float32) for k, v in parts.items()}
    out["sh_degree"] = deg
    return out


def run_multi(args):
    """Multi-asset frame: 4 models (1.8M Gaussians, SH 0..3) placed by rigid transforms,
    drawn into one 1080p image by vis_render_multi (per-model preprocess, one global sort
    and compositing); 8 views orbiting the group. Beside it: the same Gaussians merged into
    one plain scene (SH zero-padded to degree 3) through vis_render."""
    import ctypes as C
    import torch
    import paper_2512_08478_b300 as vis
    from paper_2512_08478_b300 import synth
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    scenes_np, models, cam0 = synth.workload_multi()
    W, H = cam0.W, cam0.H
    cams = [synth.look_at((14.0 * math.sin(2 * math.pi * k / 8), 3.0, 14.0 * math.cos(2 * math.pi * k / 8)),
                          (0, 0, 0), W, H, 50.0) for k in range(8)]
    cam_objs = [vis.make_camera(c) for c in cams]
    scenes = [vis.Scene.from_numpy(s) for s in scenes_np]
    handles = [s.handle for s in scenes]
    slots = vis.vis_multi_slots(handles)
    n_total = sum(s.n for s in scenes)
    opts = vis.make_opts()
    ws = vis.Workspace(slots, W, H, key_capacity=16 * slots + (1 << 20), opts=opts)
    merged = vis.Scene.from_numpy(_merged_rigid(scenes_np, models))
    wsm = vis.Workspace(merged.n, W, H, key_capacity=16 * merged.n + (1 << 20), opts=opts)
    rgb = torch.empty((3, H, W), device="cuda")
    alpha = torch.empty((H, W), device="cuda")
    stream = torch.cuda.current_stream()

    def multi(i):
        vis.vis_render_multi(handles, models, cam_objs[i % 8], W, H, (0.0, 0.0, 0.0), rgb, alpha, ws.buf, opts)

    def single(i):
        vis.vis_render(merged.handle, cam_objs[i % 8], W, H, (0.0, 0.0, 0.0), rgb, alpha, wsm.buf, opts)

    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    with ClockSampler(local) as clk:
        for i in range(args.warmup):   # warm-up right before the timed frames
            multi(i)
            single(i)
        keys = vis.vis_check(ws.buf)
        vis.vis_check(wsm.buf)
        torch.cuda.synchronize()
        e[0].record(stream)
        for i in range(args.steps):
            multi(i)
        e[1].record(stream)
        for i in range(args.steps):
            single(i)
        e[2].record(stream)
        torch.cuda.synchronize()
    vis.lib().vis_profile_begin()   # stage times from a separate pass (see run_ours)
    for i in range(args.steps):
        multi(i)
    torch.cuda.synchronize()
    stage = (C.c_double * 8)()
    ns, nr, npass = C.c_int(), C.c_int(), C.c_int()
    vis._ok(vis.lib().vis_profile_end(stage, 8, C.byref(ns), C.byref(nr), C.byref(npass)))
    vis.vis_check(ws.buf)
    vis.vis_check(wsm.buf)
    t_multi = e[0].elapsed_time(e[1]) / args.steps
    t_single = e[1].elapsed_time(e[2]) / args.steps
    stage_ms = {STAGES_DF[k]: round(stage[k] / max(nr.value, 1), 4) for k in range(8)}
    line = dict(metric="1080p multi-asset frame ms (4 models, one global sort)", value=round(t_multi, 4),
                unit="ms/frame", n_gpus=1, steps=args.steps, warmup=args.warmup, ms_per_step=round(t_multi, 4),
                higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload="4 mixture models (N log-uniform 1e5..1e6, SH 0..3) placed by rigid "
                                     "transforms on a ring, 8 orbit views r=14, 1920x1080, 50 deg vfov",
                            gaussians=[s.n for s in scenes], slots=slots, sh_degrees=[s.sh_degree for s in scenes],
                            l2="inputs larger than L2; no flush"),
                merged_scene_ms=round(t_single, 4),
                merged_note="the same Gaussians as one plain scene, SH zero-padded to degree 3",
                stage_ms=stage_ms, keys_per_frame=int(keys), gaussians_per_s=round(n_total / t_multi * 1e3, 1),
                # per frame: a preprocess per model, then the depth-first frame's kernels (scan,
                # compaction, histogram, four depth passes, touch sums, scan, emission, tile
                # counts, tile scan, tile look-back clear, tile passes, compositor)
                gpu_launches=int(args.steps * (len(scenes) + 10 + 4 + npass.value)), clocks=clk.summary())
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_e2e(args, vis, torch, sc_np, cam_objs, W, H, cap, dist, opts):
    """Every step: H2D of the scene from pinned memory, render, D2H of rgb + alpha; double
    buffered on three streams, so that frame i's upload overlaps frame i-1's render and
    read-back (the way a streaming renderer feeds the GPU)."""
    host = {k: torch.from_numpy(sc_np[k]).pin_memory() for k in vis.FIELDS}
    dev = [{k: torch.empty(host[k].shape, dtype=torch.float32, device="cuda") for k in vis.FIELDS} for _ in range(2)]
    scenes = [vis.Scene(**d, sh_degree=sc_np["sh_degree"]) for d in dev]
    ws = vis.Workspace(scenes[0].n, W, H, key_capacity=cap, opts=opts)
    rgb = [torch.empty((3, H, W), device="cuda") for _ in range(2)]
    alpha = [torch.empty((H, W), device="cuda") for _ in range(2)]
    out_rgb = [torch.empty((3, H, W)).pin_memory() for _ in range(2)]
    out_a = [torch.empty((H, W)).pin_memory() for _ in range(2)]
    h2d = sum(t.numel() * 4 for t in host.values())
    d2h = (out_rgb[0].numel() + out_a[0].numel()) * 4
    stream = torch.cuda.current_stream()
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    rendered = [torch.cuda.Event() for _ in range(2)]
    read = [torch.cuda.Event() for _ in range(2)]
    for b in range(2):
        rendered[b].record(stream)
        read[b].record(stream)

    def step(i):
        b = i & 1
        with torch.cuda.stream(up):            # scene buffer b is free once frame i-2 rendered
            up.wait_event(rendered[b])
            for k in vis.FIELDS:
                dev[b][k].copy_(host[k], non_blocking=True)
            copied[b].record(up)
        stream.wait_event(copied[b])
        stream.wait_event(read[b])             # image buffer b is free once frame i-2 was read
        vis.vis_render(scenes[b].handle, cam_objs[i % len(cam_objs)], W, H, (0.0, 0.0, 0.0), rgb[b], alpha[b],
                       ws.buf, opts)
        rendered[b].record(stream)
        with torch.cuda.stream(down):
            down.wait_event(rendered[b])
            out_rgb[b].copy_(rgb[b], non_blocking=True)
            out_a[b].copy_(alpha[b], non_blocking=True)
            read[b].record(down)

    for i in range(max(2, args.warmup)):
        step(i)
    torch.cuda.synchronize()
    vis.vis_check(ws.buf)
    steps = max(4, args.steps // 2)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    gc.collect()
    gc_was_enabled = gc.isenabled()
    gc.disable()   # no collection pause inside the timed steps (as in the device-timed regions)
    e0.record(stream)
    up.wait_event(e0)
    down.wait_event(e0)
    for i in range(steps):
        step(i)
    stream.wait_event(read[(steps - 1) & 1])
    stream.wait_event(read[steps & 1])
    e1.record(stream)
    torch.cuda.synchronize()
    if gc_was_enabled:
        gc.enable()
    vis.vis_check(ws.buf)
    t = e0.elapsed_time(e1)
    world = 1
    if dist:
        t = max_over_ranks(t, dist, "cuda")
        world = dist.get_world_size()
    return dict(value=round(t / (steps * world), 4), unit="ms/frame", h2d_bytes_per_step=int(h2d),
                d2h_bytes_per_step=int(d2h), steps=steps,
                overlap="double-buffered: frame i's upload overlaps frame i-1's render and read-back")


# ------------------------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ------------------------------------------------------------------------------------------

def _oracle_frame(oracle, sc_np, cam, stride):
    """Oracle preprocess of all Gaussians + composite of every `stride`-th tile;
    returns seconds scaled to one whole frame."""
    tiles_x, tiles_y = (cam.W + 15) // 16, (cam.H + 15) // 16
    mask = np.zeros(tiles_x * tiles_y, np.uint8)
    mask[::stride] = 1
    t0 = time.perf_counter()
    prep = oracle.preprocess(sc_np, cam)
    t1 = time.perf_counter()
    oracle.render_tiled(prep, cam.W, cam.H, tile_mask=mask)
    t2 = time.perf_counter()
    return (t1 - t0) + (t2 - t1) * (tiles_x * tiles_y) / mask.sum()


def _stride_for(workload):
    return {"1m": 8, "6m": 16, "fwdbwd": 8, "small": 1}.get(workload, 8)


def cpu_baseline(workload, sc_np, cams, desc, budget_s=20.0):
    import oracle
    stride = _stride_for(workload)
    frames, t_acc, t_start = 0, 0.0, time.perf_counter()
    while True:
        t_acc += _oracle_frame(oracle, sc_np, cams[frames % len(cams)], stride)
        frames += 1
        if time.perf_counter() - t_start > budget_s * 0.5 or frames >= 3:
            break
    return dict(value=round(t_acc / frames * 1e3, 1), unit="ms/frame", cores=oracle.num_threads(), kind="oracle",
                sample=f"{frames} view(s): FP64 preprocess of all {desc['n_gaussians']} Gaussians + composite of "
                       f"every {stride}th 16x16 tile, tile time scaled by {stride}")


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    oracle.build()
    sc_np, cams, desc, _ = load_workload(args.workload)
    stride = _stride_for(args.workload)
    for i in range(args.warmup):
        _oracle_frame(oracle, sc_np, cams[i % len(cams)], stride * 4)
    t0 = time.perf_counter()
    acc = 0.0
    for i in range(args.steps):
        acc += _oracle_frame(oracle, sc_np, cams[i % len(cams)], stride)
    wall = time.perf_counter() - t0
    value = acc / args.steps * 1e3
    cores = oracle.num_threads()
    sample = (f"per step: FP64 preprocess of all {desc['n_gaussians']} Gaussians + composite of every "
              f"{stride}th 16x16 tile, tile time scaled by {stride}")
    line = dict(impl="reference", metric=METRIC, value=round(value, 1), unit="ms/frame", n_gpus=world,
                steps=args.steps, warmup=args.warmup, ms_per_step=round(wall / args.steps * 1e3, 1),
                higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                # the workload's fields (the tile size is an implementation's choice: the sample
                # above names the oracle's own tiling)
                config={k: v for k, v in desc.items() if k != "tile"},
                cpu_baseline=dict(value=round(value, 1), unit="ms/frame", cores=cores,
                                                     kind="oracle", sample=sample),
                e2e=dict(value=round(value, 1), unit="ms/frame", h2d_bytes_per_step=0, d2h_bytes_per_step=0),
                ms_per_step_note="wall time of a sampled step; value scales the sampled tiles' time to the whole "
                                 "frame")
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=32)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="1m", choices=["1m", "6m", "fwdbwd", "small", "batch", "multi"])
    ap.add_argument("--no-autotune", action="store_true", help="batch workload: skip the autotuner")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-legs", action="store_true",
                    help="1m workload: skip the 6M, fwd+bwd and batch legs of the line")
    ap.add_argument("--sort-mode", type=int, default=None, choices=[0, 1],
                    help="0: one sort of 64-bit (tile, depth) keys; 1: depth sort then tile sort "
                         "(default: the library default)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--tile", type=int, default=None, choices=[8, 16, 32],
                    help="tile size in pixels (default: 16 or 32, the faster on the workload's first views)")
    ap.add_argument("--digit-bits", type=int, default=8, choices=[8, 10, 11],
                    help="radix digit width of the depth sort (and of 32-bit tile sorts)")
    ap.add_argument("--ppt", type=int, default=None, choices=[1, 2],
                    help="pixels per compositor thread (default: the faster on the workload's first views)")
    ap.add_argument("--depth-plane", type=float, default=None,
                    help="composite against a depth buffer holding this view depth everywhere")
    ap.add_argument("--packed", action="store_true",
                    help="render a pre-packed fp16 copy of the scene (packed once, outside the timing)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "multi":
        run_multi(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
