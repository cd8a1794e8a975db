"""Benchmark of the B300 3DGS rasterizer; prints ONE JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload 1m|6m|fwdbwd|small]

A step is one pass of the whole hot path over one frame: preprocess, key
duplication, radix sort, tile ranges and compositing of one view (fwdbwd: plus
the adjoint). The default workload is 1M Gaussians with SH degree 3 seen from a
32-camera orbit at 1920x1080 (steps cycle through the views); the attribute
arrays (236 MB) exceed the 126 MB L2, so no flush is needed between steps.

value      frame time in ms (whole job: max-over-ranks time / frames of all ranks),
           inputs resident in HBM, CUDA events on the launching stream.
e2e        the same through the C ABI with host buffers: every step copies the
           scene from pinned host memory, renders, and reads the image back.
roofline   the stage that dominates the frame, against the measured HBM copy
           bandwidth (MEASURED_PEAKS.json), algorithmic bytes per launch over the
           CUDA-event launch time.
cpu_baseline  the FP64 oracle on the host cores, a bounded sample of the same
           frame (a stride of its tiles), scaled to a frame.
--impl reference   times that oracle alone as the reference arm.
"""
from __future__ import annotations

import argparse
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

kDP = 4   # depth passes of sort_mode 1
METRIC = "1080p frame ms at 1M/6M Gaussians SH3; fwd+bwd ms; sort keys/s vs HBM peak"
STAGES = ["clear", "preprocess", "duplicate", "sort_histogram", "sort_passes", "ranges", "composite"]
# sort_mode 1 (depth first): "duplicate" = compaction + depth sort + emission in depth order,
# "sort_histogram"/"sort_passes" = the stable sort by tile id of 4-byte keys
STAGES_DF = ["clear", "preprocess", "depth_sort_and_emit", "tile_sort_histogram", "tile_sort_passes", "ranges",
             "composite"]
# sort_mode 1 with the counts-first tile sort (16-bit tile keys): stage 2 = compaction, depth sort
# and emission in depth order; stage 3 = per-tile counts (histograms, ranges); stage 4 = the tile
# passes; no ranges stage
STAGES_FUSED = ["clear", "preprocess", "depth_sort_and_emit", "tile_counts", "tile_sort_passes", "ranges",
                "composite"]


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

def run_ours(args):
    import torch
    import paper_2512_08478_b300 as vis

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    sc_np, cams, desc, extra = load_workload(args.workload)
    desc["tile"] = args.tile
    W, H = desc["width"], desc["height"]
    sc = vis.Scene.from_numpy(sc_np)
    n = sc.n
    cap = 16 * n + (1 << 20)
    if args.sort_mode is None:
        args.sort_mode = vis.make_opts().sort_mode
    opts = vis.make_opts(sort_mode=args.sort_mode, tile=args.tile, pixels_per_thread=args.ppt)
    ws = vis.Workspace(n, W, H, key_capacity=cap, opts=opts)
    rgb = torch.empty((3, H, W), device="cuda")
    alpha = torch.empty((H, W), device="cuda")
    stream = torch.cuda.current_stream()
    fwdbwd = args.workload == "fwdbwd"
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
    dynamic = args.workload == "6m" and not packed
    if dynamic:
        dyn = {k: torch.from_numpy(v).cuda() for k, v in extra.items()}
        means0 = sc.tensors["means"].clone()
        logits0 = sc.tensors["opacity_logits"].clone()
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
                                   k / n_frames, sc.tensors["means"], sc.tensors["opacity_logits"])
            if timed:
                upd_ev[i][1].record(stream)
        vis.vis_render(handle, c, W, H, (0.0, 0.0, 0.0), rgb, alpha, ws.buf, opts, depth=dbuf)
        if fwdbwd:
            torch.sub(rgb, tgt_rgb, out=d_rgb)
            d_rgb.mul_(2.0 / rgb.numel())
            vis.vis_render_backward(sc.handle, c, W, H, (0.0, 0.0, 0.0), d_rgb, d_alpha, ws.buf, grads, opts)

    if fwdbwd:   # target image of view 0 (fixed), rendered once outside the timing
        vis.vis_render(tgt.handle, cam_objs[0], W, H, (0.0, 0.0, 0.0), tgt_rgb, tgt_a, ws.buf, opts)
        vis.vis_check(ws.buf)

    for i in range(args.warmup):
        frame(i)
    num_keys = vis.vis_check(ws.buf)

    # ---- device-timed region ----
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    keys_seen = []
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for i in range(args.steps):
            frame(i)
        ev1.record(stream)
        torch.cuda.synchronize()
    vis.vis_check(ws.buf)
    t_ms = ev0.elapsed_time(ev1)
    # per-stage times: the same frames once more with events between the stages, outside the
    # timed region (an event between two kernels stops the second one's early launch)
    import ctypes as C
    vis.lib().vis_profile_begin()
    for i in range(args.steps):
        frame(i, timed=True)
    torch.cuda.synchronize()
    stage = (C.c_double * 7)()
    ns, nr, npass = C.c_int(), C.c_int(), C.c_int()
    vis._ok(vis.lib().vis_profile_end(stage, 7, C.byref(ns), C.byref(nr), C.byref(npass)))
    vis.vis_check(ws.buf)
    t_ms = max_over_ranks(t_ms, dist, "cuda")
    frames_total = args.steps * world
    value = t_ms / frames_total
    stage_ms = {STAGES[k]: stage[k] / max(nr.value, 1) for k in range(7)}
    update_ms = (sum(a.elapsed_time(b) for a, b in upd_ev) / args.steps) if dynamic else None
    fused = ws.layout().key_bytes == 2
    names = STAGES_FUSED if fused else {0: STAGES, 1: STAGES_DF}[args.sort_mode]
    passes = npass.value

    # keys per frame averaged over the views used
    # and the preprocess traffic each view requires: every Gaussian is read for the depth and
    # cull test, only those in front (z > near, opacity >= alpha_min) for the covariance, and
    # only the survivors (tiles touched > 0) for their SH coefficients and splat record
    mlist, nvis, nok = [], [], []
    lay = ws.layout()
    opac = torch.sigmoid(sc.tensors["opacity_logits"].reshape(-1))
    a_min = float(np.float32(vis.make_opts().alpha_min))
    for i in range(min(args.steps, len(cam_objs))):
        k = (view0 + i) % len(cam_objs)
        vis.vis_render(handle, cam_objs[k], W, H, (0.0, 0.0, 0.0), rgb, alpha, ws.buf, opts, depth=dbuf)
        mlist.append(vis.vis_check(ws.buf))
        touched = ws.buf[lay.off_touched: lay.off_touched + 4 * n].view(torch.int32)
        zview = ws.buf[lay.off_depth: lay.off_depth + 4 * n].view(torch.float32)
        nvis.append(int((touched != 0).sum()))
        nok.append(int(((zview > cams[k].near) & (opac >= a_min)).sum()))
    M = float(np.mean(mlist))
    n_vis, n_ok = float(np.mean(nvis)), float(np.mean(nok))

    # ---- roofline of the dominant stage ----
    peaks = _peaks()
    cands = ("preprocess", "sort_passes", "composite")
    dom = max(cands, key=lambda s: stage_ms[s])
    sh_k = (desc["sh_degree"] + 1) ** 2
    # means + logit read, depth + rect + count written: 32 B each; quaternion + log-scales: 28 B
    # for the Gaussians in front; SH (12 B per coefficient) read and 48 B record written per survivor
    bytes_pre = n * 40 + n_ok * 28 + n_vis * (12 * sh_k + 48)
    if packed:   # fp16 planes: pos 8 B for all, cov 12 B in front, colour words per survivor
        bytes_pre = n * 32 + n_ok * 12 + n_vis * (vis.vis_packed_size(1, desc["sh_degree"])[2] + 48)
    # bytes the tile sort must move: per digit pass key + value read and written; with the fused
    # binning the first pass reads 16 B per surviving splat (first copy, index, rect) and writes a
    # 2 B key + 4 B value per copy, the last reads those and writes the 4 B value
    # 16-bit keys: every pass reads 2 + 4 B per copy and writes 2 + 4 B, the last only the 4 B value
    tile_bytes = (M * (12 * passes - 2)) if fused else M * (24.0 if args.sort_mode == 0 else 16.0) * passes
    if dom == "sort_passes" and fused:
        launch_ms = stage_ms["sort_passes"] / passes
        algo = tile_bytes / passes
        unit_note = ("mean over the tile passes: 2 B key + 4 B value read and written per copy, "
                     "the last pass writes the value only")
    elif dom == "sort_passes":
        launch_ms = stage_ms["sort_passes"] / passes
        per_key = 24.0 if args.sort_mode == 0 else 16.0
        algo = per_key * M
        unit_note = (f"{int(per_key)} B per key per digit pass ({'8' if args.sort_mode == 0 else '4'} B key + "
                     f"4 B value, read and written)")
    elif dom == "preprocess":
        launch_ms = stage_ms["preprocess"]
        algo = float(bytes_pre)
        unit_note = ("40 B per Gaussian (means, logit, depth, rect, count) + 28 B per Gaussian in front "
                     "(quaternion, log-scales) + SH and 48 B record per surviving splat")
        if packed:
            unit_note = ("32 B per Gaussian (fp16 mean + opacity, depth, rect, count) + 12 B fp16 covariance per "
                         "Gaussian in front + fp16 SH words and 48 B record per surviving splat")
    else:
        launch_ms = stage_ms[dom]
        algo = M * (4 + 48) + W * H * (16 + 8)
        unit_note = "per key: value + gathered 48 B record; per pixel: rgb, alpha, T, last written"
    achieved = algo / (launch_ms * 1e-3) / 1e9
    traffic = _committed_traffic(dom, M, n)
    roof = dict(kernel=names[STAGES.index(dom)], bound="hbm", achieved=round(achieved, 1), peak=peaks["hbm_gbs"],
                unit="GB/s", frac=round(achieved / peaks["hbm_gbs"], 4), traffic=traffic,
                peak_source=peaks["source"], algorithmic_bytes_per_launch=int(algo), launch_ms=round(launch_ms, 4),
                bytes_model=unit_note)
    clk_summary = clk.summary()
    if dom == "composite":
        # the compositor is bound by FP32 issue, not HBM: count its (pixel, splat) tests and hits
        # on the first view (one extra render with statistics, outside the timed region)
        st_opts = vis.make_opts(sort_mode=args.sort_mode, tile=args.tile, pixels_per_thread=args.ppt, collect_stats=1)
        vis.vis_render(handle, cam_objs[view0 % len(cam_objs)], W, H, (0.0, 0.0, 0.0), rgb, alpha, ws.buf,
                       st_opts)
        vis.vis_check(ws.buf)
        ctrl = vis.read_ctrl(ws.buf)
        flops = 11.0 * ctrl["pair_tests"] + 13.0 * ctrl["hits"]
        mhz = clk_summary.get("sm_mhz") or _peaks().get("sm_max_mhz", 2032.0)
        n_sm = torch.cuda.get_device_properties(0).multi_processor_count
        peak_tf = n_sm * 128 * 2 * mhz * 1e6 / 1e12
        ach_tf = flops / (stage_ms["composite"] * 1e-3) / 1e12
        roof = dict(kernel="composite", bound="alu", achieved=round(ach_tf, 2), peak=round(peak_tf, 1),
                    unit="TFLOP/s", frac=round(ach_tf / peak_tf, 4), traffic=traffic,
                    peak_source=f"FP32 FMA rate: {n_sm} SMs x 128 lanes x 2 flop x {mhz:.0f} MHz (sampled clock)",
                    algorithmic_flops_per_launch=int(flops), pair_tests=ctrl["pair_tests"], hits=ctrl["hits"],
                    launch_ms=round(stage_ms["composite"], 4),
                    flop_model="11 flop per (pixel, splat) test (offset, two projections, squared norm), "
                               "13 per composited pair (alpha, transmittance, 3 colour FMAs)",
                    hbm_view=dict(achieved=round(achieved, 1), peak=peaks["hbm_gbs"], unit="GB/s",
                                  frac=round(achieved / peaks["hbm_gbs"], 4)))
        # the compositor is issue-bound: its warp instructions (per test, from the committed ncu
        # capture, times this launch's live test count) over the launch time, against one
        # instruction per clock from each of the 4 schedulers of every SM
        tj = ROOT / "profiles" / "traffic.json"
        ipt = json.loads(tj.read_text()).get("composite", {}).get("warp_inst_per_test") if tj.exists() else None
        if ipt:
            inst = ipt * ctrl["pair_tests"]
            ach_i = inst / (stage_ms["composite"] * 1e-3) / 1e9
            peak_i = n_sm * 4 * mhz * 1e6 / 1e9
            roof["issue_view"] = dict(achieved=round(ach_i, 1), peak=round(peak_i, 1), unit="G warp-inst/s",
                                      frac=round(ach_i / peak_i, 4), warp_inst_per_launch=int(inst),
                                      source="profiles/traffic.json warp_inst_per_test x live pair tests")

    # every HBM-bound stage against the copy peak (the spec bar is >= 60% for preprocess and sort)
    hbm_stages = {"preprocess": dict(bytes=int(bytes_pre), ms=round(stage_ms["preprocess"], 4),
                                     achieved_gbs=round(bytes_pre / (stage_ms["preprocess"] * 1e-3) / 1e9, 1))}
    if passes > 0:
        key = "tile_sort_pass"
        b_st = tile_bytes / passes
        ms_st = stage_ms["sort_passes"] / passes
        hbm_stages[key] = dict(bytes=int(b_st), ms=round(ms_st, 4), achieved_gbs=round(b_st / (ms_st * 1e-3) / 1e9, 1))
    for v in hbm_stages.values():
        v["frac"] = round(v["achieved_gbs"] / peaks["hbm_gbs"], 4)

    # ---- end to end through the C ABI with host buffers ----
    e2e = (run_e2e(args, vis, torch, sc_np, cam_objs, W, H, cap, dist, opts) if not (packed or dbuf is not None)
           else dict(value=None, note="not measured for a pre-packed scene or a depth buffer"))

    line = dict(metric=METRIC, value=round(value, 4), unit="ms/frame", n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=round(t_ms / args.steps, 4), higher_is_better=False,
                scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(desc, sort_mode=args.sort_mode, packed=packed, pixels_per_thread=args.ppt,
                            depth_buffer=(f"wall at view depth {args.depth_plane}" if dbuf is not None else None),
                            l2="inputs larger than L2 (attributes exceed 126 MB); no flush",
                            parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
                clocks=clk_summary, e2e=e2e,
                gpu_launches=int(args.steps * {0: 6 + passes, 1: 10 + kDP + passes}[args.sort_mode]
                                 + (2 * args.steps if fwdbwd else 0) + (args.steps if dynamic else 0)
                                 + (args.steps if dbuf is not None else 0)),
                roofline=roof, hbm_stages=hbm_stages,
                stage_ms={names[STAGES.index(k)]: round(v, 4) for k, v in stage_ms.items()},
                keys_per_frame=int(M), visible_per_frame=int(n_vis), sort_passes=passes,
                dynamic_update_ms=(round(update_ms, 4) if update_ms is not None else None),
                sort_keys_per_s=round(M / (stage_ms["sort_passes"] + stage_ms["sort_histogram"]
                                           ) * 1e3, 1),
                gaussians_per_s=round(n / value * 1e3, 1))
    if rank == 0 and world == 1 and not args.no_cpu and not packed:
        line["cpu_baseline"] = cpu_baseline(args.workload, sc_np, cams, desc, budget_s=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_batch(args):
    """16 assets x 8 cameras = 128 images: one graph-captured vis_render_batch vs 128
    sequential vis_render calls of the plain path (same options, images compared)."""
    import ctypes as C
    import torch
    import paper_2512_08478_b300 as vis
    from paper_2512_08478_b300 import synth, tuning
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    scenes_np, cams, cam_scene = synth.workload_batch()
    scenes = [vis.Scene.from_numpy(s) for s in scenes_np]
    if args.no_autotune:
        opts_d, lanes, tuned_ms = dict(tile=16, pixels_per_thread=1, sort_mode=1), 8, None
    else:
        opts_d, lanes, tuned_ms = tuning.autotune(scenes, cams, cam_scene, cache=None,
                                                  log=lambda m: print(m, file=sys.stderr))
    opts = vis.make_opts(**opts_d)
    b = vis.Batch(scenes, cams, cam_scene, lanes=lanes, opts=opts)
    b.render()
    stream = torch.cuda.current_stream()
    # sequential plain path: one workspace for the largest image
    nmax = max(s.n for s in scenes)
    Wm = max(int(c.W) for c in cams)
    Hm = max(int(c.H) for c in cams)
    ws = vis.Workspace(nmax, Wm, Hm, key_capacity=16 * nmax + (1 << 20), opts=opts)
    outs = [(torch.empty((3, c.H, c.W), device="cuda"), torch.empty((c.H, c.W), device="cuda")) for c in cams]
    cam_objs = [vis.make_camera(c) for c in cams]

    def sequential():
        for i, c in enumerate(cam_objs):
            vis.vis_render(scenes[cam_scene[i]].handle, c, cams[i].W, cams[i].H, (0.0, 0.0, 0.0), outs[i][0],
                           outs[i][1], ws.buf, opts)

    for _ in range(args.warmup):
        b.launch()
        sequential()
    b.check()
    vis.vis_check(ws.buf)
    same = all(torch.equal(b.rgb[i], outs[i][0]) and torch.equal(b.alpha[i], outs[i][1]) for i in range(len(cams)))
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e[0].record(stream)
        for _ in range(args.steps):
            b.launch()
        e[1].record(stream)
        for _ in range(args.steps):
            sequential()
        e[2].record(stream)
        torch.cuda.synchronize()
    b.check()
    vis.vis_check(ws.buf)
    t_batch = e[0].elapsed_time(e[1]) / args.steps
    t_seq = e[1].elapsed_time(e[2]) / args.steps
    n_g = sum(scenes[a].n for a in cam_scene)
    line = dict(metric="ms per 128-image heterogeneous batch (16 assets x 8 cameras)", value=round(t_batch, 4),
                unit="ms/batch", n_gpus=1, steps=args.steps, warmup=args.warmup, ms_per_step=round(t_batch, 4),
                higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload="16 assets (N log-uniform 2e4..2e6, SH 0..3) x 8 orbit cameras at "
                                     "{512^2, 1280x720, 1920x1080}", images=len(cams),
                            gaussians=[s.n for s in scenes], opts=opts_d, lanes=lanes),
                sequential_ms=round(t_seq, 4), speedup_vs_sequential=round(t_seq / t_batch, 3),
                images_identical_to_sequential=bool(same), autotune_best_ms=tuned_ms,
                gaussian_views_per_s=round(n_g / t_batch * 1e3, 1), clocks=clk.summary())
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

    for i in range(args.warmup):
        multi(i)
        single(i)
    keys = vis.vis_check(ws.buf)
    vis.vis_check(wsm.buf)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
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
    stage = (C.c_double * 7)()
    ns, nr, npass = C.c_int(), C.c_int(), C.c_int()
    vis._ok(vis.lib().vis_profile_end(stage, 7, C.byref(ns), C.byref(nr), C.byref(npass)))
    vis.vis_check(ws.buf)
    vis.vis_check(wsm.buf)
    t_multi = e[0].elapsed_time(e[1]) / args.steps
    t_single = e[1].elapsed_time(e[2]) / args.steps
    stage_ms = {STAGES_FUSED[k]: round(stage[k] / max(nr.value, 1), 4) for k in range(7)}
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
                gpu_launches=int(args.steps * (len(scenes) + 9 + kDP + npass.value)), clocks=clk.summary())
    if rank == 0:
        print(json.dumps(line), flush=True)


def _committed_traffic(kernel, M, n):
    """DRAM bytes per launch from a committed ncu capture (profiles/traffic.json), scaled
    to this launch by keys (sort, composite) or Gaussians (preprocess); None if absent."""
    p = ROOT / "profiles" / "traffic.json"
    if not p.exists():
        return None
    d = json.loads(p.read_text()).get(kernel)
    if not d:
        return None
    if "bytes_per_key" in d:
        return int(d["bytes_per_key"] * M)
    if "bytes_per_gaussian" in d:
        return int(d["bytes_per_gaussian"] * n)
    return None


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
    e0.record(stream)
    up.wait_event(e0)
    down.wait_event(e0)
    for i in range(steps):
        step(i)
    stream.wait_event(read[(steps - 1) & 1])
    stream.wait_event(read[steps & 1])
    e1.record(stream)
    torch.cuda.synchronize()
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
                config=dict(desc), cpu_baseline=dict(value=round(value, 1), unit="ms/frame", cores=cores,
                                                     kind="oracle", sample=sample),
                e2e=dict(value=round(value, 1), unit="ms/frame", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
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
    ap.add_argument("--sort-mode", type=int, default=None, choices=[0, 1],
                    help="0: one sort of 64-bit (tile, depth) keys; 1: depth sort then tile sort; "
                         "2: depth sort then counting binning (default: the library default)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--tile", type=int, default=16, choices=[8, 16, 32], help="tile size in pixels")
    ap.add_argument("--ppt", type=int, default=1, choices=[1, 2], help="pixels per compositor thread")
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
