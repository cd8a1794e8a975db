"""Autotuners: for batched renders, the tile size, the radix digit width and the compositor
block shape of a fused batch (one pipeline over all images) for a batch signature; for a
single-image workload, the compositor block shape (pick_fastest over any step callable).
Both time every candidate on the device.

Only configuration is searched here; every candidate runs the library's kernels. Results
are cached in a JSON file keyed by GPU name and batch signature (asset sizes and SH
degrees, image sizes).
"""
from __future__ import annotations

import itertools
import json
import os
from pathlib import Path

DEFAULT_CACHE = Path(os.environ.get("XDG_CACHE_HOME", str(Path.home() / ".cache"))) / "vis_autotune.json"

# tile edge (px), radix digit width of the depth sort and the (image, tile) sort, and pixels
# per compositor thread (block shape)
CANDIDATES = dict(tile=(8, 16, 32), digit_bits=(8, 10, 11), pixels_per_thread=(1, 2))


def signature(scenes, cams, cam_scene) -> str:
    sizes = tuple((s.n, s.sh_degree) for s in scenes)
    imgs = tuple(sorted((int(c.W), int(c.H), int(a)) for c, a in zip(cams, cam_scene)))
    return json.dumps([sizes, imgs])


def _time_batch(b, reps):
    import torch
    b.render()
    b.launch()
    b.check()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        b.launch()
    e1.record(s)
    b.check()
    return e0.elapsed_time(e1) / reps


def autotune(scenes, cams, cam_scene, candidates=None, reps=3, cache: Path | None = DEFAULT_CACHE, log=None):
    """Return (opts dict, ms) of the fastest candidate of a fused batch; cached per GPU and
    batch signature."""
    import torch
    import paper_2512_08478_b300 as vis
    cand = dict(CANDIDATES)
    if candidates:
        cand.update(candidates)
    key = torch.cuda.get_device_name() + "|" + signature(scenes, cams, cam_scene)
    table = {}
    if cache is not None and Path(cache).exists():
        try:
            table = json.loads(Path(cache).read_text())
        except ValueError:
            table = {}
    if key in table and "digit_bits" in table[key].get("opts", {}):
        r = table[key]
        return r["opts"], r["ms"]
    best = None
    for tile, digit_bits, ppt in itertools.product(cand["tile"], cand["digit_bits"], cand["pixels_per_thread"]):
        opts = dict(tile=tile, digit_bits=digit_bits, pixels_per_thread=ppt)
        b = vis.Batch(scenes, cams, cam_scene, lanes=0, opts=vis.make_opts(**opts))
        ms = _time_batch(b, reps)
        del b
        if log:
            log(f"autotune tile={tile} digit_bits={digit_bits} ppt={ppt}: {ms:.3f} ms")
        if best is None or ms < best[1]:
            best = (opts, ms)
    if cache is not None:
        table[key] = dict(opts=best[0], ms=best[1])
        Path(cache).parent.mkdir(parents=True, exist_ok=True)
        Path(cache).write_text(json.dumps(table, indent=1))
    return best


def pick_fastest(candidates, run, reps=4, warmup=2, log=None):
    """Time `run(c)` (one step of device work on the current stream) for every candidate c and
    return (fastest candidate, {candidate: ms per step})."""
    import torch
    s = torch.cuda.current_stream()
    times = {}
    for c in candidates:
        for _ in range(warmup):
            run(c)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            run(c)
        e1.record(s)
        torch.cuda.synchronize()
        times[c] = e0.elapsed_time(e1) / reps
        if log:
            log(f"pick_fastest {c}: {times[c]:.4f} ms")
    return min(times, key=times.get), times
