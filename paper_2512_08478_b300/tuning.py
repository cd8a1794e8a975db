"""Autotuner for batched renders: picks tile size, compositor block shape, sort mode
and lane count for a batch signature by timing the candidates on the device.

Only configuration is searched here; every candidate runs the library's kernels. The
radix digit width is fixed at 8 bits (the only width the library implements), so it
is reported but not searched. Results are cached in a JSON file keyed by GPU name and
batch signature (asset sizes and SH degrees, image sizes).
"""
from __future__ import annotations

import itertools
import json
import os
from pathlib import Path

DEFAULT_CACHE = Path(os.environ.get("XDG_CACHE_HOME", str(Path.home() / ".cache"))) / "vis_autotune.json"

CANDIDATES = dict(tile=(8, 16, 32), pixels_per_thread=(1, 2), sort_mode=(0, 1), lanes=(4, 8, 16))


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
    """Return (opts dict, lanes, ms) of the fastest candidate; cached per GPU and signature."""
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
    if key in table:
        r = table[key]
        return r["opts"], r["lanes"], r["ms"]
    best = None
    for tile, ppt, mode, lanes in itertools.product(cand["tile"], cand["pixels_per_thread"], cand["sort_mode"],
                                                    cand["lanes"]):
        opts = dict(tile=tile, pixels_per_thread=ppt, sort_mode=mode)
        b = vis.Batch(scenes, cams, cam_scene, lanes=lanes, opts=vis.make_opts(**opts))
        ms = _time_batch(b, reps)
        del b
        if log:
            log(f"autotune tile={tile} ppt={ppt} sort_mode={mode} lanes={lanes}: {ms:.3f} ms")
        if best is None or ms < best[2]:
            best = (opts, lanes, ms)
    if cache is not None:
        table[key] = dict(opts=best[0], lanes=best[1], ms=best[2], digit_bits=8)
        Path(cache).parent.mkdir(parents=True, exist_ok=True)
        Path(cache).write_text(json.dumps(table, indent=1))
    return best
