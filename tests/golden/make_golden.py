"""Writes tests/golden/oracle_tiny_render.json: a regression fixture of the FP64 oracle.

The paper prints no worked example (no image, asset or per-pixel value), so no fixture here is
the paper's. This one is written by the oracle alone (this script imports only `oracle` and the
seeded input generator) and pins the oracle against unintended change: a 20-Gaussian SH2 scene
from synth.mixture_scene(seed 7), seen at 24x20 from (0.3, -0.2, 3.5), background
(0.1, 0.2, 0.3), default options; it stores the image, the per-pixel contributor counts and the
(tile, depth, index) order of every tile. Run it only when an intended change of the oracle's
arithmetic is made (and name the passage that justifies the change in the commit message):

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2512_08478_b300 import synth  # noqa: E402

BG = (0.1, 0.2, 0.3)


def case():
    sc = synth.mixture_scene(20, 7, sh_degree=2, components=4, ball_radius=0.6, comp_std=0.3,
                             log_scale_mean=-2.2, hi_std=0.2)
    cam = synth.look_at((0.3, -0.2, 3.5), (0, 0, 0), 24, 20, 55.0)
    return sc, cam


def compute():
    sc, cam = case()
    img, prep = oracle.render(sc, cam, BG, opts=dict(tile=8))
    tiles_x = (cam.W + 7) // 8
    keys, vals = oracle.duplicate(prep, tiles_x)
    sk, sv = oracle.stable_sort_pairs(keys, vals)
    return dict(rgb=img["rgb"], alpha=img["alpha"], n_contrib=img["n_contrib"], sorted_keys=sk, sorted_vals=sv)


def main():
    r = compute()
    out = dict(
        note="regression fixture of the FP64 oracle (not a paper value: the paper prints no worked example)",
        W=24, H=20, tile=8, bg=list(BG),
        rgb=[repr(float(x)) for x in r["rgb"].ravel()],
        alpha=[repr(float(x)) for x in r["alpha"].ravel()],
        n_contrib=[int(x) for x in r["n_contrib"].ravel()],
        sorted_keys=[int(x) for x in r["sorted_keys"]],
        sorted_vals=[int(x) for x in r["sorted_vals"]],
    )
    with open(os.path.join(HERE, "oracle_tiny_render.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
