"""The stored regression fixture of the oracle (tests/golden/oracle_tiny_render.json, written
by tests/golden/make_golden.py, which calls only the oracle): the oracle still reproduces it,
and the CUDA path matches it (image within the parity bar, tile order bit for bit)."""
import importlib.util
import json
from pathlib import Path

import numpy as np
import pytest

GOLDEN = Path(__file__).resolve().parent / "golden"


def _load():
    d = json.loads((GOLDEN / "oracle_tiny_render.json").read_text())
    W, H = d["W"], d["H"]
    return dict(rgb=np.array([float(x) for x in d["rgb"]]).reshape(3, H, W),
                alpha=np.array([float(x) for x in d["alpha"]]).reshape(H, W),
                n_contrib=np.array(d["n_contrib"]).reshape(H, W),
                keys=np.array(d["sorted_keys"], np.uint64), vals=np.array(d["sorted_vals"], np.uint32),
                bg=tuple(d["bg"]), tile=d["tile"])


def _maker():
    spec = importlib.util.spec_from_file_location("make_golden", GOLDEN / "make_golden.py")
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_oracle_reproduces_the_fixture():
    g = _load()
    r = _maker().compute()
    assert np.abs(r["rgb"] - g["rgb"]).max() <= 1e-13
    assert np.abs(r["alpha"] - g["alpha"]).max() <= 1e-13
    assert np.array_equal(r["n_contrib"], g["n_contrib"])
    assert np.array_equal(r["sorted_keys"], g["keys"]) and np.array_equal(r["sorted_vals"], g["vals"])
    assert (g["alpha"] > 0).mean() > 0.2 and g["n_contrib"].max() >= 10


@pytest.mark.gpu
@pytest.mark.parametrize("sort_mode", [0, 1])
def test_cuda_path_matches_the_fixture(sort_mode):
    import paper_2512_08478_b300 as vis
    from gpu_helpers import gpu_stage_outputs, render_gpu
    g = _load()
    sc, cam = _maker().case()
    rgb, alpha, s, ws = render_gpu(sc, cam, g["bg"], vis.make_opts(tile=g["tile"], sort_mode=sort_mode,
                                                                   tile_extent=0))
    assert np.abs(rgb - g["rgb"]).max() <= 2e-4 and np.abs(alpha - g["alpha"]).max() <= 2e-4
    if sort_mode == 0:   # the 64-bit (tile, depth) keys and their Gaussian indices, bit for bit
        st = gpu_stage_outputs(s, ws)
        assert np.array_equal(st["keys"], g["keys"]) and np.array_equal(st["vals"], g["vals"])
