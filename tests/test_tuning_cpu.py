"""Host logic of the batch autotuner (tuning.py): it times every candidate, keeps the fastest,
caches the choice per GPU and batch signature, and answers from the cache next time without
timing anything. The batch and its timing are replaced by fakes; no GPU is needed."""
import json
from types import SimpleNamespace

import paper_2512_08478_b300 as vis
from paper_2512_08478_b300 import tuning


def test_autotune_picks_the_fastest_and_caches(tmp_path, monkeypatch):
    import torch
    made = []

    class FakeBatch:
        def __init__(self, scenes, cams, cam_scene, lanes, opts):
            assert lanes == 0   # the tuner times the fused pipeline
            self.key = (opts.tile, opts.digit_bits, opts.pixels_per_thread)
            made.append(self.key)

    def fake_time(b, reps):
        t, digit_bits, ppt = b.key
        return 1.0 + 0.1 * abs(t - 16) + 0.01 * abs(digit_bits - 10) + 0.05 * ppt

    monkeypatch.setattr(vis, "Batch", FakeBatch)
    monkeypatch.setattr(tuning, "_time_batch", fake_time)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "FakeGPU")
    scenes = [SimpleNamespace(n=1000, sh_degree=3), SimpleNamespace(n=50, sh_degree=0)]
    cams = [SimpleNamespace(W=64, H=48), SimpleNamespace(W=32, H=32)]
    cache = tmp_path / "tune.json"
    opts, ms = tuning.autotune(scenes, cams, [0, 1], cache=cache)
    n_cand = 1
    for v in tuning.CANDIDATES.values():
        n_cand *= len(v)
    assert len(made) == n_cand
    assert opts == dict(tile=16, digit_bits=10, pixels_per_thread=1)
    assert abs(ms - 1.05) < 1e-12
    table = json.loads(cache.read_text())
    assert len(table) == 1 and next(iter(table)).startswith("FakeGPU|")
    made.clear()
    again = tuning.autotune(scenes, cams, [0, 1], cache=cache)
    assert made == [] and again == (opts, ms)
    # another batch signature is tuned afresh
    tuning.autotune(scenes[:1], cams[:1], [0], cache=cache, candidates=dict(tile=(16,), pixels_per_thread=(1,)))
    assert len(made) == 3 and len(json.loads(cache.read_text())) == 2


def test_signature_depends_on_sizes_degrees_and_images():
    a = [SimpleNamespace(n=10, sh_degree=1)]
    c = [SimpleNamespace(W=8, H=8)]
    s0 = tuning.signature(a, c, [0])
    assert s0 != tuning.signature([SimpleNamespace(n=11, sh_degree=1)], c, [0])
    assert s0 != tuning.signature([SimpleNamespace(n=10, sh_degree=2)], c, [0])
    assert s0 != tuning.signature(a, [SimpleNamespace(W=8, H=9)], [0])
