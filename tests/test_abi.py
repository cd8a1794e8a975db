"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
function include/vis.h declares, and rejects bad arguments before any device work."""
import re
from pathlib import Path

import pytest

import paper_2512_08478_b300 as vis
from paper_2512_08478_b300 import build

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def L():
    build.build()
    return vis.lib()


def test_every_declared_function_is_exported(L):
    header = (ROOT / "include" / "vis.h").read_text()
    names = re.findall(r"^VIS_API [^(]*?\b(vis_\w+)\s*\(", header, flags=re.M)
    assert len(names) >= 11
    for n in names:
        assert hasattr(L, n), n


def test_workspace_queries_and_validation(L):
    m0 = vis.make_opts(sort_mode=0)
    b = vis.vis_workspace_size(10_000, 256, 256, 100_000, m0)
    lay = vis.vis_workspace_layout(10_000, 256, 256, b, m0)
    assert 100_000 <= lay.key_capacity < 100_100 and lay.total_bytes <= b
    assert lay.tiles_x == 16 and lay.sort_passes == 5 and lay.key_bytes == 8   # 32 depth + 8 tile bits
    lay32 = vis.vis_workspace_layout(10_000, 1920, 1080, 10 ** 9, vis.make_opts(tile=16, sort_mode=0))
    assert lay32.sort_passes == 6                                # 8160 tiles -> 13 bits
    offs = [lay.off_ctrl, lay.off_rec, lay.off_depth, lay.off_rect, lay.off_touched, lay.off_keys[0],
            lay.off_keys[1], lay.off_vals[0], lay.off_vals[1], lay.off_ranges, lay.off_tfinal, lay.off_last,
            lay.off_g2]
    assert all(o % 256 == 0 for o in offs) and len(set(offs)) == len(offs)
    for bad in (dict(n=0), dict(W=0), dict(H=20000), dict(key_capacity=0), dict(key_capacity=1 << 31)):
        a = dict(n=10, W=8, H=8, key_capacity=10)
        a.update(bad)
        with pytest.raises(vis.VisError) as e:
            vis.vis_workspace_size(**a)
        assert e.value.status == vis.VIS_ERR_INVALID_ARG
    with pytest.raises(vis.VisError):
        vis.vis_workspace_size(10, 8, 8, 10, vis.make_opts(tile=12))
    with pytest.raises(vis.VisError):
        vis.vis_workspace_size(10, 8, 8, 10, vis.make_opts(tile_extent=3))
    assert vis.make_opts().tile_extent == 2
    with pytest.raises(vis.VisError) as e:
        vis.vis_workspace_size(10, 8, 8, 10, vis.make_opts(digit_bits=4))
    assert e.value.status == vis.VIS_ERR_UNSUPPORTED
    with pytest.raises(vis.VisError):
        vis.vis_workspace_layout(10, 8, 8, 100)        # too small for even one key
    df = vis.vis_workspace_layout(10_000, 1920, 1080, 10 ** 9, vis.make_opts(sort_mode=1))
    assert df.key_bytes == 2 and df.sort_mode == 1 and df.sort_passes == 2   # 13 tile bits, 16-bit keys
    assert df.sorted_buffer == 0 and df.off_keys[0] != df.off_keys[1]
    one = vis.vis_workspace_layout(10_000, 100, 100, 10 ** 8, vis.make_opts(sort_mode=1))
    assert one.sort_passes == 1 and one.key_bytes == 2                      # 49 tiles: one pass
    wide = vis.vis_workspace_layout(10_000, 3840, 2160, 10 ** 9, vis.make_opts(sort_mode=1, tile=8))
    assert wide.key_bytes == 4 and wide.sort_passes == 3   # 129600 tiles (17 bits): counters exceed shared memory
    assert vis.vis_workspace_size(10_000, 256, 256, 100_000, vis.make_opts(sort_mode=1)) < b
    with pytest.raises(vis.VisError):
        vis.vis_workspace_size(10, 8, 8, 10, vis.make_opts(sort_mode=2))
    assert vis.vis_sort_workspace_size(0, 45) > 0
    with pytest.raises(vis.VisError):
        vis.vis_sort_workspace_size(10, 65)


def test_scene_upload_rejects_null_and_bad_degree(L):
    import ctypes as C
    h = C.c_void_p()
    st = L.vis_scene_upload(None, None, None, None, None, 0, 10, C.byref(h))
    assert st == vis.VIS_ERR_INVALID_ARG and "null" in vis.vis_last_error()
    p = C.c_void_p(1 << 20)   # never dereferenced: upload only records pointers
    st = L.vis_scene_upload(p, p, p, p, p, 4, 10, C.byref(h))
    assert st == vis.VIS_ERR_INVALID_ARG and "sh_degree" in vis.vis_last_error()
    st = L.vis_scene_upload(p, p, C.c_void_p((1 << 20) + 4), p, p, 0, 10, C.byref(h))
    assert st == vis.VIS_ERR_INVALID_ARG and "aligned" in vis.vis_last_error()
    st = L.vis_scene_upload(p, p, p, p, p, 3, 10, C.byref(h))
    assert st == vis.VIS_OK
    L.vis_scene_destroy(h)


def test_multi_scene_slots_and_validation(L):
    """vis_multi_slots pads every scene to whole 256-Gaussian blocks; vis_render_multi
    rejects null scenes and non-finite or singular model transforms before any device work."""
    import ctypes as C
    import numpy as np
    from paper_2512_08478_b300 import synth
    p = C.c_void_p(1 << 20)   # never dereferenced
    hs = []
    for n in (300, 1000, 2049, 1):
        h = C.c_void_p()
        assert L.vis_scene_upload(p, p, p, p, p, 0, n, C.byref(h)) == vis.VIS_OK
        hs.append(h)
    assert vis.vis_multi_slots(hs) == 512 + 1024 + 2304 + 256
    assert vis.vis_multi_slots(hs[:1]) == 512
    cam = vis.make_camera(synth.look_at((0, 0, 4), (0, 0, 0), 64, 64, 50.0))
    bg = (C.c_float * 3)(0, 0, 0)
    arr = (C.c_void_p * 2)(hs[0].value, hs[1].value)

    def call(models, k=2, scenes=arr):
        mp = None if models is None else np.ascontiguousarray(models, np.float32).ctypes.data_as(C.c_void_p)
        return L.vis_render_multi(scenes, mp, k, C.byref(cam), 64, 64, bg, None, p, p, p, 1 << 30, None, None)

    good = np.tile(np.concatenate([np.eye(3), np.zeros((3, 1))], 1)[None], (2, 1, 1))
    sing = good.copy()
    sing[1, 2, :3] = 0.0
    assert call(sing) == vis.VIS_ERR_INVALID_ARG and "model 1 is singular" in vis.vis_last_error()
    nan = good.copy()
    nan[0, 1, 3] = np.nan
    assert call(nan) == vis.VIS_ERR_INVALID_ARG and "non-finite" in vis.vis_last_error()
    assert call(good, k=0) == vis.VIS_ERR_INVALID_ARG and "n_scenes" in vis.vis_last_error()
    holey = (C.c_void_p * 2)(hs[0].value, None)
    assert call(good, scenes=holey) == vis.VIS_ERR_INVALID_ARG and "scene 1 is null" in vis.vis_last_error()
    with pytest.raises(vis.VisError):
        vis.vis_multi_slots([hs[0], C.c_void_p()])
    big = []
    for _ in range(3):   # 3 x 2^30 slots exceed the 2^31 - 1 a workspace indexes
        h = C.c_void_p()
        assert L.vis_scene_upload(p, p, p, p, p, 0, 1 << 30, C.byref(h)) == vis.VIS_OK
        big.append(h)
    assert vis.vis_multi_slots(big[:1]) == 1 << 30
    with pytest.raises(vis.VisError) as e:
        vis.vis_multi_slots(big)
    assert "2^31-1" in str(e.value)
    for h in hs + big:
        L.vis_scene_destroy(h)


def test_packed_scene_sizes_and_validation(L):
    import ctypes as C
    for deg, words in ((0, 2), (1, 6), (2, 14), (3, 24)):
        assert vis.vis_packed_size(1000, deg) == (8000, 12000, 4000 * words)
    with pytest.raises(vis.VisError):
        vis.vis_packed_size(0, 0)
    with pytest.raises(vis.VisError):
        vis.vis_packed_size(10, 4)
    h = C.c_void_p()
    p = C.c_void_p(1 << 20)
    assert L.vis_scene_upload_packed(p, None, p, 0, 10, C.byref(h)) == vis.VIS_ERR_INVALID_ARG
    assert "cov is null" in vis.vis_last_error()
    assert L.vis_scene_upload_packed(p, p, C.c_void_p((1 << 20) + 8), 0, 10, C.byref(h)) == vis.VIS_ERR_INVALID_ARG
    assert L.vis_scene_upload_packed(p, p, p, 2, 10, C.byref(h)) == vis.VIS_OK
    assert L.vis_scene_pack(h, p, p, p, None) == vis.VIS_ERR_INVALID_ARG     # already packed
    assert "already packed" in vis.vis_last_error()
    L.vis_scene_destroy(h)


def test_fused_batch_workspace_and_validation(L):
    """The fused batch (lanes = 0) lays out one workspace for all its images: it grows with
    the key capacity (one group's scratch: two 16-bit canvas-tile key and two value buffers,
    12 B per copy) and with every image's slots and tiles, any digit width is accepted, and
    bad images are rejected on the host before any device work."""
    import ctypes as C
    p = C.c_void_p(1 << 20)   # never dereferenced
    hs = []
    for n in (1000, 70_000):
        h = C.c_void_p()
        assert L.vis_scene_upload(p, p, p, p, p, 1, n, C.byref(h)) == vis.VIS_OK
        hs.append(h)
    scenes = (C.c_void_p * 2)(hs[0].value, hs[1].value)

    def size(cam_scene, W, H, cap, lanes=0, opts=None):
        n = len(cam_scene)
        b = C.c_size_t()
        st = L.vis_batch_workspace_size(scenes, 2, (C.c_int * n)(*cam_scene), (C.c_int * n)(*W), (C.c_int * n)(*H),
                                        n, lanes, cap, vis._opts_ref(opts), C.byref(b))
        return st, b.value

    st, a = size([0, 1], [640, 320], [480, 240], 1 << 20)
    assert st == vis.VIS_OK
    st, b = size([0, 1], [640, 320], [480, 240], 2 << 20)
    assert st == vis.VIS_OK and b - a >= 12 * (1 << 20)
    st, c = size([0, 1, 1], [640, 320, 1920], [480, 240, 1080], 1 << 20)
    assert st == vis.VIS_OK and c > a + 70_000 * 80   # a third image: its slots and tiles
    for d in (8, 10, 11):
        assert size([0, 1], [640, 320], [480, 240], 1 << 20, opts=vis.make_opts(digit_bits=d))[0] == vis.VIS_OK
    st, lane_b = size([0, 1], [640, 320], [480, 240], 1 << 20, lanes=4)
    assert st == vis.VIS_OK and lane_b != a   # the lane baseline's slices
    assert size([0, 2], [640, 320], [480, 240], 1 << 20)[0] == vis.VIS_ERR_INVALID_ARG   # no scene 2
    assert size([0, 1], [640, 0], [480, 240], 1 << 20)[0] == vis.VIS_ERR_INVALID_ARG     # empty image
    assert size([0, 1], [640, 320], [480, 240], 0)[0] == vis.VIS_ERR_INVALID_ARG         # no capacity
    assert size([0, 1], [640, 320], [480, 240], 1 << 20, opts=vis.make_opts(digit_bits=9))[0] \
        == vis.VIS_ERR_UNSUPPORTED
    for h in hs:
        L.vis_scene_destroy(h)
