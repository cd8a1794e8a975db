// vis_render_batch -- many assets seen by many cameras in one call (the paper renders
// several models per frame with one global sort, Algorithm 1).
//
// Fused (a batch created with lanes = 0, the default of the Python binding): every
// (asset, camera) image is one item of ONE preprocess launch over the work list of all of
// them (each item's Gaussians fill their own run of workspace slots, padded to whole
// blocks). The images are then taken in groups: a group's images are stacked as tile rows
// of one canvas, a tile grid as wide as its widest image and of at most 51200 tiles, and
// the preprocess writes each footprint in its canvas's rows. Every group runs the
// single-image pipeline over its canvas -- compaction of its survivors, one depth sort of
// all of them, the tile copies emitted in that order with 16-bit canvas tile ids, the
// counts-first stable sort by tile id (which yields every image's own front-to-back order),
// and one compositor launch over the canvas, longest tiles first, each CTA finding its
// image in the group's image table. The groups run on three streams, each with a scratch area
// sized for the largest group (the batch's key capacity applies to each group). The whole
// sequence is captured once into a CUDA graph and replayed by later calls with the same
// arguments; the item tables are uploaded before every launch. Each image is bit-identical
// to vis_render of the same (asset, camera, options).
//
// Lanes (lanes >= 1, kept as a baseline): images are assigned to `lanes` streams forked
// from the batch's origin stream by longest-processing-time scheduling on the estimated
// cost (Gaussians + pixels); each lane renders its images one after another with
// vis_render in its own workspace slice, and after every image a one-thread kernel
// copies the slice's status into the image's status word. The fork / render / join
// sequence is captured into a CUDA graph, so the lanes run as concurrent branches.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "vis_internal.cuh"

struct vis_batch {
    int lanes = 0;                   // 0: the fused pipeline
    cudaStream_t origin = nullptr;   // the graph is captured on and launched from this stream
    cudaEvent_t in_ev = nullptr, out_ev = nullptr;
    std::vector<cudaStream_t> streams;
    cudaEvent_t fork_ev = nullptr;
    std::vector<cudaEvent_t> join_ev;
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> key;   // serialised arguments of the captured graph
    int device = -1;
    std::vector<unsigned char> tables;   // fused: item and image tables, uploaded before each launch
    size_t tables_off = 0;               // their offset in the workspace
};

namespace vis {

__global__ void copy_status_kernel(const Ctrl* __restrict__ ctrl, uint32_t* __restrict__ status) {
    status[0] = ctrl->num_keys;
    status[1] = ctrl->error;
}

// fused batch: a group's status block (key count of the group, error bits) into the status
// word of each of its n images
__global__ void copy_status_group_kernel(const Ctrl* __restrict__ ctrl, const BatchImage* __restrict__ images,
                                         uint32_t* __restrict__ status, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int k = images[i].index;
        status[2 * k] = ctrl->num_keys;
        status[2 * k + 1] = ctrl->error;
    }
}

}  // namespace vis

namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// status words live at the start of the batch workspace: 2 x uint32 per image
size_t status_bytes(int n_images) { return align256(sizeof(uint32_t) * 2 * (size_t)n_images); }

struct Plan {
    std::vector<int> lane_of;            // image -> lane
    std::vector<std::vector<int>> order; // lane -> images in render order
    size_t slice_bytes = 0;
};

vis_status fail_b(vis_status s, const std::string& m) {
    vis::set_last_error(m.c_str());
    return s;
}

Plan make_plan(const vis_scene_t* scenes, const int* cam_scene, const int* W, const int* H, int n_images, int lanes,
               size_t slice_bytes) {
    Plan p;
    p.lane_of.assign(n_images, 0);
    p.order.assign(lanes, {});
    std::vector<double> cost(n_images), load(lanes, 0.0);
    std::vector<int> idx(n_images);
    for (int i = 0; i < n_images; ++i) {
        idx[i] = i;
        cost[i] = (double)vis::scene_size(scenes[cam_scene[i]]) + 4.0 * (double)W[i] * H[i];
    }
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    for (int i : idx) {
        int best = 0;
        for (int l = 1; l < lanes; ++l)
            if (load[l] < load[best]) best = l;
        p.lane_of[i] = best;
        p.order[best].push_back(i);
        load[best] += cost[i];
    }
    p.slice_bytes = slice_bytes;
    return p;
}

int64_t pad_blocks(int64_t n) { return (n + vis::kPrepThreads - 1) / vis::kPrepThreads * vis::kPrepThreads; }

// Plan and workspace of a fused batch: the status words (2 per image); the tables (the
// items' preprocess parameters in list order -- plain scenes, then pre-packed ones --, each
// list's first blocks, the image table in group order); the per-slot buffers of all slots
// (records, depths, footprints, counts, block sums); then one scratch area for a group's
// pipeline, sized for the largest group: the single-image layout of the group's canvas
// (make_layout) without its per-slot and adjoint buffers.
struct Group {
    int first = 0, count = 0;        // images [first, first + count) of the group order
    int cw = 0, rows = 0;            // canvas: width in tiles, height in tile rows
    int64_t slot_begin = 0, slots = 0;
};

struct Fused {
    std::vector<int> order;          // group order -> image
    std::vector<int> row0;           // image -> first canvas row
    std::vector<int64_t> slot0;      // image -> first slot
    std::vector<Group> groups;
    int64_t slots = 0;
    int n_list[2] = {0, 0};          // images of the plain and of the pre-packed list
    int64_t blocks[2] = {0, 0};      // preprocess blocks of each list
    int digit_bits = 8, tile = 16;
    int64_t cap = 0;
    size_t off_items = 0, off_blk0 = 0, off_images = 0, tables_end = 0;
    size_t off_rec = 0, off_depth = 0, off_rect = 0, off_touched = 0, off_bsum = 0, off_boff = 0;
    size_t off_scratch = 0, scratch_stride = 0, total = 0;
    int n_scratch = 1;               // scratch areas: groups run on that many streams at once
    bool layout_ok = true;           // make_layout's region order is the one group_layout assumes
};

// Streams (and scratch areas) of a fused batch: group g runs on stream g mod kFusedStreams,
// so that one group's latency-bound sort overlaps another's compositor (two, three and four
// measured: 25.0, 24.8 and 25.4 ms for the 128-image batch).
constexpr int kFusedStreams = 3;

// The single-image layout of group g's canvas, mapped onto the batch workspace: the scratch
// regions of make_layout's order -- [status block .. tile order] and [scan totals .. values]
// -- moved into the scratch area, the per-slot buffers pointing at the group's slots.
vis::Layout group_layout(const Fused& F, const Group& g, int area, size_t* scratch_bytes = nullptr,
                         bool* order_ok = nullptr) {
    vis::Layout L = vis::make_layout(g.slots, g.cw * F.tile, g.rows * F.tile, F.tile, F.cap, vis::kSortDepthFirst,
                                     F.digit_bits);
    if (order_ok)
        *order_ok = L.zero_end <= L.off_rec && L.off_order < L.off_rec && L.off_lookback_tile < L.off_rec &&
                    L.off_scan_lb < L.zero_end && L.off_boff < L.off_bsum2 &&
                    L.off_vals[1] < L.off_tfinal && L.off_ctrl < L.off_rec;
    // make_layout takes, in order: the cleared region (status .. scan look-back words), the
    // tile order and the tile look-back words, the per-slot buffers (records .. block
    // offsets), the scratch (second block sums .. values), then the adjoint and depth-buffer
    // buffers
    const size_t a_end = L.off_rec, b_begin = L.off_bsum2, b_end = L.off_tfinal;
    const size_t base = F.off_scratch + (size_t)area * F.scratch_stride, shift_b = base + a_end;
    auto mv_a = [&](size_t& o) { o += base; };
    auto mv_b = [&](size_t& o) { o = shift_b + (o - b_begin); };
    mv_a(L.off_ctrl); mv_a(L.off_hist); mv_a(L.off_hist_tile); mv_a(L.off_lookback); mv_a(L.off_ranges);
    mv_a(L.off_tdiff); mv_a(L.off_order); mv_a(L.off_lookback_tile); mv_a(L.off_scan_lb); mv_a(L.zero_begin);
    mv_a(L.zero_end);
    mv_b(L.off_bsum2); mv_b(L.off_boff2);
    for (int k = 0; k < 2; ++k) { mv_b(L.off_dkeys[k]); mv_b(L.off_dvals[k]); mv_b(L.off_keys[k]); mv_b(L.off_vals[k]); }
    L.off_rec = F.off_rec + sizeof(float4) * 3 * (size_t)g.slot_begin;
    L.off_depth = F.off_depth + sizeof(float) * (size_t)g.slot_begin;
    L.off_rect = F.off_rect + sizeof(uint4) * (size_t)g.slot_begin;
    L.off_touched = F.off_touched + sizeof(uint32_t) * (size_t)g.slot_begin;
    L.off_bsum = F.off_bsum + sizeof(uint32_t) * (size_t)(g.slot_begin / vis::kPrepThreads);
    L.off_boff = F.off_boff + sizeof(uint32_t) * (size_t)(g.slot_begin / vis::kPrepThreads);
    L.off_tfinal = L.off_last = L.off_g2 = L.off_zmax = 0;   // not used by a batch
    if (scratch_bytes) *scratch_bytes = a_end + (b_end - b_begin);
    return L;
}

Fused fused_layout(const std::vector<int64_t>& n_img, const std::vector<char>& packed, const int* W, const int* H,
                   int n_images, int tile, int64_t cap, int digit_bits) {
    Fused F;
    F.tile = tile;
    F.cap = cap;
    F.digit_bits = digit_bits;
    std::vector<int> tx(n_images), ty(n_images);
    for (int i = 0; i < n_images; ++i) {
        tx[i] = (W[i] + tile - 1) / tile;
        ty[i] = (H[i] + tile - 1) / tile;
        F.n_list[packed[i] ? 1 : 0] += 1;
        F.blocks[packed[i] ? 1 : 0] += pad_blocks(n_img[i]) / vis::kPrepThreads;
    }
    // groups: the images by decreasing width, stacked while the canvas holds at most
    // kTileFusedMaxTiles tiles (an image larger than that is a group of its own, sorted with
    // 32-bit tile ids)
    F.order.resize(n_images);
    for (int i = 0; i < n_images; ++i) F.order[i] = i;
    std::stable_sort(F.order.begin(), F.order.end(), [&](int a, int b) {
        return tx[a] != tx[b] ? tx[a] > tx[b] : ty[a] > ty[b];
    });
    F.row0.assign(n_images, 0);
    F.slot0.assign(n_images, 0);
    for (int k = 0; k < n_images; ++k) {
        const int i = F.order[k];
        if (F.groups.empty() ||
            (int64_t)(F.groups.back().rows + ty[i]) * F.groups.back().cw > (int64_t)vis::kTileFusedMaxTiles) {
            Group g;
            g.first = k;
            g.cw = tx[i];
            g.slot_begin = F.slots;
            F.groups.push_back(g);
        }
        Group& g = F.groups.back();
        F.row0[i] = g.rows;
        F.slot0[i] = F.slots;
        g.rows += ty[i];
        g.count += 1;
        F.slots += pad_blocks(n_img[i]);
        g.slots = F.slots - g.slot_begin;
    }
    size_t off = status_bytes(n_images);
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    F.off_items = take(sizeof(vis::PrepParams) * (size_t)n_images);
    F.off_blk0 = take(sizeof(uint32_t) * (size_t)n_images);
    F.off_images = take(sizeof(vis::BatchImage) * (size_t)n_images);
    F.tables_end = off;
    F.off_rec = take(sizeof(float4) * 3 * (size_t)F.slots);
    F.off_depth = take(sizeof(float) * (size_t)F.slots);
    F.off_rect = take(sizeof(uint4) * (size_t)F.slots);
    F.off_touched = take(sizeof(uint32_t) * (size_t)F.slots);
    F.off_bsum = take(sizeof(uint32_t) * (size_t)(F.slots / vis::kPrepThreads));
    F.off_boff = take(sizeof(uint32_t) * (size_t)(F.slots / vis::kPrepThreads));
    F.off_scratch = off;
    size_t scratch = 0;
    for (const Group& g : F.groups) {
        size_t b = 0;
        bool ok = true;
        group_layout(F, g, 0, &b, &ok);
        scratch = std::max(scratch, b);
        F.layout_ok = F.layout_ok && ok;
    }
    F.n_scratch = (int)std::min<size_t>(kFusedStreams, F.groups.size());
    F.scratch_stride = align256(scratch);
    F.total = F.off_scratch + (size_t)F.n_scratch * F.scratch_stride;
    return F;
}

// Per-image sizes and kinds of a batch; VIS_ERR_INVALID_ARG on a bad image.
vis_status fused_inputs(const vis_scene_t* scenes, int n_scenes, const int* cam_scene, const int* W, const int* H,
                        int n_images, std::vector<int64_t>* n_img, std::vector<char>* packed) {
    if (n_images > (1 << 16)) return fail_b(VIS_ERR_INVALID_ARG, "a fused batch holds at most 65536 images");
    n_img->assign(n_images, 0);
    packed->assign(n_images, 0);
    int64_t slots = 0, tiles = 0;
    for (int i = 0; i < n_images; ++i) {
        if (cam_scene[i] < 0 || cam_scene[i] >= n_scenes || !scenes[cam_scene[i]])
            return fail_b(VIS_ERR_INVALID_ARG, "cam_scene out of range");
        if (W[i] < 1 || H[i] < 1 || W[i] > 16384 || H[i] > 16384)
            return fail_b(VIS_ERR_INVALID_ARG, "image size out of [1, 16384]");
        (*n_img)[i] = vis::scene_size(scenes[cam_scene[i]]);
        (*packed)[i] = vis::scene_packed(scenes[cam_scene[i]]) ? 1 : 0;
        slots += pad_blocks((*n_img)[i]);
        tiles += (int64_t)((W[i] + 7) / 8) * ((H[i] + 7) / 8);
    }
    if (slots > 0x7fffffffLL) return fail_b(VIS_ERR_INVALID_ARG, "the batch's images hold more than 2^31-1 Gaussians");
    if (tiles > 0x7fffffffLL) return fail_b(VIS_ERR_INVALID_ARG, "the batch's images hold more than 2^31-1 tiles");
    return VIS_OK;
}

int64_t fused_capacity(const std::vector<int64_t>& n_img, const std::vector<char>& packed, const int* W, const int* H,
                       int n_images, int tile, int digit_bits, size_t ws_bytes) {
    if (fused_layout(n_img, packed, W, H, n_images, tile, 1, digit_bits).total > ws_bytes) return 0;
    int64_t lo = 1, hi = vis::kMaxKeys;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (fused_layout(n_img, packed, W, H, n_images, tile, mid, digit_bits).total <= ws_bytes) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

void append(std::vector<unsigned char>& k, const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    k.insert(k.end(), c, c + n);
}

}  // namespace

extern "C" {

vis_status vis_batch_create(int lanes, vis_batch_t* out) {
    if (!out) return fail_b(VIS_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (lanes < 0 || lanes > 64) return fail_b(VIS_ERR_INVALID_ARG, "lanes must be in [0, 64]");
    vis_batch* b = new (std::nothrow) vis_batch;
    if (!b) return fail_b(VIS_ERR_INVALID_ARG, "out of host memory");
    b->lanes = lanes;
    cudaGetDevice(&b->device);
    const int n_streams = lanes > 0 ? lanes : kFusedStreams;   // lanes, or the fused groups' streams
    b->streams.resize(n_streams);
    b->join_ev.resize(n_streams);
    cudaError_t e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->in_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->out_ev, cudaEventDisableTiming);
    for (int l = 0; l < n_streams && e == cudaSuccess; ++l) {
        e = cudaStreamCreateWithFlags(&b->streams[l], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev[l], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        vis_batch_destroy(b);
        return fail_b(VIS_ERR_CUDA, std::string("batch set-up: ") + cudaGetErrorString(e));
    }
    *out = b;
    vis::set_last_error("");
    return VIS_OK;
}

void vis_batch_destroy(vis_batch_t b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto s : b->streams) if (s) cudaStreamDestroy(s);
    for (auto ev : b->join_ev) if (ev) cudaEventDestroy(ev);
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    if (b->in_ev) cudaEventDestroy(b->in_ev);
    if (b->out_ev) cudaEventDestroy(b->out_ev);
    if (b->origin) cudaStreamDestroy(b->origin);
    delete b;
}

vis_status vis_batch_workspace_size(const vis_scene_t* scenes, int n_scenes, const int* cam_scene, const int* W,
                                    const int* H, int n_images, int lanes, int64_t key_capacity,
                                    const vis_render_opts* opts, size_t* bytes) {
    if (!scenes || !cam_scene || !W || !H || !bytes) return fail_b(VIS_ERR_INVALID_ARG, "null argument");
    if (n_images < 1 || n_scenes < 1 || lanes < 0) return fail_b(VIS_ERR_INVALID_ARG, "empty batch");
    if (lanes == 0) {   // fused: key_capacity counts the copies of all images together
        vis_render_opts o;
        vis_status st = vis::batch_opts(opts, &o);
        if (st) return st;
        if (key_capacity < 1 || key_capacity > (int64_t)vis::kMaxKeys)
            return fail_b(VIS_ERR_INVALID_ARG, "key_capacity must be in [1, 2^30-1]");
        std::vector<int64_t> n_img;
        std::vector<char> packed;
        if ((st = fused_inputs(scenes, n_scenes, cam_scene, W, H, n_images, &n_img, &packed))) return st;
        const Fused F = fused_layout(n_img, packed, W, H, n_images, o.tile, key_capacity, o.digit_bits);
        if (!F.layout_ok) return fail_b(VIS_ERR_UNSUPPORTED, "workspace layout order not the one the batch maps");
        *bytes = F.total;
        vis::set_last_error("");
        return VIS_OK;
    }
    size_t slice = 0;
    for (int i = 0; i < n_images; ++i) {
        if (cam_scene[i] < 0 || cam_scene[i] >= n_scenes || !scenes[cam_scene[i]])
            return fail_b(VIS_ERR_INVALID_ARG, "cam_scene out of range");
        size_t b = 0;
        vis_status st = vis_workspace_size(vis::scene_size(scenes[cam_scene[i]]), W[i], H[i], key_capacity, opts, &b);
        if (st) return st;
        if (b > slice) slice = b;
    }
    *bytes = status_bytes(n_images) + (size_t)lanes * align256(slice);
    vis::set_last_error("");
    return VIS_OK;
}

static vis_status render_fused(vis_batch_t b, const vis_scene_t* scenes, int n_scenes, const vis_camera* cams,
                               const int* cam_scene, const int* W, const int* H, int n_images, const float bg[3],
                               float* const* out_rgb, float* const* out_alpha, void* ws, size_t ws_bytes,
                               const vis_render_opts* opts, cudaStream_t stream) {
    vis_render_opts o;
    vis_status st = vis::batch_opts(opts, &o);
    if (st) return st;
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(bg[k])) return fail_b(VIS_ERR_INVALID_ARG, "bg is not finite");
    if (reinterpret_cast<uintptr_t>(ws) & 255u) return fail_b(VIS_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    std::vector<int64_t> n_img;
    std::vector<char> packed;
    if ((st = fused_inputs(scenes, n_scenes, cam_scene, W, H, n_images, &n_img, &packed))) return st;
    for (int i = 0; i < n_images; ++i)
        if (!out_rgb[i] || !out_alpha[i] || (reinterpret_cast<uintptr_t>(out_rgb[i]) & 15u) ||
            (reinterpret_cast<uintptr_t>(out_alpha[i]) & 15u))
            return fail_b(VIS_ERR_INVALID_ARG, "image outputs null or not 16-byte aligned");
    const int64_t cap = fused_capacity(n_img, packed, W, H, n_images, o.tile, o.digit_bits, ws_bytes);
    if (cap < 1) return fail_b(VIS_ERR_INVALID_ARG, "batch workspace too small");
    const Fused F = fused_layout(n_img, packed, W, H, n_images, o.tile, cap, o.digit_bits);
    if (!F.layout_ok) return fail_b(VIS_ERR_UNSUPPORTED, "workspace layout order not the one the batch maps");
    const uint32_t spin = o.spin_limit > 0 ? (uint32_t)o.spin_limit : vis::kSpinLimit;
    char* w = static_cast<char*>(ws);

    std::vector<unsigned char> key;
    append(key, &o, sizeof(o));
    append(key, &ws, sizeof(ws));
    append(key, &ws_bytes, sizeof(ws_bytes));
    append(key, bg, 3 * sizeof(float));
    append(key, &n_images, sizeof(n_images));
    for (int i = 0; i < n_images; ++i) {
        append(key, &cams[i], sizeof(vis_camera));
        append(key, &W[i], sizeof(int));
        append(key, &H[i], sizeof(int));
        append(key, &out_rgb[i], sizeof(float*));
        append(key, &out_alpha[i], sizeof(float*));
        vis::append_scene_key(key, scenes[cam_scene[i]]);
    }
    if (!b->exec || key != b->key) {
        // the item tables: preprocess parameters in list order (plain scenes, then pre-packed
        // ones, each in group order), each list's first blocks, and the image table in group
        // order
        std::vector<vis::PrepParams> items(n_images);
        std::vector<uint32_t> blk0(n_images);
        std::vector<vis::BatchImage> images(n_images);
        int pos[2] = {0, F.n_list[0]};
        int64_t nb[2] = {0, 0};
        for (int k = 0; k < n_images; ++k) {
            const int i = F.order[k];
            const int lst = packed[i] ? 1 : 0;
            vis::PrepParams p;
            if ((st = vis::batch_item(scenes[cam_scene[i]], &cams[i], W[i], H[i], o, F.slot0[i], (uint32_t)i, &p)))
                return st;
            p.canvas_row0 = (uint32_t)F.row0[i];
            items[pos[lst]] = p;
            blk0[pos[lst]] = (uint32_t)nb[lst];
            ++pos[lst];
            nb[lst] += pad_blocks(n_img[i]) / vis::kPrepThreads;
        }
        for (const Group& g : F.groups)
            for (int k = g.first; k < g.first + g.count; ++k) {
                const int i = F.order[k];
                vis::BatchImage im;
                std::memset(&im, 0, sizeof(im));
                im.slot0 = F.slot0[i] - g.slot_begin;
                im.tile0 = (uint32_t)((int64_t)F.row0[i] * g.cw);
                im.W = W[i]; im.H = H[i];
                im.tiles_x = (W[i] + o.tile - 1) / o.tile; im.tiles_y = (H[i] + o.tile - 1) / o.tile;
                im.index = i;
                im.out_rgb = out_rgb[i]; im.out_alpha = out_alpha[i];
                images[k] = im;
            }
        b->tables.assign(F.tables_end - F.off_items, 0);
        std::memcpy(b->tables.data(), items.data(), sizeof(vis::PrepParams) * n_images);
        std::memcpy(b->tables.data() + (F.off_blk0 - F.off_items), blk0.data(), sizeof(uint32_t) * n_images);
        std::memcpy(b->tables.data() + (F.off_images - F.off_items), images.data(), sizeof(vis::BatchImage) * n_images);
        b->tables_off = F.off_items;
        const vis::PrepParams* d_items = reinterpret_cast<const vis::PrepParams*>(w + F.off_items);
        const uint32_t* d_blk0 = reinterpret_cast<const uint32_t*>(w + F.off_blk0);
        const vis::BatchImage* d_images = reinterpret_cast<const vis::BatchImage*>(w + F.off_images);

        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        cudaGraph_t graph = nullptr;
        cudaStream_t s = b->origin;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return fail_b(VIS_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
        // the preprocess of every item (the per-slot buffers of all slots)
        vis::Layout Lp;
        Lp.off_rec = F.off_rec; Lp.off_depth = F.off_depth; Lp.off_rect = F.off_rect;
        Lp.off_touched = F.off_touched; Lp.off_bsum = F.off_bsum;
        vis::launch_preprocess_batch(d_items, d_blk0, F.n_list[0], F.blocks[0], false, Lp, w, s);
        vis::launch_preprocess_batch(d_items + F.n_list[0], d_blk0 + F.n_list[0], F.n_list[1], F.blocks[1], true, Lp,
                                     w, s);
        // then every group's canvas through the single-image pipeline, groups on
        // F.n_scratch streams forked from the origin, each stream with its scratch area
        cudaEventRecord(b->fork_ev, s);
        for (int k = 0; k < F.n_scratch; ++k) cudaStreamWaitEvent(b->streams[k], b->fork_ev, 0);
        for (size_t gi = 0; gi < F.groups.size(); ++gi) {
            const Group& g = F.groups[gi];
            const int area = (int)(gi % (size_t)F.n_scratch);
            cudaStream_t gs = b->streams[area];
            vis::Layout L = group_layout(F, g, area);
            L.spin_limit = spin;
            cudaMemsetAsync(w + L.zero_begin, 0, L.zero_end - L.zero_begin, gs);
            vis::launch_depth_first(L, w, gs, nullptr, 0);
            if (!L.tile_fused) vis::launch_ranges32(L, w, gs);
            vis::launch_composite_batch(L, w, d_images + g.first, g.count, L.ntiles, bg[0], bg[1], bg[2],
                                        o.alpha_min, o.alpha_max, o.t_stop, o.pixels_per_thread, gs);
            vis::copy_status_group_kernel<<<(g.count + 255) / 256, 256, 0, gs>>>(
                reinterpret_cast<const vis::Ctrl*>(w + L.off_ctrl), d_images + g.first, reinterpret_cast<uint32_t*>(w),
                g.count);
        }
        for (int k = 0; k < F.n_scratch; ++k) {
            cudaEventRecord(b->join_ev[k], b->streams[k]);
            cudaStreamWaitEvent(s, b->join_ev[k], 0);
        }
        e = cudaStreamEndCapture(s, &graph);
        if (e != cudaSuccess) return fail_b(VIS_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { b->exec = nullptr; return fail_b(VIS_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e)); }
        b->key = key;
    }
    // order the tables and the graph after the caller's prior work, and the caller's later
    // work after them
    cudaError_t e = cudaEventRecord(b->in_ev, stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->in_ev, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w + b->tables_off, b->tables.data(), b->tables.size(), cudaMemcpyHostToDevice, b->origin);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->origin);
    if (e == cudaSuccess) e = cudaEventRecord(b->out_ev, b->origin);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, b->out_ev, 0);
    if (e != cudaSuccess) return fail_b(VIS_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    vis::set_last_error("");
    return VIS_OK;
}

vis_status vis_render_batch(vis_batch_t b, const vis_scene_t* scenes, int n_scenes, const vis_camera* cams,
                            const int* cam_scene, const int* W, const int* H, int n_images, const float bg[3],
                            float* const* out_rgb, float* const* out_alpha, void* ws, size_t ws_bytes,
                            const vis_render_opts* opts, void* stream_) {
    if (!b) return fail_b(VIS_ERR_INVALID_ARG, "batch handle is null");
    if (!scenes || !cams || !cam_scene || !W || !H || !bg || !out_rgb || !out_alpha || !ws)
        return fail_b(VIS_ERR_INVALID_ARG, "null argument");
    if (n_images < 1 || n_scenes < 1) return fail_b(VIS_ERR_INVALID_ARG, "empty batch");
    if (b->lanes == 0)
        return render_fused(b, scenes, n_scenes, cams, cam_scene, W, H, n_images, bg, out_rgb, out_alpha, ws, ws_bytes,
                            opts, reinterpret_cast<cudaStream_t>(stream_));
    const size_t sb = status_bytes(n_images);
    if (ws_bytes <= sb) return fail_b(VIS_ERR_INVALID_ARG, "batch workspace too small");
    const size_t slice = ((ws_bytes - sb) / b->lanes) / 256 * 256;
    for (int i = 0; i < n_images; ++i)
        if (cam_scene[i] < 0 || cam_scene[i] >= n_scenes || !scenes[cam_scene[i]])
            return fail_b(VIS_ERR_INVALID_ARG, "cam_scene out of range");
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    char* w = static_cast<char*>(ws);

    // arguments that the captured graph depends on
    std::vector<unsigned char> key;
    vis_render_opts o;
    vis_default_opts(&o);
    if (opts) o = *opts;
    append(key, &o, sizeof(o));
    append(key, &ws, sizeof(ws));
    append(key, &ws_bytes, sizeof(ws_bytes));
    append(key, bg, 3 * sizeof(float));
    append(key, &n_images, sizeof(n_images));
    for (int i = 0; i < n_images; ++i) {
        append(key, &cams[i], sizeof(vis_camera));
        append(key, &W[i], sizeof(int));
        append(key, &H[i], sizeof(int));
        append(key, &out_rgb[i], sizeof(float*));
        append(key, &out_alpha[i], sizeof(float*));
        vis::append_scene_key(key, scenes[cam_scene[i]]);
    }
    if (!b->exec || key != b->key) {
        // validate every image before capturing (errors cannot be returned from inside)
        for (int i = 0; i < n_images; ++i) {
            vis_ws_layout L;
            vis_status st = vis_workspace_layout(vis::scene_size(scenes[cam_scene[i]]), W[i], H[i], slice, &o, &L);
            if (st) return st;
        }
        const Plan plan = make_plan(scenes, cam_scene, W, H, n_images, b->lanes, slice);
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return fail_b(VIS_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
        vis_status st = VIS_OK;
        cudaEventRecord(b->fork_ev, b->origin);
        for (int l = 0; l < b->lanes; ++l) cudaStreamWaitEvent(b->streams[l], b->fork_ev, 0);
        for (int l = 0; l < b->lanes && st == VIS_OK; ++l) {
            char* sw = w + sb + (size_t)l * slice;
            for (int i : plan.order[l]) {
                st = vis_render(scenes[cam_scene[i]], &cams[i], W[i], H[i], bg, out_rgb[i], out_alpha[i], sw, slice,
                                &o, b->streams[l]);
                if (st) break;
                vis::copy_status_kernel<<<1, 1, 0, b->streams[l]>>>(reinterpret_cast<const vis::Ctrl*>(sw),
                                                                   reinterpret_cast<uint32_t*>(w) + 2 * i);
            }
        }
        for (int l = 0; l < b->lanes; ++l) {
            cudaEventRecord(b->join_ev[l], b->streams[l]);
            cudaStreamWaitEvent(b->origin, b->join_ev[l], 0);
        }
        e = cudaStreamEndCapture(b->origin, &graph);
        if (st) { if (graph) cudaGraphDestroy(graph); return st; }
        if (e != cudaSuccess) return fail_b(VIS_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { b->exec = nullptr; return fail_b(VIS_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e)); }
        b->key = key;
    }
    // order the graph after the caller's prior work and the caller's later work after it
    cudaError_t e = cudaEventRecord(b->in_ev, stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->in_ev, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->origin);
    if (e == cudaSuccess) e = cudaEventRecord(b->out_ev, b->origin);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, b->out_ev, 0);
    if (e != cudaSuccess) return fail_b(VIS_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    vis::set_last_error("");
    return VIS_OK;
}

vis_status vis_batch_check(const void* ws, int n_images, void* stream_, int64_t* max_keys) {
    if (!ws || n_images < 1) return fail_b(VIS_ERR_INVALID_ARG, "null workspace or empty batch");
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail_b(VIS_ERR_CUDA, cudaGetErrorString(e));
    std::vector<uint32_t> st(2 * (size_t)n_images);
    e = cudaMemcpy(st.data(), ws, st.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_b(VIS_ERR_CUDA, cudaGetErrorString(e));
    uint32_t mk = 0, err = 0;
    for (int i = 0; i < n_images; ++i) {
        if (st[2 * i] > mk) mk = st[2 * i];
        err |= st[2 * i + 1];
    }
    if (max_keys) *max_keys = mk;
    if (err & vis::kErrCapacity)
        return fail_b(VIS_ERR_CAPACITY, "an image of the batch produced more keys than its workspace slice holds");
    if (err & vis::kErrTimeout) return fail_b(VIS_ERR_TIMEOUT, "a device spin wait timed out");
    vis::set_last_error("");
    return VIS_OK;
}

}  // extern "C"
