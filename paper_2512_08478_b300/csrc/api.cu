// C ABI of libvis (declared in include/vis.h): argument validation, workspace
// layout, and the per-frame launch sequence of Algorithm 1 re-planned for one GPU:
//   clear status/histograms -> preprocess -> scan + duplicate keys -> radix sort
//   -> tile ranges -> composite            (vis_render)
//   composite adjoint -> preprocess adjoint (vis_render_backward)
// Nothing here allocates device memory; every launch goes on the caller's stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "vis_internal.cuh"

struct vis_scene {
    const float* means;
    const float* log_scales;
    const float* quats;
    const float* logits;
    const float* sh;
    int deg;
    int64_t n;
    // pre-packed fp16 planes (vis_scene_upload_packed); null for an fp32 scene
    const uint32_t* pk_pos;
    const uint32_t* pk_cov;
    const uint32_t* pk_col;
};

namespace {

thread_local std::string g_err;

vis_status fail(vis_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

vis_status cuda_check(cudaError_t e, const char* what) {
    if (e != cudaSuccess) return fail(VIS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return VIS_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int ceil_log2(int64_t v) {
    int b = 0;
    while (((int64_t)1 << b) < v) ++b;
    return b;
}

vis_render_opts resolve_opts(const vis_render_opts* o) {
    vis_render_opts r;
    vis_default_opts(&r);
    if (o) r = *o;
    if (r.tile == 0) r.tile = 16;
    if (r.digit_bits == 0) r.digit_bits = vis::kRadixBits;
    if (r.pixels_per_thread == 0) r.pixels_per_thread = 1;
    return r;
}

vis_status check_opts(const vis_render_opts& o) {
    if (o.tile != 8 && o.tile != 16 && o.tile != 32) return fail(VIS_ERR_INVALID_ARG, "tile must be 8, 16 or 32 (got %d)", o.tile);
    if (o.digit_bits != 8 && o.digit_bits != 10 && o.digit_bits != 11)
        return fail(VIS_ERR_UNSUPPORTED, "digit_bits must be 8, 10 or 11 (got %d)", o.digit_bits);
    if (o.tile_extent < 0 || o.tile_extent > 2)
        return fail(VIS_ERR_INVALID_ARG, "tile_extent must be 0, 1 or 2 (got %d)", o.tile_extent);
    if (o.pixels_per_thread != 1 && o.pixels_per_thread != 2)
        return fail(VIS_ERR_INVALID_ARG, "pixels_per_thread must be 1 or 2 (got %d)", o.pixels_per_thread);
    if (o.sort_mode != vis::kSortTileDepth && o.sort_mode != vis::kSortDepthFirst)
        return fail(VIS_ERR_INVALID_ARG, "sort_mode must be 0 or 1 (got %d)", o.sort_mode);
    if (!(o.dilation >= 0.f) || !std::isfinite(o.dilation)) return fail(VIS_ERR_INVALID_ARG, "dilation must be finite and >= 0");
    if (!(o.alpha_min > 0.f && o.alpha_min < 1.f)) return fail(VIS_ERR_INVALID_ARG, "alpha_min must be in (0, 1)");
    if (!(o.alpha_max > 0.f && o.alpha_max < 1.f)) return fail(VIS_ERR_INVALID_ARG, "alpha_max must be in (0, 1)");
    if (!(o.t_stop >= 0.f && o.t_stop < 1.f)) return fail(VIS_ERR_INVALID_ARG, "t_stop must be in [0, 1)");
    if (o.spin_limit < 0 || (uint32_t)o.spin_limit > vis::kMaxSpinLimit)
        return fail(VIS_ERR_INVALID_ARG, "spin_limit must be in [0, 2^30] (got %d)", o.spin_limit);
    return VIS_OK;
}

vis_status check_size(int64_t n, int W, int H) {
    if (n < 1 || n > 0x7fffffffLL) return fail(VIS_ERR_INVALID_ARG, "n must be in [1, 2^31-1] (got %lld)", (long long)n);
    if (W < 1 || H < 1 || W > 16384 || H > 16384) return fail(VIS_ERR_INVALID_ARG, "W, H must be in [1, 16384] (got %d x %d)", W, H);
    return VIS_OK;
}

vis_status check_camera(const vis_camera* c) {
    if (!c) return fail(VIS_ERR_INVALID_ARG, "camera is null");
    const float* f = reinterpret_cast<const float*>(c);
    for (int k = 0; k < 17; ++k)
        if (!std::isfinite(f[k])) return fail(VIS_ERR_INVALID_ARG, "camera has a non-finite value");
    if (!(c->fx > 0.f && c->fy > 0.f)) return fail(VIS_ERR_INVALID_ARG, "fx, fy must be > 0");
    if (!(c->near_z > 0.f)) return fail(VIS_ERR_INVALID_ARG, "near_z must be > 0");
    return VIS_OK;
}

// Preprocess parameters for one view (camera centre and guard limits in double).
vis::PrepParams make_params(const vis_scene* s, const vis_camera* c, int W, int H, const vis::Layout& L,
                            const vis_render_opts& o) {
    vis::PrepParams p;
    std::memset(&p, 0, sizeof(p));
    p.means = s->means; p.log_scales = s->log_scales; p.quats = s->quats; p.logits = s->logits; p.sh = s->sh;
    p.pk_pos = reinterpret_cast<const uint2*>(s->pk_pos); p.pk_cov = s->pk_cov; p.pk_col = s->pk_col;
    p.col_words = vis::packed_col_words(s->deg);
    p.deg = s->deg; p.n = (int)s->n; p.n_pad = (int)s->n; p.index_offset = 0;
    for (int k = 0; k < 9; ++k) p.R[k] = c->R[k];
    for (int k = 0; k < 3; ++k) p.t[k] = c->t[k];
    p.fx = c->fx; p.fy = c->fy; p.cx = c->cx; p.cy = c->cy; p.near_z = c->near_z;
    for (int j = 0; j < 3; ++j) {
        double a = 0;
        for (int r = 0; r < 3; ++r) a -= (double)c->R[3 * r + j] * (double)c->t[r];
        p.cam_pos[j] = (float)a;
    }
    p.limx = (float)(1.3 * (W / (2.0 * c->fx)));
    p.limy = (float)(1.3 * (H / (2.0 * c->fy)));
    p.W = W; p.H = H; p.tile = L.tile; p.tiles_x = L.tiles_x; p.tiles_y = L.tiles_y;
    p.dilation = o.dilation; p.alpha_min = o.alpha_min;
    p.wscale = (float)std::sqrt(0.5 / std::log(2.0));
    p.tight_extent = o.tile_extent;
    p.count_survivors = L.mode == vis::kSortDepthFirst;
    vis::sh_constants(p.shc);
    return p;
}

constexpr int kMaxScenes = 1 << 16;   // scenes per multi-scene render

// adjugate and determinant of a 3x3 row-major matrix
double adjugate3(const double A[9], double adj[9]) {
    adj[0] = A[4] * A[8] - A[5] * A[7]; adj[1] = A[2] * A[7] - A[1] * A[8]; adj[2] = A[1] * A[5] - A[2] * A[4];
    adj[3] = A[5] * A[6] - A[3] * A[8]; adj[4] = A[0] * A[8] - A[2] * A[6]; adj[5] = A[2] * A[3] - A[0] * A[5];
    adj[6] = A[3] * A[7] - A[4] * A[6]; adj[7] = A[1] * A[6] - A[0] * A[7]; adj[8] = A[0] * A[4] - A[1] * A[3];
    return A[0] * adj[0] + A[1] * adj[3] + A[2] * adj[6];
}

// A model transform [A | b] (row-major 3x4) must be finite with A invertible.
vis_status check_model(const float* m, int k) {
    for (int j = 0; j < 12; ++j)
        if (!std::isfinite(m[j])) return fail(VIS_ERR_INVALID_ARG, "model %d has a non-finite value", k);
    double A[9], adj[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) A[3 * r + c] = m[4 * r + c];
    const double det = adjugate3(A, adj);
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return fail(VIS_ERR_INVALID_ARG, "model %d is singular", k);
    for (int j = 0; j < 9; ++j)
        if (!std::isfinite(adj[j] / det)) return fail(VIS_ERR_INVALID_ARG, "model %d is singular", k);
    return VIS_OK;
}

// Fold a model transform M = [A | b] into the view (Algorithm 1: x_w = M [mu; 1], then the
// camera): x_c = R (A mu + b) + t = (R A) mu + (R b + t). R A and R b + t are formed in double
// and stored as float pairs (value + residue). The SH ray starts at the camera centre seen
// from the model, A^-1 (c - b) with c = -R^T t, so colours are evaluated in the model's frame.
void fold_model(vis::PrepParams& p, const vis_camera* c, const float* m) {
    double A[9], b[3], R[9], t[3], adj[9];
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) { A[3 * r + k] = m[4 * r + k]; R[3 * r + k] = c->R[3 * r + k]; }
        b[r] = m[4 * r + 3];
        t[r] = c->t[r];
    }
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) {
            const double v = R[3 * r + 0] * A[k] + R[3 * r + 1] * A[3 + k] + R[3 * r + 2] * A[6 + k];
            p.R[3 * r + k] = (float)v;
            p.R_lo[3 * r + k] = (float)(v - (double)p.R[3 * r + k]);
        }
        const double v = R[3 * r + 0] * b[0] + R[3 * r + 1] * b[1] + R[3 * r + 2] * b[2] + t[r];
        p.t[r] = (float)v;
        p.t_lo[r] = (float)(v - (double)p.t[r]);
    }
    const double det = adjugate3(A, adj);
    double w[3];
    for (int j = 0; j < 3; ++j) w[j] = -(R[j] * t[0] + R[3 + j] * t[1] + R[6 + j] * t[2]) - b[j];
    for (int r = 0; r < 3; ++r)
        p.cam_pos[r] = (float)((adj[3 * r] * w[0] + adj[3 * r + 1] * w[1] + adj[3 * r + 2] * w[2]) / det);
}

// Workspace slots of a list of scenes: each scene starts at a multiple of kPrepThreads
// (its Gaussians fill whole preprocess blocks) when `padded`, else the scene's own size.
int64_t scene_slots(const vis_scene* const* scenes, int n_scenes, bool padded, int64_t* offsets) {
    int64_t off = 0;
    for (int k = 0; k < n_scenes; ++k) {
        if (offsets) offsets[k] = off;
        const int64_t n = scenes[k]->n;
        off += padded ? (n + vis::kPrepThreads - 1) / vis::kPrepThreads * vis::kPrepThreads : n;
    }
    return off;
}

// ---- per-stage profiling (vis_profile_begin / vis_profile_end) ----
constexpr int kProfStages = 8;
constexpr int kProfRing = 1024;
struct Profiler {
    bool on = false;
    int count = 0;
    int passes = 0;
    cudaEvent_t ev[kProfRing][kProfStages + 1];
    bool created = false;
};
Profiler g_prof;

// Record event `k` (0 = start, k = end of stage k-1) of the current render.
void prof_mark(int k, cudaStream_t stream) {
    if (!g_prof.on || g_prof.count >= kProfRing) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    cudaEventRecord(g_prof.ev[g_prof.count][k], stream);
}

// Marks k and k + 1 (an empty stage k): the 64-bit key sort has no tile-count stage.
void prof_mark_twice(int k, cudaStream_t stream) {
    prof_mark(k, stream);
    prof_mark(k + 1, stream);
}

}  // namespace

namespace vis {

void set_last_error(const char* msg) { g_err = msg ? msg : ""; }

bool pdl_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("VIS_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

int64_t scene_size(vis_scene_t s) { return s ? s->n : 0; }

void append_scene_key(std::vector<unsigned char>& key, vis_scene_t s) {
    const unsigned char* c = reinterpret_cast<const unsigned char*>(s);
    key.insert(key.end(), c, c + sizeof(vis_scene));
}

vis_status batch_opts(const vis_render_opts* in, vis_render_opts* out) {
    *out = resolve_opts(in);
    return check_opts(*out);
}

vis_status batch_item(vis_scene_t s, const vis_camera* cam, int W, int H, const vis_render_opts& o, int64_t slot0,
                      uint32_t image, PrepParams* out) {
    if (!s) return fail(VIS_ERR_INVALID_ARG, "scene of image %u is null", image);
    vis_status st = check_size(s->n, W, H);
    if (st) return st;
    if ((st = check_camera(cam))) return st;
    const Layout L = make_layout(1, W, H, o.tile, 1, kSortDepthFirst, o.digit_bits);
    *out = make_params(s, cam, W, H, L, o);
    out->index_offset = slot0;
    out->n_pad = (int)((s->n + kPrepThreads - 1) / kPrepThreads * kPrepThreads);
    out->batch_image = image;
    return VIS_OK;
}

bool scene_packed(vis_scene_t s) { return s && s->pk_pos != nullptr; }

QScale q_scale() {
    const double c = 0.5 / std::log(2.0);   // log2(e) / 2
    return QScale{(float)(9.0 * c), (float)(1.0 / c)};
}

// K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!); the real SH polynomials in (x, y, z)
// on the unit sphere (Condon-Shortley phase) are products of these with
// (-1)^m d^m P_l/dz^m and Re/Im (x + i y)^m, so the constants below are:
//   [0] K_1^0             [1] sqrt2 K_1^1
//   [2] K_2^0 / 2         [3] 3 sqrt2 K_2^1     [4] 3 sqrt2 K_2^2
//   [5] K_3^0 / 2         [6] 3/2 sqrt2 K_3^1   [7] 15 sqrt2 K_3^2   [8] 15 sqrt2 K_3^3
//   [9] K_0^0
void sh_constants(float out[12]) {
    auto fact = [](int n) { double f = 1; for (int k = 2; k <= n; ++k) f *= k; return f; };
    const double pi = 3.14159265358979323846;
    auto K = [&](int l, int m) { return std::sqrt((2.0 * l + 1.0) / (4.0 * pi) * fact(l - m) / fact(l + m)); };
    const double r2 = std::sqrt(2.0);
    out[0] = (float)K(1, 0);
    out[1] = (float)(r2 * K(1, 1));
    out[2] = (float)(K(2, 0) / 2.0);
    out[3] = (float)(3.0 * r2 * K(2, 1));
    out[4] = (float)(3.0 * r2 * K(2, 2));
    out[5] = (float)(K(3, 0) / 2.0);
    out[6] = (float)(1.5 * r2 * K(3, 1));
    out[7] = (float)(15.0 * r2 * K(3, 2));
    out[8] = (float)(15.0 * r2 * K(3, 3));
    out[9] = (float)K(0, 0);
    out[10] = out[11] = 0.f;
}

Layout make_layout(int64_t n, int W, int H, int tile, int64_t cap, int mode, int digit_bits) {
    Layout L;
    L.n = n; L.W = W; L.H = H; L.tile = tile;
    L.tiles_x = (W + tile - 1) / tile;
    L.tiles_y = (H + tile - 1) / tile;
    L.ntiles = (int64_t)L.tiles_x * L.tiles_y;
    L.mode = mode;
    L.tile_bits = ceil_log2(L.ntiles);
    L.cap = cap;
    L.prep_blocks = (n + kPrepThreads - 1) / kPrepThreads;
    const bool df = mode == kSortDepthFirst;
    // the digit width applies to the 32-bit sorts of the depth-first order (the depth sort
    // and a tile sort of 32-bit ids); the 64-bit keys of sort_mode 0 and the 16-bit tile ids
    // always take 8-bit digits
    L.digit_bits = df ? digit_bits : kRadixBits;
    L.depth_passes = df ? passes_for(32, L.digit_bits) : 0;
    L.key_bits = df ? L.tile_bits : 32 + L.tile_bits;
    L.passes = passes_for(L.key_bits, L.digit_bits);
    L.key_bytes = df ? 4 : 8;
    L.sort_parts = df ? (cap + (int64_t)kSortThreads * 16 - 1) / ((int64_t)kSortThreads * 16)
                      : sort_parts<uint64_t>(cap);
    L.sorted_buffer = L.passes & 1;
    // depth-first mode: counts-first tile sort of 16-bit tile keys when the per-tile counters
    // fit in shared memory; it runs at least one pass (the last writes values only)
    L.tile_fused = mode == kSortDepthFirst && L.ntiles <= kTileFusedMaxTiles;
    int tile_digit = L.digit_bits;
    if (L.tile_fused) {
        L.passes = L.tile_bits > kRadixBits ? 2 : 1;
        L.key_bytes = 2;
        L.sort_parts = sort_parts<uint16_t>(cap);
        L.sorted_buffer = L.passes & 1;
        tile_digit = kRadixBits;
    }
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    // cleared every frame: status block, histograms, look-back words, tile ranges
    L.zero_begin = off;
    L.off_ctrl = take(sizeof(Ctrl));
    L.off_hist = take(sizeof(uint32_t) * kMaxPasses * ((size_t)1 << L.digit_bits));
    L.off_hist_tile = take(sizeof(uint32_t) * kMaxPasses * ((size_t)1 << tile_digit));
    L.lookback_words_depth =
        df ? (size_t)L.depth_passes * lookback_rows(depth_sort_parts(n, L.digit_bits), lookback_group(4, L.digit_bits)) *
                 ((size_t)1 << L.digit_bits)
           : 0;
    const int tile_group = lookback_group(L.tile_fused ? 2 : L.key_bytes, tile_digit);
    const size_t tile_lb_words = (size_t)L.passes * lookback_rows(L.sort_parts, tile_group) * ((size_t)1 << tile_digit);
    L.off_lookback = take(sizeof(uint32_t) * (L.lookback_words_depth + (L.tile_fused ? 0 : tile_lb_words)));
    if (!L.tile_fused) L.off_lookback_tile = L.off_lookback + sizeof(uint32_t) * L.lookback_words_depth;
    L.off_ranges = take(sizeof(uint2) * (size_t)L.ntiles);
    if (L.tile_fused) L.off_tdiff = take(sizeof(int) * (size_t)L.ntiles);
    L.scan_slot_words = scan_parts(L.prep_blocks);
    L.off_scan_lb = take(sizeof(unsigned long long) * 2 * (size_t)L.scan_slot_words);
    L.zero_end = off;
    if (L.tile_fused) {
        L.off_order = take(sizeof(uint32_t) * (size_t)L.ntiles);
        L.off_lookback_tile = take(sizeof(uint32_t) * tile_lb_words);
    }
    L.off_rec = take(sizeof(float4) * 3 * (size_t)n);
    L.off_depth = take(sizeof(float) * (size_t)n);
    L.off_rect = take(sizeof(uint4) * (size_t)n);
    L.off_touched = take(sizeof(uint32_t) * (size_t)n);
    L.off_bsum = take(sizeof(uint32_t) * (size_t)L.prep_blocks);
    L.off_boff = take(sizeof(uint32_t) * (size_t)L.prep_blocks);
    if (df) {
        L.off_bsum2 = take(sizeof(uint32_t) * (size_t)L.prep_blocks);
        L.off_boff2 = take(sizeof(uint32_t) * (size_t)L.prep_blocks);
        for (int b = 0; b < 2; ++b) L.off_dkeys[b] = take(sizeof(uint32_t) * (size_t)n);
        for (int b = 0; b < 2; ++b) L.off_dvals[b] = take(sizeof(uint32_t) * (size_t)n);
    }

    L.off_keys[0] = take((size_t)L.key_bytes * (size_t)cap);
    L.off_keys[1] = take((size_t)L.key_bytes * (size_t)cap);
    L.off_vals[0] = take(sizeof(uint32_t) * (size_t)cap);
    L.off_vals[1] = take(sizeof(uint32_t) * (size_t)cap);
    L.off_tfinal = take(sizeof(float) * (size_t)W * H);
    L.off_zmax = take(sizeof(float) * (size_t)L.ntiles);
    L.off_last = take(sizeof(int32_t) * (size_t)W * H);
    L.off_g2 = take(sizeof(float) * 9 * (size_t)n);
    L.total = off;
    return L;
}

int64_t capacity_for(int64_t n, int W, int H, int tile, int mode, size_t ws_bytes, int digit_bits) {
    if (make_layout(n, W, H, tile, 1, mode, digit_bits).total > ws_bytes) return 0;
    int64_t lo = 1, hi = kMaxKeys;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (make_layout(n, W, H, tile, mid, mode, digit_bits).total <= ws_bytes) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace vis

extern "C" {

void vis_default_opts(vis_render_opts* o) {
    if (!o) return;
    o->tile = 16;
    o->digit_bits = vis::kRadixBits;
    o->dilation = 0.3f;
    o->alpha_min = 1.0f / 255.0f;
    o->alpha_max = 0.99f;
    o->t_stop = 1e-4f;
    o->sort_mode = vis::kSortDepthFirst;
    o->pixels_per_thread = 1;
    o->tile_extent = 2;
    o->collect_stats = 0;
    o->spin_limit = 0;
}

const char* vis_last_error(void) { return g_err.c_str(); }

vis_status vis_scene_upload(const float* means, const float* log_scales, const float* quats,
                            const float* opacity_logits, const float* sh, int sh_degree, int64_t n,
                            vis_scene_t* out) {
    if (!out) return fail(VIS_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (sh_degree < 0 || sh_degree > 3) return fail(VIS_ERR_INVALID_ARG, "sh_degree must be 0..3 (got %d)", sh_degree);
    if (n < 1 || n > 0x7fffffffLL) return fail(VIS_ERR_INVALID_ARG, "n must be in [1, 2^31-1] (got %lld)", (long long)n);
    const void* ptrs[5] = {means, log_scales, quats, opacity_logits, sh};
    const char* names[5] = {"means", "log_scales", "quats", "opacity_logits", "sh"};
    for (int k = 0; k < 5; ++k) {
        if (!ptrs[k]) return fail(VIS_ERR_INVALID_ARG, "%s is null", names[k]);
        if (!aligned16(ptrs[k])) return fail(VIS_ERR_INVALID_ARG, "%s is not 16-byte aligned", names[k]);
    }
    vis_scene* s = new (std::nothrow) vis_scene;
    if (!s) return fail(VIS_ERR_INVALID_ARG, "out of host memory");
    std::memset(s, 0, sizeof(*s));
    s->means = means; s->log_scales = log_scales; s->quats = quats; s->logits = opacity_logits; s->sh = sh;
    s->deg = sh_degree; s->n = n;
    *out = s;
    g_err.clear();
    return VIS_OK;
}

vis_status vis_packed_size(int64_t n, int sh_degree, size_t* pos_bytes, size_t* cov_bytes, size_t* col_bytes) {
    if (sh_degree < 0 || sh_degree > 3) return fail(VIS_ERR_INVALID_ARG, "sh_degree must be 0..3 (got %d)", sh_degree);
    if (n < 1 || n > 0x7fffffffLL) return fail(VIS_ERR_INVALID_ARG, "n must be in [1, 2^31-1] (got %lld)", (long long)n);
    if (pos_bytes) *pos_bytes = 8 * (size_t)n;
    if (cov_bytes) *cov_bytes = 12 * (size_t)n;
    if (col_bytes) *col_bytes = 4 * (size_t)vis::packed_col_words(sh_degree) * (size_t)n;
    g_err.clear();
    return VIS_OK;
}

vis_status vis_scene_upload_packed(const void* pos, const void* cov, const void* col, int sh_degree, int64_t n,
                                   vis_scene_t* out) {
    if (!out) return fail(VIS_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    vis_status st = vis_packed_size(n, sh_degree, nullptr, nullptr, nullptr);
    if (st) return st;
    const void* ptrs[3] = {pos, cov, col};
    const char* names[3] = {"pos", "cov", "col"};
    for (int k = 0; k < 3; ++k) {
        if (!ptrs[k]) return fail(VIS_ERR_INVALID_ARG, "%s is null", names[k]);
        if (!aligned16(ptrs[k])) return fail(VIS_ERR_INVALID_ARG, "%s is not 16-byte aligned", names[k]);
    }
    vis_scene* s = new (std::nothrow) vis_scene;
    if (!s) return fail(VIS_ERR_INVALID_ARG, "out of host memory");
    std::memset(s, 0, sizeof(*s));
    s->pk_pos = static_cast<const uint32_t*>(pos);
    s->pk_cov = static_cast<const uint32_t*>(cov);
    s->pk_col = static_cast<const uint32_t*>(col);
    s->deg = sh_degree; s->n = n;
    *out = s;
    g_err.clear();
    return VIS_OK;
}

vis_status vis_scene_pack(vis_scene_t scene, void* pos, void* cov, void* col, void* stream_) {
    if (!scene) return fail(VIS_ERR_INVALID_ARG, "scene is null");
    if (scene->pk_pos) return fail(VIS_ERR_INVALID_ARG, "scene is already packed");
    const void* ptrs[3] = {pos, cov, col};
    for (int k = 0; k < 3; ++k)
        if (!ptrs[k] || !aligned16(ptrs[k])) return fail(VIS_ERR_INVALID_ARG, "packed plane %d null or misaligned", k);
    vis::launch_pack(scene->means, scene->log_scales, scene->quats, scene->logits, scene->sh, scene->deg, scene->n,
                     static_cast<uint2*>(pos), static_cast<uint32_t*>(cov), static_cast<uint32_t*>(col),
                     reinterpret_cast<cudaStream_t>(stream_));
    vis_status st = cuda_check(cudaGetLastError(), "launch");
    if (st) return st;
    g_err.clear();
    return VIS_OK;
}

void vis_scene_destroy(vis_scene_t s) { delete s; }

vis_status vis_workspace_size(int64_t n, int W, int H, int64_t key_capacity, const vis_render_opts* opts,
                              size_t* bytes) {
    if (!bytes) return fail(VIS_ERR_INVALID_ARG, "bytes is null");
    vis_status st = check_size(n, W, H);
    if (st) return st;
    const vis_render_opts o = resolve_opts(opts);
    if ((st = check_opts(o))) return st;
    if (key_capacity < 1 || key_capacity > (int64_t)vis::kMaxKeys)
        return fail(VIS_ERR_INVALID_ARG, "key_capacity must be in [1, 2^30-1]");
    *bytes = vis::make_layout(n, W, H, o.tile, key_capacity, o.sort_mode, o.digit_bits).total;
    return VIS_OK;
}

vis_status vis_workspace_layout(int64_t n, int W, int H, size_t ws_bytes, const vis_render_opts* opts,
                                vis_ws_layout* out) {
    if (!out) return fail(VIS_ERR_INVALID_ARG, "out is null");
    vis_status st = check_size(n, W, H);
    if (st) return st;
    const vis_render_opts o = resolve_opts(opts);
    if ((st = check_opts(o))) return st;
    const int64_t cap = vis::capacity_for(n, W, H, o.tile, o.sort_mode, ws_bytes, o.digit_bits);
    if (cap < 1) return fail(VIS_ERR_INVALID_ARG, "workspace of %zu bytes holds no keys", ws_bytes);
    const vis::Layout L = vis::make_layout(n, W, H, o.tile, cap, o.sort_mode, o.digit_bits);
    out->total_bytes = L.total;
    out->key_capacity = L.cap;
    out->tiles_x = L.tiles_x; out->tiles_y = L.tiles_y;
    out->sort_passes = L.passes; out->sorted_buffer = L.sorted_buffer;
    out->off_ctrl = L.off_ctrl; out->off_rec = L.off_rec; out->off_depth = L.off_depth;
    out->off_rect = L.off_rect; out->off_touched = L.off_touched;
    out->off_keys[0] = L.off_keys[0]; out->off_keys[1] = L.off_keys[1];
    out->off_vals[0] = L.off_vals[0]; out->off_vals[1] = L.off_vals[1];
    out->off_ranges = L.off_ranges; out->off_tfinal = L.off_tfinal; out->off_last = L.off_last;
    out->off_order = L.tile_fused ? L.off_order : 0;
    out->off_g2 = L.off_g2;
    out->key_bytes = L.key_bytes;
    out->sort_mode = L.mode;
    return VIS_OK;
}

// Validates a render's arguments for a list of scenes and lays out the workspace over their
// slots (a single scene: its own n; several: each padded to whole preprocess blocks).
static vis_status prepare(const vis_scene_t* scenes, int n_scenes, bool padded, const float* models,
                          const vis_camera* cam, int W, int H, const float bg[3], void* ws, size_t ws_bytes,
                          const vis_render_opts* opts, vis_render_opts* o, vis::Layout* L,
                          std::vector<int64_t>* offsets) {
    if (!scenes) return fail(VIS_ERR_INVALID_ARG, "scenes is null");
    if (n_scenes < 1 || n_scenes > kMaxScenes)
        return fail(VIS_ERR_INVALID_ARG, "n_scenes must be in [1, %d] (got %d)", kMaxScenes, n_scenes);
    for (int k = 0; k < n_scenes; ++k) {
        if (!scenes[k]) return fail(VIS_ERR_INVALID_ARG, "scene %d is null", k);
        if (models) {
            vis_status st = check_model(models + 12 * (size_t)k, k);
            if (st) return st;
        }
    }
    offsets->assign(n_scenes, 0);
    const int64_t slots = scene_slots(scenes, n_scenes, padded, offsets->data());
    vis_status st = check_size(slots, W, H);
    if (st) return st;
    if ((st = check_camera(cam))) return st;
    if (!bg) return fail(VIS_ERR_INVALID_ARG, "bg is null");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(bg[k])) return fail(VIS_ERR_INVALID_ARG, "bg is not finite");
    *o = resolve_opts(opts);
    if ((st = check_opts(*o))) return st;
    if (!ws || !aligned16(ws)) return fail(VIS_ERR_INVALID_ARG, "workspace is null or not 16-byte aligned");
    const int64_t cap = vis::capacity_for(slots, W, H, o->tile, o->sort_mode, ws_bytes, o->digit_bits);
    if (cap < 1) return fail(VIS_ERR_INVALID_ARG, "workspace of %zu bytes holds no keys", ws_bytes);
    *L = vis::make_layout(slots, W, H, o->tile, cap, o->sort_mode, o->digit_bits);
    L->spin_limit = o->spin_limit > 0 ? (uint32_t)o->spin_limit : vis::kSpinLimit;
    return VIS_OK;
}

// Preprocess parameters of scene k of a (multi-)scene render.
static vis::PrepParams scene_params(const vis_scene_t* scenes, const float* models, int k, bool padded,
                                    const std::vector<int64_t>& offsets, const vis_camera* cam, int W, int H,
                                    const vis::Layout& L, const vis_render_opts& o) {
    vis::PrepParams p = make_params(scenes[k], cam, W, H, L, o);
    p.index_offset = offsets[k];
    if (padded) p.n_pad = (int)((scenes[k]->n + vis::kPrepThreads - 1) / vis::kPrepThreads * vis::kPrepThreads);
    if (models) fold_model(p, cam, models + 12 * (size_t)k);
    return p;
}

// The per-frame update arrays of a dynamic frame (vis_render_dynamic).
struct DynFrame {
    const float* velocity;
    const float* amp;
    const float* freq;
    const float* phase;
    float t;
};

// One image of one or more scenes: every scene is preprocessed into its slots (with its
// model transform folded into the view), then one global sort and one compositing pass run
// over all slots (Algorithm 1). dyn: a dynamic frame of the one scene (else null).
static vis_status render_impl(const vis_scene_t* scenes, const float* models, int n_scenes, bool padded,
                              const vis_camera* cam, int W, int H, const float bg[3],
                              const float* zlim, float* out_rgb, float* out_alpha, void* ws, size_t ws_bytes,
                              const vis_render_opts* opts, void* stream_, const DynFrame* dyn = nullptr) {
    vis_render_opts o;
    vis::Layout L;
    std::vector<int64_t> offsets;
    vis_status st = prepare(scenes, n_scenes, padded, models, cam, W, H, bg, ws, ws_bytes, opts, &o, &L, &offsets);
    if (st) return st;
    if (!out_rgb || !out_alpha || !aligned16(out_rgb) || !aligned16(out_alpha))
        return fail(VIS_ERR_INVALID_ARG, "out_rgb / out_alpha null or not 16-byte aligned");
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    char* w = static_cast<char*>(ws);
    prof_mark(0, stream);
    if ((st = cuda_check(cudaMemsetAsync(w + L.zero_begin, 0, L.zero_end - L.zero_begin, stream), "clear workspace")))
        return st;
    prof_mark(1, stream);
    if (zlim) vis::launch_tile_zmax(L, w, zlim, stream);
    for (int k = 0; k < n_scenes; ++k) {
        vis::PrepParams p = scene_params(scenes, models, k, padded, offsets, cam, W, H, L, o);
        if (zlim) p.tile_zmax = reinterpret_cast<const float*>(w + L.off_zmax);
        if (dyn) {
            p.dyn_velocity = dyn->velocity; p.dyn_amp = dyn->amp; p.dyn_freq = dyn->freq; p.dyn_phase = dyn->phase;
            p.dyn_t = dyn->t;
            p.dyn_flags = &reinterpret_cast<vis::Ctrl*>(w + L.off_ctrl)->flags;
        }
        vis::launch_preprocess(p, L, w, stream);
    }
    prof_mark(2, stream);
    if (L.mode == vis::kSortDepthFirst) {
        // marks 3 (after the depth sort), 4 (after the emission), 5 (after the tile counts or
        // the tile histogram)
        vis::launch_depth_first(L, w, stream, g_prof.on ? &prof_mark : nullptr, 3);
        prof_mark(6, stream);
        if (!L.tile_fused) vis::launch_ranges32(L, w, stream);   // the counts-first tile sort wrote them
    } else {
        vis::launch_scan_and_duplicate(L, w, L.n, stream);
        prof_mark(3, stream);
        vis::launch_sort(L, w, stream, g_prof.on ? &prof_mark_twice : nullptr, 4);
        prof_mark(6, stream);
        vis::launch_ranges(L, w, stream);
    }
    prof_mark(7, stream);
    vis::launch_composite(L, w, bg[0], bg[1], bg[2], o.alpha_min, o.alpha_max, o.t_stop, o.pixels_per_thread,
                          o.collect_stats != 0, out_rgb, out_alpha, zlim, stream);
    prof_mark(8, stream);
    if (g_prof.on && g_prof.count < kProfRing) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
            ++g_prof.count;
            g_prof.passes = L.passes;
        }
    }
    if ((st = cuda_check(cudaGetLastError(), "launch"))) return st;
    g_err.clear();
    return VIS_OK;
}

vis_status vis_render(vis_scene_t scene, const vis_camera* cam, int W, int H, const float bg[3], float* out_rgb,
                      float* out_alpha, void* ws, size_t ws_bytes, const vis_render_opts* opts, void* stream_) {
    return render_impl(&scene, nullptr, 1, false, cam, W, H, bg, nullptr, out_rgb, out_alpha, ws, ws_bytes, opts,
                       stream_);
}

vis_status vis_render_dynamic(vis_scene_t scene, const float* velocity, const float* amp, const float* freq,
                              const float* phase, float t, const vis_camera* cam, int W, int H, const float bg[3],
                              float* out_rgb, float* out_alpha, void* ws, size_t ws_bytes,
                              const vis_render_opts* opts, void* stream_) {
    if (!scene) return fail(VIS_ERR_INVALID_ARG, "scene is null");
    if (scene->pk_pos) return fail(VIS_ERR_UNSUPPORTED, "a pre-packed scene has no fp32 frame-0 attributes to update");
    if (!std::isfinite(t)) return fail(VIS_ERR_INVALID_ARG, "t is not finite");
    const void* ptrs[4] = {velocity, amp, freq, phase};
    for (int k = 0; k < 4; ++k)
        if (!ptrs[k] || !aligned16(ptrs[k])) return fail(VIS_ERR_INVALID_ARG, "dynamic array %d null or misaligned", k);
    const DynFrame dyn = {velocity, amp, freq, phase, t};
    return render_impl(&scene, nullptr, 1, false, cam, W, H, bg, nullptr, out_rgb, out_alpha, ws, ws_bytes, opts,
                       stream_, &dyn);
}

vis_status vis_render_depth(vis_scene_t scene, const vis_camera* cam, int W, int H, const float bg[3],
                            const float* depth, float* out_rgb, float* out_alpha, void* ws, size_t ws_bytes,
                            const vis_render_opts* opts, void* stream_) {
    if (!depth || !aligned16(depth)) return fail(VIS_ERR_INVALID_ARG, "depth buffer null or not 16-byte aligned");
    return render_impl(&scene, nullptr, 1, false, cam, W, H, bg, depth, out_rgb, out_alpha, ws, ws_bytes, opts,
                       stream_);
}

vis_status vis_multi_slots(const vis_scene_t* scenes, int n_scenes, int64_t* slots) {
    if (!slots) return fail(VIS_ERR_INVALID_ARG, "slots is null");
    if (!scenes) return fail(VIS_ERR_INVALID_ARG, "scenes is null");
    if (n_scenes < 1 || n_scenes > kMaxScenes)
        return fail(VIS_ERR_INVALID_ARG, "n_scenes must be in [1, %d] (got %d)", kMaxScenes, n_scenes);
    for (int k = 0; k < n_scenes; ++k)
        if (!scenes[k]) return fail(VIS_ERR_INVALID_ARG, "scene %d is null", k);
    *slots = scene_slots(scenes, n_scenes, true, nullptr);
    if (*slots > 0x7fffffffLL) return fail(VIS_ERR_INVALID_ARG, "the scenes hold more than 2^31-1 slots");
    g_err.clear();
    return VIS_OK;
}

vis_status vis_render_multi(const vis_scene_t* scenes, const float* models, int n_scenes, const vis_camera* cam,
                            int W, int H, const float bg[3], const float* depth, float* out_rgb, float* out_alpha,
                            void* ws, size_t ws_bytes, const vis_render_opts* opts, void* stream_) {
    if (depth && !aligned16(depth)) return fail(VIS_ERR_INVALID_ARG, "depth buffer not 16-byte aligned");
    return render_impl(scenes, models, n_scenes, true, cam, W, H, bg, depth, out_rgb, out_alpha, ws, ws_bytes, opts,
                       stream_);
}

vis_status vis_check(const void* ws, void* stream_, int64_t* num_keys) {
    if (!ws) return fail(VIS_ERR_INVALID_ARG, "workspace is null");
    vis::Ctrl c;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    vis_status st = cuda_check(cudaStreamSynchronize(stream), "synchronize");
    if (st) return st;
    if ((st = cuda_check(cudaMemcpy(&c, ws, sizeof(c), cudaMemcpyDeviceToHost), "read status"))) return st;
    if (num_keys) *num_keys = c.num_keys;
    if (c.error & vis::kErrCapacity)
        return fail(VIS_ERR_CAPACITY, "%u keys exceed the workspace capacity", c.num_keys);
    if (c.error & vis::kErrTimeout) return fail(VIS_ERR_TIMEOUT, "a device spin wait timed out");
    if (c.error & vis::kErrNoAdjoint)
        return fail(VIS_ERR_UNSUPPORTED, "no adjoint of a dynamic frame: its updated attributes were never stored "
                                         "(update the scene with vis_dynamic_update and render it with vis_render)");
    g_err.clear();
    return VIS_OK;
}

// Adjoint of render_impl: the compositing adjoint over all slots, then each scene's
// preprocess adjoint into its own gradient buffers.
static vis_status backward_impl(const vis_scene_t* scenes, const float* models, int n_scenes, bool padded,
                                const vis_camera* cam, int W, int H, const float bg[3], const float* zlim,
                                const float* d_rgb, const float* d_alpha, void* ws, size_t ws_bytes,
                                const vis_render_opts* opts, const vis_scene_grads* grads, void* stream_) {
    vis_render_opts o;
    vis::Layout L;
    std::vector<int64_t> offsets;
    vis_status st = prepare(scenes, n_scenes, padded, models, cam, W, H, bg, ws, ws_bytes, opts, &o, &L, &offsets);
    if (st) return st;
    if (!d_rgb || !d_alpha || !aligned16(d_rgb) || !aligned16(d_alpha))
        return fail(VIS_ERR_INVALID_ARG, "d_rgb / d_alpha null or not 16-byte aligned");
    if (!grads) return fail(VIS_ERR_INVALID_ARG, "grads is null");
    for (int k = 0; k < n_scenes; ++k)
        if (scenes[k]->pk_pos)
            return fail(VIS_ERR_UNSUPPORTED, "scene %d is pre-packed (fp16): it has no parameter gradients", k);
    for (int k = 0; k < n_scenes; ++k) {
        const vis_scene_grads& g = grads[k];
        const void* ptrs[5] = {g.d_means, g.d_log_scales, g.d_quats, g.d_opacity_logits, g.d_sh};
        for (int j = 0; j < 5; ++j)
            if (!ptrs[j] || !aligned16(ptrs[j]))
                return fail(VIS_ERR_INVALID_ARG, "gradient buffer %d of scene %d null or misaligned", j, k);
    }
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    char* w = static_cast<char*>(ws);
    vis::launch_composite_backward(L, w, bg, o.alpha_min, o.alpha_max, o.pixels_per_thread, d_rgb, d_alpha, zlim,
                                   stream);
    for (int k = 0; k < n_scenes; ++k) {
        const vis_scene_grads& g = grads[k];
        vis::launch_preprocess_backward(scene_params(scenes, models, k, padded, offsets, cam, W, H, L, o), L, w,
                                        g.d_means, g.d_log_scales, g.d_quats, g.d_opacity_logits, g.d_sh, stream);
    }
    if ((st = cuda_check(cudaGetLastError(), "launch"))) return st;
    g_err.clear();
    return VIS_OK;
}

static vis_status backward_one(vis_scene_t scene, const vis_camera* cam, int W, int H, const float bg[3],
                               const float* zlim, const float* d_rgb, const float* d_alpha, void* ws,
                               size_t ws_bytes, const vis_render_opts* opts, float* d_means, float* d_log_scales,
                               float* d_quats, float* d_opacity_logits, float* d_sh, void* stream_) {
    const vis_scene_grads g = {d_means, d_log_scales, d_quats, d_opacity_logits, d_sh};
    return backward_impl(&scene, nullptr, 1, false, cam, W, H, bg, zlim, d_rgb, d_alpha, ws, ws_bytes, opts, &g,
                         stream_);
}

vis_status vis_render_backward(vis_scene_t scene, const vis_camera* cam, int W, int H, const float bg[3],
                               const float* d_rgb, const float* d_alpha, void* ws, size_t ws_bytes,
                               const vis_render_opts* opts, float* d_means, float* d_log_scales, float* d_quats,
                               float* d_opacity_logits, float* d_sh, void* stream_) {
    return backward_one(scene, cam, W, H, bg, nullptr, d_rgb, d_alpha, ws, ws_bytes, opts, d_means, d_log_scales,
                        d_quats, d_opacity_logits, d_sh, stream_);
}

vis_status vis_render_backward_depth(vis_scene_t scene, const vis_camera* cam, int W, int H, const float bg[3],
                                     const float* depth, const float* d_rgb, const float* d_alpha, void* ws,
                                     size_t ws_bytes, const vis_render_opts* opts, float* d_means,
                                     float* d_log_scales, float* d_quats, float* d_opacity_logits, float* d_sh,
                                     void* stream_) {
    if (!depth || !aligned16(depth)) return fail(VIS_ERR_INVALID_ARG, "depth buffer null or not 16-byte aligned");
    return backward_one(scene, cam, W, H, bg, depth, d_rgb, d_alpha, ws, ws_bytes, opts, d_means, d_log_scales,
                        d_quats, d_opacity_logits, d_sh, stream_);
}

vis_status vis_render_backward_multi(const vis_scene_t* scenes, const float* models, int n_scenes,
                                     const vis_camera* cam, int W, int H, const float bg[3], const float* depth,
                                     const float* d_rgb, const float* d_alpha, void* ws, size_t ws_bytes,
                                     const vis_render_opts* opts, const vis_scene_grads* grads, void* stream_) {
    if (depth && !aligned16(depth)) return fail(VIS_ERR_INVALID_ARG, "depth buffer not 16-byte aligned");
    return backward_impl(scenes, models, n_scenes, true, cam, W, H, bg, depth, d_rgb, d_alpha, ws, ws_bytes, opts,
                         grads, stream_);
}

vis_status vis_dynamic_update(const float* means0, const float* velocity, const float* logits0, const float* amp,
                              const float* freq, const float* phase, float t, int64_t n, float* means_out,
                              float* logits_out, void* stream_) {
    if (n < 1 || n > 0x7fffffffLL) return fail(VIS_ERR_INVALID_ARG, "n must be in [1, 2^31-1]");
    if (!std::isfinite(t)) return fail(VIS_ERR_INVALID_ARG, "t is not finite");
    const void* ptrs[8] = {means0, velocity, logits0, amp, freq, phase, means_out, logits_out};
    for (int k = 0; k < 8; ++k)
        if (!ptrs[k] || !aligned16(ptrs[k])) return fail(VIS_ERR_INVALID_ARG, "dynamic update buffer %d null or misaligned", k);
    if ((const void*)means_out == (const void*)means0 || (const void*)logits_out == (const void*)logits0)
        return fail(VIS_ERR_INVALID_ARG, "outputs must not alias the inputs");
    vis::launch_dynamic_update(means0, velocity, logits0, amp, freq, phase, t, n, means_out, logits_out,
                               reinterpret_cast<cudaStream_t>(stream_));
    vis_status st = cuda_check(cudaGetLastError(), "launch");
    if (st) return st;
    g_err.clear();
    return VIS_OK;
}

vis_status vis_profile_begin(void) {
    if (!g_prof.created) {
        for (int r = 0; r < kProfRing; ++r)
            for (int k = 0; k <= kProfStages; ++k) {
                vis_status st = cuda_check(cudaEventCreate(&g_prof.ev[r][k]), "create profiling events");
                if (st) return st;
            }
        g_prof.created = true;
    }
    g_prof.on = true;
    g_prof.count = 0;
    g_err.clear();
    return VIS_OK;
}

vis_status vis_profile_end(double* stage_ms, int max_stages, int* n_stages, int* n_renders, int* n_passes) {
    if (!g_prof.on) return fail(VIS_ERR_INVALID_ARG, "profiling was not begun");
    g_prof.on = false;
    const int n = g_prof.count < kProfStages ? g_prof.count : kProfStages;
    (void)n;
    double sum[kProfStages] = {0};
    for (int r = 0; r < g_prof.count; ++r) {
        vis_status st = cuda_check(cudaEventSynchronize(g_prof.ev[r][kProfStages]), "profiling sync");
        if (st) return st;
        for (int k = 0; k < kProfStages; ++k) {
            float ms = 0.f;
            if ((st = cuda_check(cudaEventElapsedTime(&ms, g_prof.ev[r][k], g_prof.ev[r][k + 1]), "elapsed")))
                return st;
            sum[k] += ms;
        }
    }
    const int w = max_stages < kProfStages ? max_stages : kProfStages;
    for (int k = 0; k < w && stage_ms; ++k) stage_ms[k] = sum[k];
    if (n_stages) *n_stages = w;
    if (n_renders) *n_renders = g_prof.count;
    if (n_passes) *n_passes = g_prof.passes;
    g_err.clear();
    return VIS_OK;
}

// Standalone sort workspace: status block, histograms, look-back words, one
// ping-pong key/value buffer.
static size_t sort_ws_layout(int64_t m, int passes, size_t* off_hist, size_t* off_lb, size_t* off_k, size_t* off_v,
                             int64_t* parts) {
    *parts = vis::sort_parts<uint64_t>(m);
    size_t off = align_up(sizeof(vis::Ctrl), 256);
    *off_hist = off; off = align_up(off + sizeof(uint32_t) * vis::kMaxPasses * vis::kRadix, 256);
    *off_lb = off;
    off = align_up(off + sizeof(uint32_t) * (size_t)passes * vis::lookback_rows(*parts, vis::lookback_group(8, 8)) *
                             vis::kRadix,
                   256);
    const size_t zero_end = off;
    *off_k = off; off = align_up(off + sizeof(uint64_t) * (size_t)m, 256);
    *off_v = off; off = align_up(off + sizeof(uint32_t) * (size_t)m, 256);
    (void)zero_end;
    return off;
}

vis_status vis_sort_workspace_size(int64_t m, int key_bits, size_t* bytes) {
    if (!bytes) return fail(VIS_ERR_INVALID_ARG, "bytes is null");
    if (m < 0 || m > (int64_t)vis::kMaxKeys) return fail(VIS_ERR_INVALID_ARG, "m must be in [0, 2^30-1]");
    if (key_bits < 1 || key_bits > 64) return fail(VIS_ERR_INVALID_ARG, "key_bits must be in [1, 64]");
    const int passes = (key_bits + vis::kRadixBits - 1) / vis::kRadixBits;
    size_t a, b, c, d;
    int64_t parts;
    *bytes = sort_ws_layout(m, passes, &a, &b, &c, &d, &parts);
    return VIS_OK;
}

vis_status vis_sort_pairs(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out, uint32_t* vals_out,
                          int64_t m, int key_bits, void* ws, size_t ws_bytes, void* stream_) {
    size_t need = 0;
    vis_status st = vis_sort_workspace_size(m, key_bits, &need);
    if (st) return st;
    if (!ws || !aligned16(ws) || ws_bytes < need)
        return fail(VIS_ERR_INVALID_ARG, "sort workspace null, misaligned or smaller than %zu bytes", need);
    if (m == 0) { g_err.clear(); return VIS_OK; }
    const void* ptrs[4] = {keys_in, vals_in, keys_out, vals_out};
    for (int k = 0; k < 4; ++k)
        if (!ptrs[k] || !aligned16(ptrs[k])) return fail(VIS_ERR_INVALID_ARG, "sort buffer %d null or misaligned", k);
    if ((const void*)keys_in == (const void*)keys_out || (const void*)vals_in == (const void*)vals_out)
        return fail(VIS_ERR_INVALID_ARG, "sort input and output must not alias");
    const int passes = (key_bits + vis::kRadixBits - 1) / vis::kRadixBits;
    size_t off_hist, off_lb, off_k, off_v;
    int64_t parts;
    sort_ws_layout(m, passes, &off_hist, &off_lb, &off_k, &off_v, &parts);
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    char* w = static_cast<char*>(ws);
    vis::Ctrl* ctrl = reinterpret_cast<vis::Ctrl*>(w);
    if ((st = cuda_check(cudaMemsetAsync(w, 0, off_k, stream), "clear sort workspace"))) return st;
    vis::launch_set_u32(&ctrl->num_keys, (uint32_t)m, stream);
    vis::launch_sort_generic<uint64_t>(keys_in, vals_in, keys_out, vals_out, reinterpret_cast<uint64_t*>(w + off_k),
                                       reinterpret_cast<uint32_t*>(w + off_v), m, &ctrl->num_keys, passes,
                                       reinterpret_cast<uint32_t*>(w + off_hist), reinterpret_cast<uint32_t*>(w + off_lb),
                                       ctrl->part_counter, &ctrl->error, stream, nullptr, 0,
                                       key_bits - vis::kRadixBits * (passes - 1));
    if ((st = cuda_check(cudaGetLastError(), "launch"))) return st;
    g_err.clear();
    return VIS_OK;
}

}  // extern "C"
