// Internal declarations shared by the CUDA translation units of libvis.
// Nothing here is part of the C ABI (see include/vis.h).
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <mutex>
#include <stdint.h>

#include <vector>

#include "../../include/vis.h"

namespace vis {

constexpr int kPrepThreads = 256;        // Gaussians per preprocess / duplicate block
constexpr int kSortThreads = 256;        // threads per radix-sort CTA
// keys per thread per partition, by key width (8 for 64-bit keys keeps three CTAs per SM)
template <typename K> struct SortKPT;
template <> struct SortKPT<uint64_t> { static constexpr int value = 8; };
template <> struct SortKPT<uint32_t> { static constexpr int value = 16; };
template <> struct SortKPT<uint16_t> { static constexpr int value = 16; };
// counts-first tile sort of sort_mode 1 (tile_sort.cu): used when the tile grid has at most
// kTileFusedMaxTiles tiles (its per-tile counters live in shared memory)
constexpr int kTileFusedMaxTiles = 51200;
// Compositing order: bucket of a tile's key count c, 0 for the largest counts: two
// log-spaced buckets per octave (the bit after the leading one), the empty tiles last.
constexpr int kOrderBits = 6;
constexpr int kOrderBuckets = 1 << kOrderBits;
__device__ __forceinline__ int order_bucket(uint32_t c) {
    if (c == 0) return kOrderBuckets - 1;
    const int lg = 31 - __clz(c);
    const int k = lg * 2 + (lg >= 1 ? (int)((c >> (lg - 1)) & 1u) : 0);
    return kOrderBuckets - 2 - (k < kOrderBuckets - 2 ? k : kOrderBuckets - 2);
}
template <typename K> constexpr int64_t sort_partition() { return (int64_t)kSortThreads * SortKPT<K>::value; }
template <typename K> constexpr int64_t sort_parts(int64_t cap) {
    return (cap + sort_partition<K>() - 1) / sort_partition<K>();
}
// The depth sort of a scene of at most kSmallDepthSort Gaussians uses half-size partitions
// (8 keys per thread): a pass over ~1M keys is a single wave of short-lived CTAs, twice as
// many of them, instead of half a wave of long ones.
constexpr int64_t kSmallDepthSort = (int64_t)2 << 20;
inline int depth_sort_kpt(int64_t n, int digit_bits = 8) {
    return (n <= kSmallDepthSort && digit_bits == 8) ? 8 : SortKPT<uint32_t>::value;
}
inline int64_t depth_sort_parts(int64_t n, int digit_bits = 8) {
    const int64_t part = (int64_t)kSortThreads * depth_sort_kpt(n, digit_bits);
    return (n + part - 1) / part;
}
// Look-back region of one radix pass over `parts` partitions (onesweep.cuh): a row of
// 2^digit_bits words per partition, then a row per group of lookback_group consecutive
// partitions (the group's counts and arrivals). The group is one look-back window wide.
constexpr int lookback_group(int key_bytes, int digit_bits) {
    return digit_bits > 8 ? 4 : (key_bytes == 2 ? 8 : 16);
}
__host__ __device__ inline int64_t lookback_rows(int64_t parts, int group) { return parts + (parts + group - 1) / group; }
// passes of a key of `bits` significant bits at digit_bits per pass
inline int passes_for(int bits, int digit_bits) { return bits <= 0 ? 0 : (bits + digit_bits - 1) / digit_bits; }
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kMaxDigitBits = 11;        // widest radix digit (vis_render_opts.digit_bits)
constexpr int kMaxPasses = 8;
constexpr uint32_t kMaxKeys = (1u << 30) - 1;   // look-back words hold 30-bit counts

// ctrl->error bits
constexpr uint32_t kErrCapacity = 1u;
constexpr uint32_t kErrTimeout = 2u;
constexpr uint32_t kErrNoAdjoint = 4u;   // an adjoint was asked of a render that has none
// ctrl->flags bits
constexpr uint32_t kFlagNoAdjoint = 1u;  // a dynamic frame: its attributes were never stored

// Default look-back spin limit, in polls (each poll ~ a few hundred ns with the backoff);
// far beyond any legitimate wait, it only bounds a wait that can never end. A render's
// vis_render_opts.spin_limit overrides it.
constexpr uint32_t kSpinLimit = 1u << 22;
constexpr uint32_t kMaxSpinLimit = 1u << 30;

// Sort modes (vis_render_opts.sort_mode)
constexpr int kSortTileDepth = 0;   // one sort of 64-bit (tile << 32 | depth) keys
constexpr int kSortDepthFirst = 1;  // depth sort of the surviving splats, then a tile sort

struct Layout {
    int mode = kSortTileDepth;
    int64_t n = 0;
    int W = 0, H = 0, tile = 16;
    int tiles_x = 0, tiles_y = 0;
    int64_t ntiles = 0;
    int tile_bits = 0, key_bits = 0, passes = 0;
    int digit_bits = kRadixBits;           // digit of the depth sort and of a 32-bit tile sort
    int depth_passes = 4;                  // passes of the depth sort (32-bit keys)
    size_t off_hist_tile = 0;              // histograms of the tile sort (after the depth sort's)
    int64_t cap = 0;
    int64_t prep_blocks = 0;
    int64_t sort_parts = 0;
    size_t off_ctrl = 0, off_rec = 0, off_depth = 0, off_rect = 0, off_touched = 0;
    size_t off_bsum = 0, off_boff = 0;
    // look-back words of a render's (at most two) block-sum scans: two slots of
    // scan_parts(prep_blocks) 64-bit words each, in the cleared region
    size_t off_scan_lb = 0;
    int64_t scan_slot_words = 0;
    size_t off_keys[2] = {0, 0}, off_vals[2] = {0, 0};
    size_t off_hist = 0, off_lookback = 0, off_ranges = 0;
    // look-back words of the tile sort's passes: after the depth sort's, inside the cleared
    // region; with the counts-first tile sort a region of their own, of which each render clears
    // only the rows its passes read (clear_tile_lookback, beside the depth sort)
    size_t off_lookback_tile = 0;
    size_t off_tfinal = 0, off_last = 0, off_g2 = 0;
    size_t off_zmax = 0;     // float[tiles]: largest depth-buffer value per tile (depth-tested renders)
    // depth-first mode only
    size_t off_dkeys[2] = {0, 0}, off_dvals[2] = {0, 0}, off_bsum2 = 0, off_boff2 = 0;
    size_t lookback_words_depth = 0;
    int key_bytes = 8;
    // depth-first mode with the counts-first tile sort of 16-bit keys (tile_sort.cu)
    bool tile_fused = false;
    size_t off_tdiff = 0;
    size_t off_order = 0;    // compositing order of the tiles (counts-first tile sort only)
    size_t zero_begin = 0, zero_end = 0;   // region cleared before every render
    size_t total = 0;
    int sorted_buffer = 0;
    uint32_t spin_limit = kSpinLimit;      // polls a look-back wait may make (from the render options)
};

// Workspace layout for n Gaussians, W x H, tile size, key capacity `cap`, sort mode, radix
// digit width.
Layout make_layout(int64_t n, int W, int H, int tile, int64_t cap, int mode, int digit_bits = kRadixBits);
// Largest capacity whose layout fits ws_bytes (0 if none).
int64_t capacity_for(int64_t n, int W, int H, int tile, int mode, size_t ws_bytes, int digit_bits = kRadixBits);

struct Ctrl {
    uint32_t num_keys;
    uint32_t error;
    uint32_t part_counter[2 * kMaxPasses];   // partition tickets of up to two sorts per render
    uint32_t num_visible;                    // Gaussians that survive culling (depth-first sort)
    uint32_t flags;                          // kFlagNoAdjoint: the render was a dynamic frame
    unsigned long long pair_tests;           // compositor statistics (collect_stats only)
    unsigned long long hits;
    uint32_t scan_ticket[2];                 // chunk tickets of the render's block-sum scans
    uint32_t reserved[38];
};
static_assert(sizeof(Ctrl) == 256, "ctrl block is 256 bytes");

// Per-view preprocess parameters (passed by value).
struct PrepParams {
    const float* means;
    const float* log_scales;
    const float* quats;
    const float* logits;
    const float* sh;
    int deg;
    int n;
    float R[9], t[3];
    // rounding residues of R and t (zero for a plain camera): a model transform M_k = [A | b]
    // is folded into the camera as R A and R b + t, computed in double and carried as float
    // pairs so that the camera-space position keeps float-float accuracy
    float R_lo[9], t_lo[3];
    float fx, fy, cx, cy, near_z;
    float cam_pos[3];        // camera centre in the scene's own frame (A^-1 (c - b) under a model)
    float limx, limy;
    int W, H, tile, tiles_x, tiles_y;
    float dilation, alpha_min;
    float wscale;            // sqrt(log2(e)/2): scales the whitening rows of the record
    int tight_extent;        // 1: tile rect from the tight opacity-aware 3-sigma box
    int count_survivors;     // block sums count survivors (depth-first sorts), else tiles touched
    // depth-tested renders: largest depth limit per tile (NaN counted as +inf), or null; a
    // splat deeper than the limit of every tile of its footprint is culled
    const float* tile_zmax;
    // pre-packed scene (Algorithm 1 pre-pack, fp16 pairs in uint32 words; null for fp32 SoA):
    // pos (mu_x, mu_y), (mu_z, alpha); cov (xx, xy), (xz, yy), (yz, zz); col: SH halves,
    // col_words words per Gaussian
    const uint2* pk_pos;
    const uint32_t* pk_cov;
    const uint32_t* pk_col;
    int col_words;
    int64_t index_offset;    // workspace slot of the scene's first Gaussian (a multiple of kPrepThreads)
    int n_pad;               // n rounded up to kPrepThreads in a multi-scene render (else n)
    float shc[12];           // SH polynomial constants, see sh_constants()
    uint32_t batch_image;    // a fused batch: the item's image index (kept in the footprints)
    uint32_t canvas_row0;    // a fused batch: the image's first tile row in its group's canvas
    // a dynamic frame (vis_render_dynamic): means and logits hold frame 0; the preprocess
    // applies the update of dynamic.cuh at time dyn_t with these arrays (null otherwise) and
    // marks the status block (dyn_flags) as a render with no adjoint
    const float* dyn_velocity;
    const float* dyn_amp;
    const float* dyn_freq;
    const float* dyn_phase;
    uint32_t* dyn_flags;
    float dyn_t;
    uint32_t dyn_pad;
};

// One image of a fused batch (vis_render_batch with lanes = 0): its (asset, camera) item's
// Gaussians occupy the workspace slots [slot0, slot0 + n), and its tiles the rows
// [tile0 / cw, tile0 / cw + tiles_y) x columns [0, tiles_x) of its group's canvas, a tile grid
// cw tiles wide (tile0 = its first row times cw). A group's images are listed in increasing
// tile0.
struct BatchImage {
    int64_t slot0;
    uint32_t tile0;
    int W, H, tiles_x, tiles_y;
    int index;          // the image's index in the batch (its status word)
    float* out_rgb;     // [3][H][W]
    float* out_alpha;   // [H][W]
};

// SH polynomial constants from the normalisation K_l^m (computed in double).
void sh_constants(float out[12]);

// ---------------------------------------------------------------------------
// Error-free transforms and float-float arithmetic (Dekker / Knuth), used to
// carry the camera transform and perspective division beyond float precision.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {   // |a| >= |b|
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return make_float2(s, e);
}
__device__ __forceinline__ float2 two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return make_float2(p, e);
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    float2 s = two_sum(a.x, b.x);
    float e = __fadd_rn(s.y, __fadd_rn(a.y, b.y));
    return fast_two_sum(s.x, e);
}
// a.hi/a.lo divided by b.hi/b.lo
__device__ __forceinline__ float2 ff_div(float2 a, float2 b) {
    float q = __fdiv_rn(a.x, b.x);
    float r = __fmaf_rn(-q, b.x, a.x);          // exact remainder of a.x - q b.x
    r = __fadd_rn(r, __fsub_rn(a.y, __fmul_rn(q, b.y)));
    float ql = __fdiv_rn(r, b.x);
    return fast_two_sum(q, ql);
}

// Kahan's accurate a*b - c*d
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
    float w = __fmul_rn(c, d);
    float e = __fmaf_rn(-c, d, w);
    float f = __fmaf_rn(a, b, -w);
    return __fadd_rn(f, e);
}

// uint32 words per Gaussian of a packed colour plane: 3 (deg+1)^2 halves, rounded up to an
// even number of words (8-byte rows)
__host__ __device__ __forceinline__ int packed_col_words(int deg) {
    const int words = (3 * (deg + 1) * (deg + 1) + 1) / 2;
    return words + (words & 1);
}

// Programmatic dependent launch (Hopper and later): a kernel of the render path may be launched
// before its predecessor in the stream has finished. At entry it waits for the predecessor
// grids to complete (their memory visible) and at once lets its own successor be launched, so
// a kernel's launch and CTA start-up overlap the previous kernel's tail. Every kernel launched
// with the attribute calls this before touching global memory.
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// False when the environment sets VIS_PDL=0 (plain stream ordering for every launch).
bool pdl_enabled();
// Launch `kernel` on `stream`; with pdl (and pdl_enabled()) as a programmatic dependent of
// the stream's previous kernel. The kernel must start with pdl_entry().
template <typename... KArgs, typename... Args>
inline void launch_k(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                     Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    if (pdl && pdl_enabled()) {
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Runs setup() for the current device unless it has already succeeded there (function
// attributes such as cudaFuncSetAttribute apply to the current device only). The device's
// bit in `done` is published only after setup() has returned true, and concurrent callers
// wait on `mu`, so every launch that follows a return of this function on that device sees
// the attributes set; a failed set-up is retried by the next call. Returns false if setup()
// failed.
template <typename F>
inline bool set_up_per_device(std::atomic<uint64_t>& done, std::mutex& mu, F setup) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return setup();
    const uint64_t bit = 1ull << dev;
    if (done.load(std::memory_order_acquire) & bit) return true;
    std::lock_guard<std::mutex> lock(mu);
    if (done.load(std::memory_order_relaxed) & bit) return true;
    if (!setup()) return false;
    done.fetch_or(bit, std::memory_order_release);
    return true;
}

// Launchers (host side, enqueue on `stream`).
void launch_preprocess(const PrepParams& p, const Layout& L, char* ws, cudaStream_t stream);
// The preprocess of a fused batch over its work list: items[k] (device) are the items'
// parameters, blk0[k] (device, n_items entries) their first blocks, `blocks` the total;
// only plain (packed = false) or only pre-packed scenes per launch.
void launch_preprocess_batch(const PrepParams* items, const uint32_t* blk0, int n_items, int64_t blocks,
                             bool packed, const Layout& L, char* ws, cudaStream_t stream);
// Per-tile maximum of a depth buffer zlim [H,W] into ws + L.off_zmax.
void launch_tile_zmax(const Layout& L, char* ws, const float* zlim, cudaStream_t stream);
// Pre-pack (Algorithm 1, once per scene): fp32 SoA attributes -> fp16 planes pos, cov, col.
void launch_pack(const float* means, const float* log_scales, const float* quats, const float* logits,
                 const float* sh, int deg, int64_t n, uint2* pos, uint32_t* cov, uint32_t* col, cudaStream_t stream);
void launch_scan_and_duplicate(const Layout& L, char* ws, int64_t n, cudaStream_t stream);
// Sorts keys[0] -> keys[L.sorted_buffer] over L.passes digit passes. If `mark` is
// given it is called with (mark_index, stream) after the histogram, i.e. between
// the histogram and the first digit pass.
typedef void (*StageMark)(int, cudaStream_t);
void launch_sort(const Layout& L, char* ws, cudaStream_t stream, StageMark mark = nullptr, int mark_index = 0);
void launch_ranges(const Layout& L, char* ws, cudaStream_t stream);
// Exclusive scan of nblocks per-block sums into boff, the total into *total, in one pass over
// chunks of kScanPart sums (keys.cu). When cap > 0 a total above cap sets kErrCapacity in *error;
// a look-back that gives up sets kErrTimeout there. lb: scan_parts(nblocks) zeroed 64-bit
// look-back words; ticket: a zeroed counter (one of each per scan in a render).
constexpr int kScanPart = 2048;
inline int64_t scan_parts(int64_t nblocks) { return nblocks <= 0 ? 1 : (nblocks + kScanPart - 1) / kScanPart; }
void launch_scan_sums(const uint32_t* bsum, uint32_t* boff, int64_t nblocks, uint32_t* total, uint32_t* error,
                      int64_t cap, unsigned long long* lb, uint32_t* ticket, uint32_t spin_limit,
                      cudaStream_t stream);
// Depth-first mode: compaction and depth sort (then mark(mark_index)), emission (then
// mark(mark_index + 1)), tile counts or the tile histogram (then mark(mark_index + 2)), tile
// passes. Beyond the counts-first grids the 32-bit tile sort runs; ranges for its keys:
void launch_depth_first(const Layout& L, char* ws, cudaStream_t stream, StageMark mark, int mark_index);
// Compaction of the surviving splats and their stable sort by depth (result in dvals[0]).
void launch_depth_sort(const Layout& L, char* ws, cudaStream_t stream);
void launch_ranges32(const Layout& L, char* ws, cudaStream_t stream);
// q' = q * log2(e)/2 units: the 3-sigma cut is q' <= 9 log2(e)/2
struct QScale {
    float qcut;        // 9 log2(e) / 2
    float inv_scale;   // 2 / log2(e) = 2 ln 2
};
QScale q_scale();
// zlim: [H,W] depth buffer for the depth-tested compositing, or null
void launch_composite(const Layout& L, char* ws, float bg0, float bg1, float bg2, float alpha_min,
                      float alpha_max, float t_stop, int ppt, bool stats, float* out_rgb, float* out_alpha,
                      const float* zlim, cudaStream_t stream);
// Compositor over the canvas of one group of a fused batch (L: the group's layout, its
// canvas L.tiles_x tiles wide; `images`: the group's n_images entries of the image table in
// device memory), forward only; with the counts-first tile sort the tiles are taken longest
// first.
void launch_composite_batch(const Layout& L, char* ws, const BatchImage* images, int n_images, int64_t total_tiles,
                            float bg0, float bg1, float bg2, float alpha_min, float alpha_max, float t_stop, int ppt,
                            cudaStream_t stream);
// Adjoint of the compositing: clears and accumulates the screen-space gradients g2 of
// all L.n slots (ppt pixels per thread, 1 or 2; zlim as in launch_composite).
void launch_composite_backward(const Layout& L, char* ws, const float bg[3], float alpha_min, float alpha_max,
                               int ppt, const float* d_rgb, const float* d_alpha, const float* zlim,
                               cudaStream_t stream);
// Adjoint of the preprocess of one scene (slots p.index_offset ..): g2 -> the scene's
// parameter gradients.
void launch_preprocess_backward(const PrepParams& p, const Layout& L, const char* ws, float* d_means,
                                float* d_log_scales, float* d_quats, float* d_logits, float* d_sh,
                                cudaStream_t stream);

// Stable LSD radix sort of (K key, uint32 value) pairs over `passes` digits of digit_bits
// bits (8; 10 or 11 for 32-bit keys). Reads keys_in/vals_in, ping-pongs between the a and b
// buffers and leaves the result in a. `lookback` must hold passes * parts * 2^digit_bits
// words (parts = sort_parts_for(cap, kpt, digit_bits)), `hist` passes * 2^digit_bits words
// and `part_counters` passes words, all zeroed; the key count is read from num_keys_dev
// (<= cap). If `mark` is given it is called after the histogram. last_bits: significant
// bits of the last pass's digit (key bits - digit_bits (passes - 1)). With last_keys false the
// last pass writes only the values (keys_a then holds the previous pass's keys).
template <typename K>
void launch_sort_generic(const K* keys_in, const uint32_t* vals_in, K* keys_a, uint32_t* vals_a, K* keys_b,
                         uint32_t* vals_b, int64_t cap, const uint32_t* num_keys_dev, int passes, uint32_t* hist,
                         uint32_t* lookback, uint32_t* part_counters, uint32_t* error, cudaStream_t stream,
                         StageMark mark = nullptr, int mark_index = 0, int last_bits = kRadixBits, int kpt = 0,
                         uint32_t spin_limit = kSpinLimit, int digit_bits = kRadixBits, bool last_keys = true);

// One sort_pass over the keys (digit (key >> shift) & 255 with nbits significant bits,
// histogram hist_pass); keys_out may be null. `lookback` holds sort_parts<K>(cap) * kRadix
// zeroed words, *part_counter is zero.
template <typename K>
void launch_sort_pass(const K* keys_in, const uint32_t* vals_in, K* keys_out, uint32_t* vals_out, int64_t cap,
                      const uint32_t* num_keys_dev, int shift, int nbits, const uint32_t* hist_pass,
                      uint32_t* lookback, uint32_t* part_counter, uint32_t* error, cudaStream_t stream,
                      uint32_t spin_limit = kSpinLimit);

// Counts-first tile sort of sort_mode 1 (tile_sort.cu): per-tile counts -> digit histograms
// and ranges; then the passes over the 16-bit tile keys emitted in depth order.
void launch_tile_counts(const Layout& L, char* ws, cudaStream_t stream);

// A second stream of the calling host thread for a main stream on the current device, with a
// fork and a join event, for work that can run beside the main stream's: side_stream(stream)
// creates it on first use and keeps it for the thread's lifetime (nullptr if creation failed
// or 64 are in use -- the caller then runs the work in order). side_fork makes the side stream wait for the main stream's work
// so far; side_join_point records the join event after the side stream's work (false if that
// failed, after the host waited for the side stream); the main stream then waits on `join`.
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
SideStream* side_stream(cudaStream_t stream);
bool side_fork(SideStream* side, cudaStream_t stream);
bool side_join_point(SideStream* side, cudaStream_t stream);
void launch_tile_passes(const Layout& L, char* ws, cudaStream_t stream);

void launch_dynamic_update(const float* means0, const float* velocity, const float* logits0, const float* amp,
                           const float* freq, const float* phase, float t, int64_t n, float* means_out,
                           float* logits_out, cudaStream_t stream);

// Scene accessors for the batch planner (the scene struct is private to api.cu).
int64_t scene_size(vis_scene_t s);
void append_scene_key(std::vector<unsigned char>& key, vis_scene_t s);
bool scene_packed(vis_scene_t s);
// Render options with the defaults filled in, validated (sets the error message).
vis_status batch_opts(const vis_render_opts* in, vis_render_opts* out);
// Validated preprocess parameters of image `image` of a fused batch: scene s seen by cam at
// W x H, its Gaussians at workspace slots slot0 .. (a multiple of kPrepThreads).
vis_status batch_item(vis_scene_t s, const vis_camera* cam, int W, int H, const vis_render_opts& o, int64_t slot0,
                      uint32_t image, PrepParams* out);

// Sets the thread-local message returned by vis_last_error().
void set_last_error(const char* msg);

// *ptr = value, enqueued on the stream (no host synchronisation).
void launch_set_u32(uint32_t* ptr, uint32_t value, cudaStream_t stream);

}  // namespace vis
