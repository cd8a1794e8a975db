// Depth-first ordering of the splats: the sort of Algorithm 1 ("Radix Sort" over the
// depths of the surviving splats, section 3.4), followed by a stable bucketing of
// their tile copies by tile.
//
//   1. compact_visible: surviving Gaussians (tiles touched > 0; the preprocess counts them
//      per block), in index order, as
//      (float bits of depth, index) pairs; the count goes to the status block.
//   2. a stable radix sort of those pairs by the 32-bit depth key (4 passes of 8 bits;
//      equal depths keep index order);
//   3. depth_touch_sums / scan / emit_tiles: every sorted splat emits one (tile id,
//      index) pair per tile of its rectangle, in depth order (same deterministic
//      warp-cooperative emission as the index-order duplication);
//   4. a stable radix sort of those pairs by the tile id alone (ceil(tile bits / 8)
//      passes of 32-bit keys);
//   5. ranges_kernel32: [start, end) of every tile.
// Stability makes the final order (tile, depth, index) -- identical to sorting the
// 64-bit (tile << 32 | depth) keys -- while the sort moves 4-byte keys, and only the
// N surviving splats (not the M tile copies) take part in the four depth passes.
#include <map>
#include <utility>

#include "vis_internal.cuh"
#include "footprint.cuh"

namespace vis {

// exclusive warp scan helper
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Both kernels below take kBlocksPerCta blocks of kPrepThreads slots per CTA, each thread one
// slot of every block, so that a thread has that many independent loads in flight (one per
// block) instead of one; the per-block results are those of one CTA per block.
constexpr int kBlocksPerCta = 4;

__global__ void __launch_bounds__(kPrepThreads)
compact_visible(const uint32_t* __restrict__ touched, const float* __restrict__ depth, int64_t n,
                int64_t nblocks, const uint32_t* __restrict__ boff, uint32_t* __restrict__ dkeys,
                uint32_t* __restrict__ dvals) {
    pdl_entry();
    __shared__ uint32_t ws[kBlocksPerCta][kPrepThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t b0 = (int64_t)blockIdx.x * kBlocksPerCta;
    bool f[kBlocksPerCta];
    float z[kBlocksPerCta];
#pragma unroll
    for (int k = 0; k < kBlocksPerCta; ++k) {
        const int64_t i = (b0 + k) * kPrepThreads + threadIdx.x;
        f[k] = i < n && touched[i] > 0;
        z[k] = i < n ? depth[i] : 0.f;
    }
    uint32_t bal[kBlocksPerCta];
#pragma unroll
    for (int k = 0; k < kBlocksPerCta; ++k) {
        bal[k] = __ballot_sync(0xffffffffu, f[k]);
        if (lane == 0) ws[k][warp] = __popc(bal[k]);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kBlocksPerCta; ++k) {
        if (b0 + k >= nblocks) break;
        uint32_t off = boff[b0 + k];
        for (int w = 0; w < warp; ++w) off += ws[k][w];
        if (f[k]) {
            const uint32_t o = off + __popc(bal[k] & ((1u << lane) - 1u));
            dkeys[o] = __float_as_uint(z[k]);   // z > near > 0: bit order = numeric order
            dvals[o] = (uint32_t)((b0 + k) * kPrepThreads + threadIdx.x);
        }
    }
}

// Block sums of tiles touched, in depth order. After a failed depth sort (a look-back
// that timed out) the sorted indices are not trustworthy: every block sum is then zero and
// nothing is read through them.
__global__ void __launch_bounds__(kPrepThreads)
depth_touch_sums(const uint32_t* __restrict__ dvals, const uint32_t* __restrict__ touched, int64_t n,
                 int64_t nblocks, const Ctrl* __restrict__ ctrl, uint32_t* __restrict__ bsum) {
    pdl_entry();
    __shared__ uint32_t ws[kBlocksPerCta][kPrepThreads / 32];
    const int64_t nv = ctrl->error ? 0 : min((int64_t)ctrl->num_visible, n);
    const int64_t b0 = (int64_t)blockIdx.x * kBlocksPerCta;
    uint32_t g[kBlocksPerCta], c[kBlocksPerCta];
#pragma unroll
    for (int k = 0; k < kBlocksPerCta; ++k) {
        const int64_t j = (b0 + k) * kPrepThreads + threadIdx.x;
        g[k] = (j < nv) ? dvals[j] : 0xffffffffu;
    }
#pragma unroll
    for (int k = 0; k < kBlocksPerCta; ++k) c[k] = (g[k] < (uint64_t)n) ? touched[g[k]] : 0u;
#pragma unroll
    for (int k = 0; k < kBlocksPerCta; ++k) {
        uint32_t v = c[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) ws[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < kBlocksPerCta && b0 + threadIdx.x < nblocks) {
        uint32_t t = 0;
        for (int w = 0; w < kPrepThreads / 32; ++w) t += ws[threadIdx.x][w];
        bsum[b0 + threadIdx.x] = t;
    }
}

// KT: uint32_t tile ids, or uint16_t on grids of at most 65536 tiles; tile ids are
// y * tiles_x + x.
template <typename KT>
__global__ void __launch_bounds__(kPrepThreads)
emit_tiles(const uint32_t* __restrict__ dvals, const uint4* __restrict__ rect, int64_t n,
           const uint32_t* __restrict__ boff, int tiles_x,
           const Ctrl* __restrict__ ctrl, KT* __restrict__ keys, uint32_t* __restrict__ vals) {
    pdl_entry();
    if (ctrl->error) return;   // capacity exceeded, or a sort that timed out
    // per splat slot: start of its copies in the warp's run, and its footprint unrolled into
    // row segments: a = (index, first top-row tile, top width, end of the middle copies),
    // b = (first middle tile, box width, first bottom-row tile, row stride)
    __shared__ uint32_t s_start[kPrepThreads];
    __shared__ uint4 s_a[kPrepThreads], s_b[kPrepThreads];
    __shared__ uint32_t warp_tot[kPrepThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nv = min((int64_t)ctrl->num_visible, n);
    const int64_t j = (int64_t)blockIdx.x * kPrepThreads + threadIdx.x;
    uint32_t cnt = 0;
    uint4 sa = make_uint4(0, 0, 0, 0), sb = make_uint4(0, 1, 0, 0);
    const uint32_t g = j < nv ? dvals[j] : 0xffffffffu;
    if (g < (uint64_t)n) {   // one gather per splat
        const uint4 r = rect[g];
        const Footprint f = fp_unpack(r);
        cnt = fp_count(f);
        if (cnt > 0) {
            const uint32_t tx = (uint32_t)tiles_x, t0 = 0;
            const uint32_t W = f.x1 - f.x0, rows = f.y1 - f.y0;
            const uint32_t wt = fp_top_width(f);
            const uint32_t mid = rows > 1 ? (rows - 2) * W : 0;
            sa = make_uint4(g, t0 + f.y0 * tx + f.x0 + (f.trims & 0xffu), wt, wt + mid);
            sb = make_uint4(t0 + (f.y0 + 1) * tx + f.x0, W, t0 + (f.y1 - 1) * tx + f.x0 + ((f.trims >> 16) & 0xffu),
                            tx);
        }
    }
    const uint32_t incl = warp_incl_scan(cnt, lane);
    s_start[threadIdx.x] = incl - cnt;
    s_a[threadIdx.x] = sa;
    s_b[threadIdx.x] = sb;
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    uint32_t warp_base = boff[blockIdx.x];
    for (int w = 0; w < warp; ++w) warp_base += warp_tot[w];
    const uint32_t run = warp_tot[warp];
    const int g0 = warp * 32;
    const uint32_t start = incl - cnt;
    const bool has = cnt > 0;
    for (uint32_t q0 = 0; q0 < run; q0 += 32) {
        // owner of copy q0 + lane: the slots with copies are a prefix of the warp (every
        // survivor has one, the slots past the last survivor none), their runs in slot order,
        // so the owner is the number of runs that start at or before the copy, minus one: the
        // runs starting before q0 (a ballot) plus those starting in q0 .. q0 + lane (an OR of
        // their start bits)
        const uint32_t nb = __popc(__ballot_sync(0xffffffffu, has && start < q0));
        const uint32_t in = __reduce_or_sync(0xffffffffu, (has && start >= q0 && start - q0 < 32u) ? 1u << (start - q0)
                                                                                                 : 0u);
        const uint32_t q = q0 + lane;
        if (q >= run) continue;   // the last round; no collective follows in it
        const int owner = (int)(nb + __popc(in & (0xffffffffu >> (31 - lane)))) - 1;
        const int lo = owner < 0 ? 0 : owner;
        const uint4 a = s_a[g0 + lo];
        const uint32_t k = q - s_start[g0 + lo];
        uint32_t tile;
        if (k < a.z) {
            tile = a.y + k;                           // top row
        } else {
            const uint4 b = s_b[g0 + lo];
            if (k < a.w) {                            // middle rows: row = kk / W
                const uint32_t kk = k - a.z;
                uint32_t r = (uint32_t)((float)kk * __frcp_rn((float)b.y));
                if (r * b.y > kk) --r;
                else if ((r + 1) * b.y <= kk) ++r;
                tile = b.x + r * b.w + (kk - r * b.y);
            } else {
                tile = b.z + (k - a.w);               // bottom row
            }
        }
        keys[warp_base + q] = (KT)tile;
        vals[warp_base + q] = a.x;
    }
}

__global__ void ranges_kernel32(const uint32_t* __restrict__ keys, const Ctrl* __restrict__ ctrl, int64_t cap,
                                uint2* __restrict__ ranges) {
    if (ctrl->error) return;
    const int64_t m = min((int64_t)ctrl->num_keys, cap);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = keys[j];
        if (j == 0 || keys[j - 1] != t) ranges[t].x = (uint32_t)j;
        if (j == m - 1 || keys[j + 1] != t) ranges[t].y = (uint32_t)(j + 1);
    }
}

static int sms() {
    int dev = 0, s = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    return s;
}

void launch_depth_sort(const Layout& L, char* ws, cudaStream_t stream) {
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.off_ctrl);
    const uint32_t* touched = reinterpret_cast<const uint32_t*>(ws + L.off_touched);
    const int blocks_n = (int)L.prep_blocks;
    uint32_t* bvis = reinterpret_cast<uint32_t*>(ws + L.off_bsum);
    uint32_t* bvis_off = reinterpret_cast<uint32_t*>(ws + L.off_boff);
    uint32_t* dk0 = reinterpret_cast<uint32_t*>(ws + L.off_dkeys[0]);
    uint32_t* dk1 = reinterpret_cast<uint32_t*>(ws + L.off_dkeys[1]);
    uint32_t* dv0 = reinterpret_cast<uint32_t*>(ws + L.off_dvals[0]);
    uint32_t* dv1 = reinterpret_cast<uint32_t*>(ws + L.off_dvals[1]);
    uint32_t* hist = reinterpret_cast<uint32_t*>(ws + L.off_hist);
    uint32_t* lb = reinterpret_cast<uint32_t*>(ws + L.off_lookback);
    // 1. compaction of the surviving splats, in index order (the preprocess wrote the
    //    per-block survivor counts)
    launch_scan_sums(bvis, bvis_off, L.prep_blocks, &ctrl->num_visible, &ctrl->error, 0,
                     reinterpret_cast<unsigned long long*>(ws + L.off_scan_lb), &ctrl->scan_ticket[0], L.spin_limit,
                     stream);
    // the compaction writes buffer 1 when the depth sort has an odd number of passes, so
    // that the passes ping-pong (a pass never writes its own input) and end in buffer 0
    const bool odd = (L.depth_passes & 1) != 0;
    uint32_t* ck = odd ? dk1 : dk0;
    uint32_t* cv = odd ? dv1 : dv0;
    launch_k(true, compact_visible, (blocks_n + kBlocksPerCta - 1) / kBlocksPerCta, kPrepThreads, 0, stream,
             touched, reinterpret_cast<const float*>(ws + L.off_depth), L.n, (int64_t)blocks_n,
             (const uint32_t*)bvis_off, ck, cv);
    // 2. sort by depth; the sorted indices land in buffer 0 (the sorted depths are not needed:
    //    the last pass writes only the indices)
    launch_sort_generic<uint32_t>(ck, cv, dk0, dv0, dk1, dv1, L.n, &ctrl->num_visible, L.depth_passes, hist, lb,
                                  ctrl->part_counter, &ctrl->error, stream, nullptr, 0,
                                  32 - L.digit_bits * (L.depth_passes - 1), depth_sort_kpt(L.n, L.digit_bits),
                                  L.spin_limit, L.digit_bits, false);
}

SideStream* side_stream(cudaStream_t stream) {
    // one side stream per (device, main stream) of this host thread, so that renders issued
    // on different streams (as the lanes of a batch) keep their independence
    constexpr size_t kMaxSides = 64;
    thread_local std::map<std::pair<int, cudaStream_t>, SideStream> sides;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    const auto key = std::make_pair(dev, stream);
    auto it = sides.find(key);
    if (it == sides.end()) {
        if (sides.size() >= kMaxSides) return nullptr;
        SideStream sd;
        if (cudaStreamCreateWithFlags(&sd.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sd.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&sd.join, cudaEventDisableTiming) != cudaSuccess)
            sd.s = nullptr;
        it = sides.emplace(key, sd).first;
    }
    return it->second.s ? &it->second : nullptr;
}

bool side_fork(SideStream* side, cudaStream_t stream) {
    return cudaEventRecord(side->fork, stream) == cudaSuccess &&
           cudaStreamWaitEvent(side->s, side->fork, 0) == cudaSuccess;
}

bool side_join_point(SideStream* side, cudaStream_t stream) {
    if (cudaEventRecord(side->join, side->s) == cudaSuccess) return true;
    // cannot join: let the host wait for the side stream instead (a capture in progress is
    // invalid after the failed call and ends with an error)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone)
        cudaStreamSynchronize(side->s);
    return false;
}

void launch_depth_first(const Layout& L, char* ws, cudaStream_t stream, StageMark mark, int mark_index) {
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.off_ctrl);
    const uint32_t* touched = reinterpret_cast<const uint32_t*>(ws + L.off_touched);
    const int blocks_n = (int)L.prep_blocks;
    uint32_t* dv0 = reinterpret_cast<uint32_t*>(ws + L.off_dvals[0]);
    // The per-tile counts of the counts-first tile sort need only the footprints: outside a
    // profiled render they run on a side stream, beside the depth sort and the emission
    // (which leave most SMs idle at a million splats), and join before the tile passes.
    SideStream* side = (L.tile_fused && !mark) ? side_stream(stream) : nullptr;
    if (side && !side_fork(side, stream)) side = nullptr;
    bool counted = false;   // the counts were queued on the side stream
    if (side) {
        launch_tile_counts(L, ws, side->s);
        counted = true;
        if (!side_join_point(side, stream)) side = nullptr;
    }
    launch_depth_sort(L, ws, stream);
    if (mark) mark(mark_index, stream);
    // 3. tile copies in depth order
    uint32_t* bsum2 = reinterpret_cast<uint32_t*>(ws + L.off_bsum2);
    uint32_t* boff2 = reinterpret_cast<uint32_t*>(ws + L.off_boff2);
    launch_k(true, depth_touch_sums, (blocks_n + kBlocksPerCta - 1) / kBlocksPerCta, kPrepThreads, 0, stream,
             (const uint32_t*)dv0, touched, L.n, (int64_t)blocks_n, (const Ctrl*)ctrl, bsum2);
    launch_scan_sums(bsum2, boff2, L.prep_blocks, &ctrl->num_keys, &ctrl->error, L.cap,
                     reinterpret_cast<unsigned long long*>(ws + L.off_scan_lb) + L.scan_slot_words,
                     &ctrl->scan_ticket[1], L.spin_limit, stream);
    if (L.tile_fused) {
        // 3'-5'. 16-bit tile keys in depth order; per-tile counts -> histograms and ranges;
        // the passes (tile_sort.cu)
        launch_k(true, emit_tiles<uint16_t>, blocks_n, kPrepThreads, 0, stream, (const uint32_t*)dv0,
                 reinterpret_cast<const uint4*>(ws + L.off_rect), L.n, (const uint32_t*)boff2, L.tiles_x,
                 (const Ctrl*)ctrl, reinterpret_cast<uint16_t*>(ws + L.off_keys[0]),
                 reinterpret_cast<uint32_t*>(ws + L.off_vals[0]));
        if (mark) mark(mark_index + 1, stream);
        if (side) cudaStreamWaitEvent(stream, side->join, 0);
        else if (!counted) launch_tile_counts(L, ws, stream);
        if (mark) mark(mark_index + 2, stream);
        launch_tile_passes(L, ws, stream);
        return;
    }
    uint32_t* k0 = reinterpret_cast<uint32_t*>(ws + L.off_keys[0]);
    uint32_t* k1 = reinterpret_cast<uint32_t*>(ws + L.off_keys[1]);
    uint32_t* v0 = reinterpret_cast<uint32_t*>(ws + L.off_vals[0]);
    uint32_t* v1 = reinterpret_cast<uint32_t*>(ws + L.off_vals[1]);
    emit_tiles<uint32_t><<<blocks_n, kPrepThreads, 0, stream>>>(
        dv0, reinterpret_cast<const uint4*>(ws + L.off_rect), L.n, boff2, L.tiles_x, ctrl, k0, v0);
    if (mark) mark(mark_index + 1, stream);
    // 4. stable sort by tile id; the result lands in buffer L.sorted_buffer
    const int tp = L.passes;
    uint32_t* ka = L.sorted_buffer ? k1 : k0;
    uint32_t* va = L.sorted_buffer ? v1 : v0;
    uint32_t* kb = L.sorted_buffer ? k0 : k1;
    uint32_t* vb = L.sorted_buffer ? v0 : v1;
    launch_sort_generic<uint32_t>(k0, v0, ka, va, kb, vb, L.cap, &ctrl->num_keys, tp,
                                  reinterpret_cast<uint32_t*>(ws + L.off_hist_tile),
                                  reinterpret_cast<uint32_t*>(ws + L.off_lookback_tile),
                                  ctrl->part_counter + kMaxPasses, &ctrl->error, stream, mark, mark_index + 2,
                                  L.tile_bits - L.digit_bits * (tp - 1), 16, L.spin_limit, L.digit_bits);
    (void)sms;
}

void launch_ranges32(const Layout& L, char* ws, cudaStream_t stream) {
    const int64_t want = (L.cap + 255) / 256, lim = (int64_t)sms() * 8;
    const int blocks = (int)(want < 1 ? 1 : (want < lim ? want : lim));
    ranges_kernel32<<<blocks, 256, 0, stream>>>(reinterpret_cast<const uint32_t*>(ws + L.off_keys[L.sorted_buffer]),
                                                reinterpret_cast<const Ctrl*>(ws + L.off_ctrl), L.cap,
                                                reinterpret_cast<uint2*>(ws + L.off_ranges));
}

}  // namespace vis
