// Counts-first tile sort of the depth-sorted splats' copies (sort_mode 1 on tile grids of
// at most kTileFusedMaxTiles tiles): the stable sort by tile id that turns the depth order
// of Algorithm 1's radix sort (section 3.4) into every tile's front-to-back list.
//
//   tile_count_kernel  per-tile copy counts from the splats' footprints: every tile
//                      box adds +1/-1/-1/+1 at its four corners of a 2D difference
//                      array (shared memory per CTA, flushed with one global atomic per
//                      non-zero entry), and the trimmed ends of its top and bottom rows
//                      are taken out again the same way;
//   tile_scan_kernel   2D prefix sums -> counts; the digit histograms of both radix
//                      passes and every tile's [start, end) range follow from the
//                      counts alone (exclusive scan over the tiles in raster order),
//                      so no pass over the keys builds histograms or finds ranges;
//   passes             sort_pass<uint16_t> over the 16-bit tile ids emitted in depth
//                      order (emit_tiles), low byte then high byte; the last pass
//                      writes only the Gaussian indices.
// The result is the (tile, depth, index) order of the 64-bit key sort, bit for bit.
#include "onesweep.cuh"
#include "footprint.cuh"

namespace vis {

// ---- per-tile counts ----
__global__ void __launch_bounds__(1024)
tile_count_kernel(const uint4* __restrict__ rect, int64_t n, int tiles_x, int tiles_y, int* __restrict__ gdiff) {
    pdl_entry();
    extern __shared__ int diff[];
    const int nt = tiles_x * tiles_y;
    const uint32_t tx = (uint32_t)tiles_x, ty = (uint32_t)tiles_y;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) diff[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        fp_add_to_diff(diff, fp_unpack(rect[i]), tx, ty);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nt; i += blockDim.x)
        if (diff[i]) atomicAdd(&gdiff[i], diff[i]);
}

// inclusive warp scan of one value per lane
__device__ __forceinline__ int warp_scan_incl(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// One CTA of 1024 threads. hist: [2][256] digit histograms (low byte, high byte of the
// tile id); ranges: [start, end) per tile, (0, 0) for an empty tile. The 2D prefix sums run
// one warp per row, then one warp per column, 32 entries at a time with warp scans, on rows
// padded to tiles_x + 1 words (an odd stride: the column pass reads 32 rows without bank
// conflicts). The histograms are plain sums (low byte: tiles d, d + 256, ...; high byte: a
// block of 256); the ranges come from an exclusive scan in raster order taken 1024 tiles per
// round (warp scans, then a scan of the 32 warp totals), written coalesced.
__global__ void __launch_bounds__(1024)
tile_scan_kernel(const int* __restrict__ gdiff, int tiles_x, int tiles_y, uint32_t* __restrict__ hist,
                 uint2* __restrict__ ranges, uint32_t* __restrict__ order) {
    pdl_entry();
    extern __shared__ int P[];
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    __shared__ uint32_t s_bucket[kOrderBuckets];
    const int nt = tiles_x * tiles_y;
    const int ld = tiles_x + 1;   // padded row stride
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < nt; i += 1024) {
        const int y = i / tiles_x;
        P[y * ld + (i - y * tiles_x)] = gdiff[i];
    }
    if (tid == 0) s_carry = 0;
    for (int i = tid; i < kOrderBuckets; i += 1024) s_bucket[i] = 0;
    __syncthreads();
    for (int y = warp; y < tiles_y; y += 32) {   // prefix along each row
        int carry = 0;
        for (int x0 = 0; x0 < tiles_x; x0 += 32) {
            const int x = x0 + lane;
            const int v = x < tiles_x ? P[y * ld + x] : 0;
            const int incl = warp_scan_incl(v, lane) + carry;
            if (x < tiles_x) P[y * ld + x] = incl;
            carry = __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    __syncthreads();
    for (int x = warp; x < tiles_x; x += 32) {   // then along each column: counts
        int carry = 0;
        for (int y0 = 0; y0 < tiles_y; y0 += 32) {
            const int y = y0 + lane;
            const int v = y < tiles_y ? P[y * ld + x] : 0;
            const int incl = warp_scan_incl(v, lane) + carry;
            if (y < tiles_y) P[y * ld + x] = incl;
            carry = __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    __syncthreads();
    auto count = [&](int t) { const int y = t / tiles_x; return (uint32_t)P[y * ld + (t - y * tiles_x)]; };
    // digit histograms of the two passes
    if (tid < kRadix) {
        uint32_t h = 0;
        for (int t = tid; t < nt; t += kRadix) h += count(t);
        hist[tid] = h;
    }
    for (int d = warp; d < kRadix; d += 32) {
        uint32_t h = 0;
        for (int t = d * kRadix + lane; t < min(nt, (d + 1) * kRadix); t += 32) h += count(t);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
        if (lane == 0) hist[kRadix + d] = h;
    }
    // exclusive scan of the counts in raster order, 1024 tiles per round
    for (int t0 = 0; t0 < nt; t0 += 1024) {
        const int t = t0 + tid;
        const uint32_t c = t < nt ? count(t) : 0u;
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = s_warp[lane];
            uint32_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += v;
            }
            s_warp[lane] = wi - w;   // exclusive warp offsets
        }
        __syncthreads();
        const uint32_t start = s_carry + s_warp[warp] + incl - c;
        if (t < nt) ranges[t] = c ? make_uint2(start, start + c) : make_uint2(0u, 0u);
        __syncthreads();
        if (tid == 1023) s_carry = start + c;
        __syncthreads();
    }
    // compositing order: tiles by decreasing count (log-spaced buckets, two per octave), so
    // that the longest tiles start first and the launch ends on short ones. The lanes of a
    // warp with the same bucket (found with one ballot per bucket bit) add to it once.
    const int nt32 = (nt + 31) & ~31;
    auto peers_of = [&](int b) {
        uint32_t pm = __ballot_sync(0xffffffffu, b >= 0);
#pragma unroll
        for (int k = 0; k < kOrderBits; ++k) {
            const uint32_t bit = (uint32_t)(b >> k) & 1u;
            const uint32_t bal = __ballot_sync(0xffffffffu, bit);
            pm &= bit ? bal : ~bal;
        }
        return pm;
    };
    for (int t = tid; t < nt32; t += 1024) {   // a warp's 32 tiles are all in or all out of the loop
        const int b = t < nt ? order_bucket(count(t)) : -1;
        const uint32_t peers = peers_of(b);
        if (b >= 0 && lane == __ffs(peers) - 1) atomicAdd(&s_bucket[b], (uint32_t)__popc(peers));
    }
    __syncthreads();
    static_assert(kOrderBuckets == 64, "the bucket scan below takes two buckets per lane");
    if (warp == 0) {   // exclusive scan of the bucket sizes, kOrderBuckets = 2 x 32
        const uint32_t v0 = s_bucket[2 * lane], v1 = s_bucket[2 * lane + 1], tot = v0 + v1;
        uint32_t incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += x;
        }
        s_bucket[2 * lane] = incl - tot;
        s_bucket[2 * lane + 1] = incl - tot + v0;
    }
    __syncthreads();
    for (int t = tid; t < nt32; t += 1024) {
        const int b = t < nt ? order_bucket(count(t)) : -1;
        const uint32_t peers = peers_of(b);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (b >= 0 && lane == leader) base = atomicAdd(&s_bucket[b], (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (b >= 0) order[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)t;
    }
}

// Clears the look-back rows the tile passes of this render read, in their own region (not in
// the cleared workspace region): per pass, the rows of the partitions of min(copies, cap) keys
// and those of their groups. The copies are the sum of the first pass's digit histogram, which
// the tile scan has just written.
__global__ void __launch_bounds__(256)
clear_tile_lookback(const uint32_t* __restrict__ hist, int64_t cap, int64_t parts_cap, int passes,
                    uint32_t* __restrict__ lb) {
    pdl_entry();
    constexpr int64_t kPart = sort_partition<uint16_t>();
    constexpr int kGroup = lookback_group(2, kRadixBits);
    __shared__ uint32_t s_m;
    if (threadIdx.x < 32) {
        uint32_t v = 0;
        for (int i = threadIdx.x; i < kRadix; i += 32) v += hist[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) s_m = v;
    }
    __syncthreads();
    const int64_t m = min((int64_t)s_m, cap);
    const int64_t parts = min((m + kPart - 1) / kPart, parts_cap), groups = (parts + kGroup - 1) / kGroup;
    const int64_t row4 = kRadix / 4;   // 16-byte words per row
    const int64_t pass4 = lookback_rows(parts_cap, kGroup) * row4;
    const int64_t n1 = parts * row4, n2 = groups * row4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    for (int p = 0; p < passes; ++p) {
        uint4* base = reinterpret_cast<uint4*>(lb) + p * pass4;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2; i += stride)
            base[i < n1 ? i : parts_cap * row4 + (i - n1)] = z;
    }
}

static int sm_count_ts() {
    int dev = 0, s = 148;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        s = 148;
    return s;
}

void launch_tile_counts(const Layout& L, char* ws, cudaStream_t stream) {
    static std::atomic<uint64_t> attr_dev{0};   // devices whose attributes are set
    static std::mutex attr_mu;
    set_up_per_device(attr_dev, attr_mu, [] {
        // the largest per-tile counter array of the fused path; the scan's rows are padded by one
        // word (at most 1024 rows at 16-pixel tiles) and it adds ~0.2 KB of static shared
        // memory, within the 227 KB a CTA may use
        const int most = (int)(sizeof(int) * kTileFusedMaxTiles);
        return cudaFuncSetAttribute(tile_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, most) ==
                   cudaSuccess &&
               cudaFuncSetAttribute(tile_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    most + (int)sizeof(int) * 2048) == cudaSuccess;
    });
    const size_t smem = sizeof(int) * (size_t)L.ntiles;
    int* gdiff = reinterpret_cast<int*>(ws + L.off_tdiff);
    const int64_t want = (L.n + 4095) / 4096;
    const int64_t lim = 2 * (int64_t)sm_count_ts();
    const int grid = (int)(want < 1 ? 1 : (want < lim ? want : lim));
    launch_k(true, tile_count_kernel, grid, 1024, smem, stream, reinterpret_cast<const uint4*>(ws + L.off_rect), L.n,
             L.tiles_x, L.tiles_y, gdiff);
    const size_t scan_smem = sizeof(int) * (size_t)(L.tiles_x + 1) * L.tiles_y;
    launch_k(true, tile_scan_kernel, 1, 1024, scan_smem, stream, (const int*)gdiff, L.tiles_x, L.tiles_y,
             reinterpret_cast<uint32_t*>(ws + L.off_hist_tile),
             reinterpret_cast<uint2*>(ws + L.off_ranges), reinterpret_cast<uint32_t*>(ws + L.off_order));
    launch_k(true, clear_tile_lookback, sm_count_ts() / 2, 256, 0, stream,
             (const uint32_t*)(ws + L.off_hist_tile), L.cap, L.sort_parts, L.passes,
             reinterpret_cast<uint32_t*>(ws + L.off_lookback_tile));
}

void launch_tile_passes(const Layout& L, char* ws, cudaStream_t stream) {
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.off_ctrl);
    uint32_t* hist = reinterpret_cast<uint32_t*>(ws + L.off_hist_tile);
    uint32_t* lb = reinterpret_cast<uint32_t*>(ws + L.off_lookback_tile);
    uint16_t* k0 = reinterpret_cast<uint16_t*>(ws + L.off_keys[0]);
    uint16_t* k1 = reinterpret_cast<uint16_t*>(ws + L.off_keys[1]);
    uint32_t* v0 = reinterpret_cast<uint32_t*>(ws + L.off_vals[0]);
    uint32_t* v1 = reinterpret_cast<uint32_t*>(ws + L.off_vals[1]);
    const size_t words = (size_t)lookback_rows(L.sort_parts, lookback_group(2, kRadixBits)) * kRadix;
    // emitted copies in buffer 0; one pass -> values in 1, two passes -> keys + values in 1, then values in 0
    const int low_bits = L.tile_bits < kRadixBits ? L.tile_bits : kRadixBits;
    if (L.passes == 1) {
        launch_sort_pass<uint16_t>(k0, v0, nullptr, v1, L.cap, &ctrl->num_keys, 0, low_bits, hist, lb,
                                   &ctrl->part_counter[kMaxPasses], &ctrl->error, stream, L.spin_limit);
        return;
    }
    launch_sort_pass<uint16_t>(k0, v0, k1, v1, L.cap, &ctrl->num_keys, 0, low_bits, hist, lb,
                               &ctrl->part_counter[kMaxPasses], &ctrl->error, stream, L.spin_limit);
    launch_sort_pass<uint16_t>(k1, v1, nullptr, v0, L.cap, &ctrl->num_keys, kRadixBits, L.tile_bits - kRadixBits,
                               hist + kRadix, lb + words, &ctrl->part_counter[kMaxPasses + 1], &ctrl->error, stream,
                               L.spin_limit);
}

}  // namespace vis
