// Tile-first ordering of the splats (sort_mode 3): every tile's list in front-to-back order
// (the order of Algorithm 1's depth sort, section 3.4, restricted to the tile), without a
// global sort.
//
//   tf_count_kernel   CTA b takes a contiguous range of Gaussians, adds their footprints to
//                     a 2D difference array in shared memory and turns it into its per-tile
//                     copy counts (2D prefix sums); one global atomic per (CTA, tile)
//                     reserves the CTA's slice of the tile's list: within[b][t];
//   tf_scan_kernel    per-tile totals -> starts (exclusive scan in raster order), ranges,
//                     the copy count M (capacity checked), and the tiles sorted into work
//                     lists by size (<= 1024, <= 4096, <= 16384, larger);
//   tf_emit_kernel    the same CTAs enumerate their Gaussians' copies again and place each
//                     at start[t] + within[b][t] + (running count in shared memory), as the
//                     64-bit key (float bits of the view depth) << 32 | Gaussian index;
//   tf_sort_kernel    each tile's keys sorted in shared memory by a bitonic network (keys
//                     padded to a power of two with all-ones); the sorted indices are the
//                     tile's list. Keys are unique (the index is in the low word), so the
//                     order is (depth, index) whatever order the emission left;
//   tf_merge_kernel   tiles above 16384 copies are sorted as runs of 16384 by
//                     tf_sort_kernel and merged pairwise, one round per launch (a key's
//                     place in the merged run is its place in its own run plus its rank in
//                     the other, found by binary search).
// The result is bit for bit the (tile, depth, index) order of the other sort modes.
#include "vis_internal.cuh"
#include "footprint.cuh"

namespace vis {

constexpr int kTfThreads = 512;

// ---- per-CTA counts and reservations ----
__global__ void __launch_bounds__(kTfThreads)
tf_count_kernel(const uint4* __restrict__ rect, int64_t n, int64_t chunk, int tiles_x, int tiles_y,
                uint32_t* __restrict__ total, uint32_t* __restrict__ within) {
    extern __shared__ int P[];
    const int nt = tiles_x * tiles_y;
    const uint32_t tx = (uint32_t)tiles_x, ty = (uint32_t)tiles_y;
    for (int i = threadIdx.x; i < nt; i += kTfThreads) P[i] = 0;
    __syncthreads();
    const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kTfThreads) fp_add_to_diff(P, fp_unpack(rect[i]), tx, ty);
    __syncthreads();
    for (int y = threadIdx.x; y < tiles_y; y += kTfThreads) {   // prefix along each row
        int run = 0;
        for (int x = 0; x < tiles_x; ++x) { run += P[y * tiles_x + x]; P[y * tiles_x + x] = run; }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < tiles_x; x += kTfThreads) {   // then along each column
        int run = 0;
        for (int y = 0; y < tiles_y; ++y) { run += P[y * tiles_x + x]; P[y * tiles_x + x] = run; }
    }
    __syncthreads();
    uint32_t* row = within + (size_t)blockIdx.x * nt;
    for (int t = threadIdx.x; t < nt; t += kTfThreads) {
        const int c = P[t];
        if (c > 0) row[t] = atomicAdd(&total[t], (uint32_t)c);
    }
}

// ---- starts, ranges, M, work lists ----
// lists: [0, nt) tiles of <= 1024 copies, [nt, 2nt) <= 4096, [2nt, 3nt) tiles above 16384,
// [3nt, ...) tiles of <= 16384 and the runs of 16384 of the larger ones (item = tile |
// run << 16; at most nt + M / 16384 + nt items).
__global__ void __launch_bounds__(1024)
tf_scan_kernel(const uint32_t* __restrict__ total, int nt, int64_t cap, uint2* __restrict__ ranges,
               uint32_t* __restrict__ start_out, uint32_t* __restrict__ lists, Ctrl* __restrict__ ctrl) {
    __shared__ unsigned long long s_warp[32];
    __shared__ uint32_t s_cnt[4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 4) s_cnt[tid] = 0;
    const int per = (nt + 1023) / 1024;
    const int t0 = tid * per, t1 = min(nt, t0 + per);
    unsigned long long local = 0;
    for (int t = t0; t < t1; ++t) local += total[t];
    unsigned long long incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    unsigned long long start = incl - local, all = 0;
    for (int w = 0; w < 32; ++w) {
        if (w < warp) start += s_warp[w];
        all += s_warp[w];
    }
    const bool over = all > (unsigned long long)cap;
    for (int t = t0; t < t1; ++t) {
        const uint32_t c = total[t];
        const uint32_t s = (uint32_t)min(start, (unsigned long long)0xffffffffu);
        ranges[t] = (c && !over) ? make_uint2(s, s + c) : make_uint2(0u, 0u);
        start_out[t] = s;
        start += c;
        if (c == 0 || over) continue;
        if (c <= 1024) lists[atomicAdd(&s_cnt[0], 1u)] = (uint32_t)t;
        else if (c <= 4096) lists[nt + atomicAdd(&s_cnt[1], 1u)] = (uint32_t)t;
        else if (c <= 16384) lists[3 * nt + atomicAdd(&s_cnt[2], 1u)] = (uint32_t)t;
        else {
            if (c > (16384u << kTfMergeRounds)) atomicOr(&ctrl->error, kErrTileOverflow);
            lists[2 * nt + atomicAdd(&s_cnt[3], 1u)] = (uint32_t)t;
            for (uint32_t r = 0; r * 16384u < c; ++r) lists[3 * nt + atomicAdd(&s_cnt[2], 1u)] = (uint32_t)t | (r << 16);
        }
    }
    __syncthreads();
    if (tid < 4) ctrl->tf_count[tid] = s_cnt[tid];
    if (tid == 0) {
        ctrl->num_keys = (uint32_t)min(all, (unsigned long long)0xffffffffu);
        if (over) atomicOr(&ctrl->error, kErrCapacity);
    }
}

// ---- emission into the reserved slices ----
__global__ void __launch_bounds__(kTfThreads)
tf_emit_kernel(const uint4* __restrict__ rect, const float* __restrict__ depth, int64_t n, int64_t chunk,
               int tiles_x, int nt, const uint32_t* __restrict__ start, const uint32_t* __restrict__ within,
               const Ctrl* __restrict__ ctrl, uint64_t* __restrict__ keys) {
    extern __shared__ uint32_t slot[];   // nt: next position of this CTA's copies per tile
    __shared__ uint32_t s_start[kTfThreads];
    __shared__ uint4 s_a[kTfThreads], s_b[kTfThreads];
    if (ctrl->error & kErrCapacity) return;
    const uint32_t* row = within + (size_t)blockIdx.x * nt;
    for (int t = threadIdx.x; t < nt; t += kTfThreads) slot[t] = start[t] + row[t];   // untouched tiles: unused
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g0 = warp * 32;
    const uint32_t tx = (uint32_t)tiles_x;
    const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    for (int64_t base = i0; base < i1; base += kTfThreads) {
        // per Gaussian: copies unrolled into row segments (as in the depth-order emission)
        const int64_t i = base + threadIdx.x;
        uint32_t cnt = 0;
        uint4 sa = make_uint4(0, 0, 0, 0), sb = make_uint4(0, 1, 0, 0);
        if (i < i1) {
            const Footprint f = fp_unpack(rect[i]);
            cnt = fp_count(f);
            if (cnt > 0) {
                const uint32_t W = f.x1 - f.x0, rows = f.y1 - f.y0, wt = fp_top_width(f);
                const uint32_t mid = rows > 1 ? (rows - 2) * W : 0;
                sa = make_uint4((uint32_t)i, f.y0 * tx + f.x0 + (f.trims & 0xffu), wt, wt + mid);
                sb = make_uint4((f.y0 + 1) * tx + f.x0, W, (f.y1 - 1) * tx + f.x0 + ((f.trims >> 16) & 0xffu),
                                __float_as_uint(depth[i]));
            }
        }
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const uint32_t run = __shfl_sync(0xffffffffu, incl, 31);
        s_start[threadIdx.x] = incl - cnt;
        s_a[threadIdx.x] = sa;
        s_b[threadIdx.x] = sb;
        __syncwarp();
        for (uint32_t q = lane; q < run; q += 32) {
            int lo = 0;   // owner: the last slot whose start is <= q (it has copies)
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (s_start[g0 + lo + step] <= q) lo += step;
            const uint4 a = s_a[g0 + lo], b = s_b[g0 + lo];
            const uint32_t k = q - s_start[g0 + lo];
            uint32_t tile;
            if (k < a.z) {
                tile = a.y + k;
            } else if (k < a.w) {
                const uint32_t kk = k - a.z;
                uint32_t r = (uint32_t)((float)kk * __frcp_rn((float)b.y));
                if (r * b.y > kk) --r;
                else if ((r + 1) * b.y <= kk) ++r;
                tile = b.x + r * tx + (kk - r * b.y);
            } else {
                tile = b.z + (k - a.w);
            }
            const uint32_t pos = atomicAdd(&slot[tile], 1u);
            keys[pos] = ((uint64_t)b.w << 32) | a.x;
        }
        __syncwarp();
    }
}

// ---- per-tile bitonic sort in shared memory ----
// items: tile ids (or tile | run << 16 for runs of tiles above NMAX copies); persistent
// CTAs take items grid-strided. Whole tiles write their indices to vals; runs write their
// sorted keys back for the merge.
template <int NMAX, int T>
__global__ void __launch_bounds__(T)
tf_sort_kernel(const uint32_t* __restrict__ items, const uint32_t* __restrict__ count,
               const uint2* __restrict__ ranges, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    extern __shared__ uint64_t s[];   // NMAX keys
    const uint32_t n_items = *count;
    for (uint32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const uint32_t item = items[it];
        const uint32_t t = item & 0xffffu, run = item >> 16;
        const uint2 rg = ranges[t];
        const uint32_t len = rg.y - rg.x;
        const bool whole = len <= (uint32_t)NMAX;
        const uint32_t first = rg.x + run * (uint32_t)NMAX;
        const uint32_t n = whole ? len : min((uint32_t)NMAX, len - run * (uint32_t)NMAX);
        uint32_t N = 2;
        while (N < n) N <<= 1;
        for (uint32_t i = threadIdx.x; i < N; i += T) s[i] = i < n ? keys[first + i] : ~0ull;
        __syncthreads();
        for (uint32_t k = 2; k <= N; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t p = threadIdx.x; p < N / 2; p += T) {
                    const uint32_t i0 = ((p & ~(j - 1)) << 1) | (p & (j - 1)), i1 = i0 + j;
                    const uint64_t a = s[i0], b = s[i1];
                    const bool up = (i0 & k) == 0;
                    if ((a > b) == up) { s[i0] = b; s[i1] = a; }
                }
                __syncthreads();
            }
        }
        if (whole) {
            for (uint32_t i = threadIdx.x; i < n; i += T) vals[first + i] = (uint32_t)s[i];
        } else {
            for (uint32_t i = threadIdx.x; i < n; i += T) keys[first + i] = s[i];
        }
        __syncthreads();
    }
}

// one pairwise merge round of the runs of the tiles above NMAX copies: runs of L = NMAX << r
// keys, run 2q merged with run 2q + 1 through tmp; the last round writes the indices to vals
template <int NMAX>
__global__ void __launch_bounds__(1024)
tf_merge_kernel(const uint32_t* __restrict__ big, const uint32_t* __restrict__ count, const uint2* __restrict__ ranges,
                int r, bool last, uint64_t* __restrict__ keys, uint64_t* __restrict__ tmp,
                uint32_t* __restrict__ vals) {
    const uint32_t n_big = *count;
    for (uint32_t it = blockIdx.x; it < n_big; it += gridDim.x) {
        const uint2 rg = ranges[big[it]];
        const uint32_t len = rg.y - rg.x;
        const uint64_t L = (uint64_t)NMAX << r;
        if (L < len) {   // runs to merge at this round
            for (uint32_t i = threadIdx.x; i < len; i += 1024) {
                const uint64_t x = keys[rg.x + i];
                const uint64_t run = i / L, own0 = run * L;
                const uint64_t pair0 = (run & ~1ull) * L;
                const uint64_t other0 = (run & 1) ? own0 - L : own0 + L;
                uint64_t pos = i;
                if (other0 < len) {
                    // rank of x in the other run (keys are unique)
                    uint64_t lo = other0, hi = min((uint64_t)len, other0 + L);
                    while (lo < hi) {
                        const uint64_t mid = (lo + hi) >> 1;
                        if (keys[rg.x + mid] < x) lo = mid + 1; else hi = mid;
                    }
                    pos = pair0 + (i - own0) + (lo - other0);
                }
                tmp[rg.x + pos] = x;
            }
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < len; i += 1024) keys[rg.x + i] = tmp[rg.x + i];
            __syncthreads();
        }
        if (last)
            for (uint32_t i = threadIdx.x; i < len; i += 1024) vals[rg.x + i] = (uint32_t)keys[rg.x + i];
        __syncthreads();
    }
}

static int sm_count_tf() {
    int dev = 0, s = 148;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        s = 148;
    return s;
}

int64_t tf_grid(int64_t n, int64_t ntiles) {
    // CTAs of the count and emission kernels: two per SM while their per-tile shared arrays
    // allow it, at least 2048 Gaussians each
    const int64_t sms = sm_count_tf();
    const int64_t per_sm = ntiles * 4 <= 100 * 1024 ? 2 : 1;
    int64_t g = (n + 2047) / 2048;
    if (g > sms * per_sm) g = sms * per_sm;
    return g < 1 ? 1 : g;
}

void launch_tile_first(const Layout& L, char* ws, cudaStream_t stream, StageMark mark, int mark_index) {
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.off_ctrl);
    const int nt = (int)L.ntiles;
    const uint4* rect = reinterpret_cast<const uint4*>(ws + L.off_rect);
    uint32_t* total = reinterpret_cast<uint32_t*>(ws + L.off_tf_total);
    uint32_t* within = reinterpret_cast<uint32_t*>(ws + L.off_tf_within);
    uint32_t* start = reinterpret_cast<uint32_t*>(ws + L.off_tf_start);
    uint32_t* lists = reinterpret_cast<uint32_t*>(ws + L.off_tf_lists);
    uint2* ranges = reinterpret_cast<uint2*>(ws + L.off_ranges);
    uint64_t* keys = reinterpret_cast<uint64_t*>(ws + L.off_keys[0]);
    uint64_t* tmp = reinterpret_cast<uint64_t*>(ws + L.off_keys[1]);
    uint32_t* vals = reinterpret_cast<uint32_t*>(ws + L.off_vals[0]);
    const int grid = (int)L.tf_grid;
    const size_t tsm = sizeof(uint32_t) * (size_t)nt;
    static std::atomic<uint64_t> attr_dev{0};   // devices whose attributes are set
    if (once_per_device(attr_dev)) {
        const int most = (int)(sizeof(uint32_t) * kTileFusedMaxTiles);
        cudaFuncSetAttribute(tf_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        cudaFuncSetAttribute(tf_emit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        cudaFuncSetAttribute(tf_sort_kernel<1024, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, 1024 * 8);
        cudaFuncSetAttribute(tf_sort_kernel<4096, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4096 * 8);
        cudaFuncSetAttribute(tf_sort_kernel<16384, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 * 8);
    }
    tf_count_kernel<<<grid, kTfThreads, tsm, stream>>>(rect, L.n, L.tf_chunk, L.tiles_x, L.tiles_y, total, within);
    tf_scan_kernel<<<1, 1024, 0, stream>>>(total, nt, L.cap, ranges, start, lists, ctrl);
    if (mark) mark(mark_index, stream);
    tf_emit_kernel<<<grid, kTfThreads, tsm, stream>>>(rect, reinterpret_cast<const float*>(ws + L.off_depth), L.n,
                                                      L.tf_chunk, L.tiles_x, nt, start, within, ctrl, keys);
    if (mark) mark(mark_index + 1, stream);
    const int sms = sm_count_tf();
    tf_sort_kernel<1024, 256><<<8 * sms, 256, 1024 * 8, stream>>>(lists, &ctrl->tf_count[0], ranges, keys, vals);
    tf_sort_kernel<4096, 512><<<3 * sms, 512, 4096 * 8, stream>>>(lists + nt, &ctrl->tf_count[1], ranges, keys, vals);
    tf_sort_kernel<16384, 1024><<<sms, 1024, 16384 * 8, stream>>>(lists + 3 * nt, &ctrl->tf_count[2], ranges, keys,
                                                                   vals);
    for (int r = 0; r < kTfMergeRounds; ++r)
        tf_merge_kernel<16384><<<sms, 1024, 0, stream>>>(lists + 2 * nt, &ctrl->tf_count[3], ranges, r,
                                                         r == kTfMergeRounds - 1, keys, tmp, vals);
}

}  // namespace vis
