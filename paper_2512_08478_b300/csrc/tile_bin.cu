// Stable counting binning of depth-sorted splats into tiles (sort_mode 2).
//
// After the depth sort of the surviving splats (Algorithm 1's "Radix Sort" over
// depths), each tile's list must hold its splats in that depth order. Instead of
// emitting (tile, splat) keys and radix-sorting them by tile, the depth-sorted list
// is cut into chunks of C consecutive splats and binned with counts:
//   bin_count       per chunk, a shared-memory histogram of the tiles its splats
//                   cover -> row c of a chunks x tiles count matrix;
//   bin_scan_tiles  per tile, exclusive prefix of its column over the chunks (the
//                   chunk's base inside the tile's list) and the tile's total;
//   (scan of the totals -> start of every tile's list, total M, capacity check)
//   bin_ranges      [start, start + total) of every tile;
//   bin_emit        per chunk again, each warp walks its share of the chunk in depth
//                   order, enumerating (splat, tile) pairs in order; pairs of one
//                   32-pair round that fall in the same tile are ranked with
//                   __match_any_sync, and a per-warp running count per tile (packed
//                   16-bit counters in shared memory, initialised to the exclusive
//                   prefix over the chunk's earlier warps) gives every pair its
//                   final slot: start[t] + chunk base + warp base + rank.
// Every pair of a tile therefore lands in depth order (ties by index, from the
// stable depth sort): the same order as the 64-bit (tile, depth) key sort, with no
// keys stored and the tile ranges produced by the scan.
#include "vis_internal.cuh"
#include "footprint.cuh"

namespace vis {

__global__ void __launch_bounds__(256)
bin_count_kernel(const uint32_t* __restrict__ dvals, const uint4* __restrict__ rect,
                 const uint32_t* __restrict__ num_visible, int64_t C, int ntiles, int tiles_x,
                 uint32_t* __restrict__ counts) {
    extern __shared__ uint32_t cnt[];
    const int64_t nv = *num_visible;
    const int64_t j0 = (int64_t)blockIdx.x * C;
    if (j0 >= nv) return;
    const int64_t j1 = min(nv, j0 + C);
    for (int i = threadIdx.x; i < ntiles; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const Footprint f = fp_unpack(rect[dvals[j]]);
        const uint32_t n = fp_count(f);
        for (uint32_t k = 0; k < n; ++k) atomicAdd(&cnt[fp_tile(f, k, (uint32_t)tiles_x)], 1u);
    }
    __syncthreads();
    uint32_t* row = counts + (size_t)blockIdx.x * ntiles;
    for (int i = threadIdx.x; i < ntiles; i += blockDim.x) row[i] = cnt[i];
}

// One lane per tile, eight warps splitting the chunks of its column.
__global__ void __launch_bounds__(256)
bin_scan_tiles_kernel(const uint32_t* __restrict__ counts, const uint32_t* __restrict__ num_visible, int64_t C,
                      int ntiles, uint32_t* __restrict__ chunk_base, uint32_t* __restrict__ totals) {
    __shared__ uint32_t seg[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nv = *num_visible;
    const int64_t nchunks = (nv + C - 1) / C;
    const int t = blockIdx.x * 32 + lane;
    const bool vt = t < ntiles;
    const int64_t S = (nchunks + 7) / 8;
    const int64_t c0 = warp * S, c1 = min(nchunks, c0 + S);
    uint32_t sum = 0;
    for (int64_t c = c0; c < c1; ++c)
        if (vt) sum += counts[(size_t)c * ntiles + t];
    seg[warp][lane] = sum;
    __syncthreads();
    uint32_t run = 0, tot = 0;
    for (int w = 0; w < 8; ++w) {
        const uint32_t x = seg[w][lane];
        if (w < warp) run += x;
        tot += x;
    }
    if (warp == 0 && vt) totals[t] = tot;
    for (int64_t c = c0; c < c1; ++c)
        if (vt) {
            const uint32_t v = counts[(size_t)c * ntiles + t];
            chunk_base[(size_t)c * ntiles + t] = run;
            run += v;
        }
}

__global__ void bin_ranges_kernel(const uint32_t* __restrict__ tile_start, const uint32_t* __restrict__ totals,
                                  int ntiles, const Ctrl* __restrict__ ctrl, uint2* __restrict__ ranges) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    if (ctrl->error) { ranges[t] = make_uint2(0, 0); return; }
    ranges[t] = make_uint2(tile_start[t], tile_start[t] + totals[t]);
}

template <int NW>
__global__ void __launch_bounds__(NW * 32)
bin_emit_kernel(const uint32_t* __restrict__ dvals, const uint32_t* __restrict__ touched,
                const uint4* __restrict__ rect, const uint32_t* __restrict__ num_visible, int64_t C, int ntiles,
                int tiles_x, const uint32_t* __restrict__ chunk_base, const uint32_t* __restrict__ tile_start,
                const Ctrl* __restrict__ ctrl, int64_t cap, uint32_t* __restrict__ vals_out) {
    extern __shared__ uint32_t wc[];   // [NW][words]: two 16-bit counters per word
    if (ctrl->error & kErrCapacity) return;
    const int64_t nv = *num_visible;
    const int64_t j0 = (int64_t)blockIdx.x * C;
    if (j0 >= nv) return;
    const int64_t j1 = min(nv, j0 + C);
    const int words = (ntiles + 1) >> 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < NW * words; i += NW * 32) wc[i] = 0;
    __syncthreads();
    // this warp's share of the chunk, in depth order
    const int64_t cw = (j1 - j0 + NW - 1) / NW;
    const int64_t s0 = j0 + warp * cw, s1 = min(j1, s0 + cw);
    uint32_t* mine = wc + (size_t)warp * words;
    for (int64_t j = s0 + lane; j < s1; j += 32) {
        const Footprint f = fp_unpack(rect[dvals[j]]);
        const uint32_t n = fp_count(f);
        for (uint32_t k = 0; k < n; ++k) {
            const uint32_t t = fp_tile(f, k, (uint32_t)tiles_x);
            atomicAdd(&mine[t >> 1], 1u << ((t & 1) * 16));
        }
    }
    __syncthreads();
    // exclusive prefix over the warps, per tile (both halves of a word at once)
    for (int i = threadIdx.x; i < words; i += NW * 32) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t v = wc[(size_t)w * words + i];
            wc[(size_t)w * words + i] = run;
            run += v;   // halves never carry: a chunk holds at most 65535 pairs per tile
        }
    }
    __syncthreads();
    const uint32_t* cb = chunk_base + (size_t)blockIdx.x * ntiles;
    const uint32_t lt = (1u << lane) - 1u;
    for (int64_t gb = s0; gb < s1; gb += 32) {
        const int64_t j = gb + lane;
        uint32_t g = 0, cnt = 0;
        uint4 r = make_uint4(0, 0, 0, 0);
        if (j < s1) { g = dvals[j]; cnt = touched[g]; r = rect[g]; }
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const uint32_t start = incl - cnt;
        const uint32_t run = __shfl_sync(0xffffffffu, incl, 31);
        for (uint32_t q0 = 0; q0 < run; q0 += 32) {
            const uint32_t q = q0 + lane;
            const bool active = q < run;
            // owner: the last lane whose start is <= q (zero counts share starts)
            int lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint32_t st = __shfl_sync(0xffffffffu, start, lo + step);
                if (st <= q) lo += step;
            }
            const uint32_t og = __shfl_sync(0xffffffffu, g, lo);
            uint4 orr;
            orr.x = __shfl_sync(0xffffffffu, r.x, lo);
            orr.y = __shfl_sync(0xffffffffu, r.y, lo);
            orr.z = __shfl_sync(0xffffffffu, r.z, lo);
            orr.w = 0;
            const uint32_t ost = __shfl_sync(0xffffffffu, start, lo);
            uint32_t t = 0;
            if (active) t = fp_tile(fp_unpack(orr), q - ost, (uint32_t)tiles_x);
            const uint32_t peers = __match_any_sync(0xffffffffu, active ? t : (0x80000000u | (uint32_t)lane));
            const int leader = __ffs(peers) - 1;
            uint32_t base = 0;
            if (active && lane == leader) {
                const uint32_t sh = (t & 1u) * 16u;
                base = (atomicAdd(&mine[t >> 1], (uint32_t)__popc(peers) << sh) >> sh) & 0xffffu;
            }
            base = __shfl_sync(0xffffffffu, base, leader);
            if (active) {
                const uint64_t pos = (uint64_t)tile_start[t] + cb[t] + base + __popc(peers & lt);
                if (pos < (uint64_t)cap) vals_out[pos] = og;
            }
        }
    }
}

// Chunk length for n Gaussians: about two chunks per SM, a multiple of 256, in [2048, 32768].
int64_t bin_chunk(int64_t n) {
    static int sms = 0;   // SM count of the first device asked (148 if none answers)
    if (sms == 0) {
        int dev = 0, s = 148;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            s = 148;
        sms = s;
    }
    int64_t c = (n + 2 * sms - 1) / (2 * sms);
    c = (c + 255) / 256 * 256;
    if (c < 2048) c = 2048;
    if (c > 32768) c = 32768;
    return c;
}

void launch_tile_bin(const Layout& L, char* ws, cudaStream_t stream, StageMark mark) {
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.off_ctrl);
    const uint32_t* dvals = reinterpret_cast<const uint32_t*>(ws + L.off_dvals[0]);
    const uint4* rect = reinterpret_cast<const uint4*>(ws + L.off_rect);
    const uint32_t* touched = reinterpret_cast<const uint32_t*>(ws + L.off_touched);
    uint32_t* counts = reinterpret_cast<uint32_t*>(ws + L.off_counts);
    uint32_t* chunk_base = reinterpret_cast<uint32_t*>(ws + L.off_chunk_base);
    uint32_t* totals = reinterpret_cast<uint32_t*>(ws + L.off_totals);
    uint32_t* tile_start = reinterpret_cast<uint32_t*>(ws + L.off_tile_start);
    const int nt = (int)L.ntiles;
    const int grid = (int)L.bin_chunks;
    static std::atomic<uint64_t> attr_dev{0};   // devices whose attributes are set
    const int emit_nw = (nt <= kBinMaxTiles8) ? 8 : 4;
    const size_t emit_smem = (size_t)emit_nw * ((nt + 1) / 2) * sizeof(uint32_t);
    const size_t count_smem = (size_t)nt * sizeof(uint32_t);
    if (once_per_device(attr_dev)) {
        cudaFuncSetAttribute(bin_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        cudaFuncSetAttribute(bin_emit_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        cudaFuncSetAttribute(bin_emit_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    }
    bin_count_kernel<<<grid, 256, count_smem, stream>>>(dvals, rect, &ctrl->num_visible, L.bin_chunk, nt, L.tiles_x,
                                                        counts);
    bin_scan_tiles_kernel<<<(nt + 31) / 32, 256, 0, stream>>>(counts, &ctrl->num_visible, L.bin_chunk, nt, chunk_base,
                                                              totals);
    launch_scan_sums(totals, tile_start, nt, &ctrl->num_keys, &ctrl->error, L.cap, stream);
    bin_ranges_kernel<<<(nt + 255) / 256, 256, 0, stream>>>(tile_start, totals, nt, ctrl,
                                                           reinterpret_cast<uint2*>(ws + L.off_ranges));
    if (mark) mark(4, stream);
    uint32_t* vals = reinterpret_cast<uint32_t*>(ws + L.off_vals[0]);
    if (emit_nw == 8)
        bin_emit_kernel<8><<<grid, 256, emit_smem, stream>>>(dvals, touched, rect, &ctrl->num_visible, L.bin_chunk, nt,
                                                             L.tiles_x, chunk_base, tile_start, ctrl, L.cap, vals);
    else
        bin_emit_kernel<4><<<grid, 128, emit_smem, stream>>>(dvals, touched, rect, &ctrl->num_visible, L.bin_chunk, nt,
                                                             L.tiles_x, chunk_base, tile_start, ctrl, L.cap, vals);
}

}  // namespace vis
