// K2 -- tile-key duplication, and K4 -- per-tile ranges.
//
// Algorithm 1 appends every surviving splat with an atomic counter, which makes
// the order (and so the tie order of the sort) run-dependent. Here the offsets are
// an exclusive prefix sum of the tiles-touched counts in Gaussian-index order, so
// the key list -- and the sorted result -- is deterministic:
//   1. scan_block_sums: one CTA scans the per-block sums written by the preprocess
//      and stores the total key count M in the status block (capacity checked);
//   2. duplicate_kernel: each block rescans its 256 counts (warp shuffles), then
//      every warp emits its Gaussians' keys cooperatively, lane j writing key j of
//      the warp's contiguous output run, so stores are coalesced whatever the
//      per-Gaussian counts. key = (tile id << 32) | float bits of the view depth,
//      val = Gaussian index; tiles in the footprint's row-major order (footprint.cuh).
//   3. ranges_kernel: [start, end) of every tile in the sorted keys.
#include "vis_internal.cuh"
#include "footprint.cuh"

namespace vis {

// Exclusive scan of per-block sums; the total goes to *total, and if `error` is given
// a total above `cap` sets kErrCapacity there. One CTA of 1024 threads works through the
// sums in chunks of kScanChunk: a coalesced load of the chunk into shared memory, a
// sequential sum of each thread's contiguous run of it, a scan of the 1024 run totals,
// the run's offsets written back in place, and a coalesced store; a carry links chunks.
// kScanChunk (8192 sums, 32 KB of static shared memory) is declared in vis_internal.cuh.

__global__ void __launch_bounds__(1024)
scan_block_sums(const uint32_t* __restrict__ bsum, uint32_t* __restrict__ boff, int64_t nblocks,
                uint32_t* total_out, uint32_t* error, int64_t cap) {
    pdl_entry();
    __shared__ uint32_t s[kScanChunk];
    __shared__ unsigned long long warp_tot[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int per = kScanChunk / 1024;
    unsigned long long carry = 0;
    for (int64_t c0 = 0; c0 < nblocks; c0 += kScanChunk) {
        const int n = (int)min((int64_t)kScanChunk, nblocks - c0);
        for (int i = threadIdx.x; i < kScanChunk; i += 1024) s[i] = i < n ? bsum[c0 + i] : 0u;
        __syncthreads();
        const int r0 = threadIdx.x * per;
        unsigned long long run = 0;
#pragma unroll
        for (int i = 0; i < per; ++i) run += s[r0 + i];
        unsigned long long incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        unsigned long long excl = carry + incl - run, all = 0;
        for (int w = 0; w < 32; ++w) {
            const unsigned long long x = warp_tot[w];
            if (w < warp) excl += x;
            all += x;
        }
#pragma unroll
        for (int i = 0; i < per; ++i) {
            const uint32_t v = s[r0 + i];
            s[r0 + i] = (uint32_t)min(excl, (unsigned long long)0xffffffffu);
            excl += v;
        }
        carry += all;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += 1024) boff[c0 + i] = s[i];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *total_out = (uint32_t)min(carry, (unsigned long long)0xffffffffu);
        if (error && carry > (unsigned long long)cap) atomicOr(error, kErrCapacity);
    }
}

// Beyond one chunk the scan runs on one CTA per chunk: scan_chunk_totals sums each chunk
// into chunk_tot[c]; scan_chunks adds, per CTA, the totals of the chunks before its own to
// the same in-chunk scan as scan_block_sums, and the last chunk's CTA writes the total.
__global__ void __launch_bounds__(1024)
scan_chunk_totals(const uint32_t* __restrict__ bsum, int64_t nblocks, unsigned long long* __restrict__ chunk_tot) {
    pdl_entry();
    __shared__ unsigned long long warp_tot[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t c0 = (int64_t)blockIdx.x * kScanChunk;
    const int n = (int)min((int64_t)kScanChunk, nblocks - c0);
    unsigned long long v = 0;
    for (int i = threadIdx.x; i < n; i += 1024) v += bsum[c0 + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) warp_tot[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < 32; ++w) t += warp_tot[w];
        chunk_tot[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024)
scan_chunks(const uint32_t* __restrict__ bsum, uint32_t* __restrict__ boff, int64_t nblocks,
            const unsigned long long* __restrict__ chunk_tot, uint32_t* total_out, uint32_t* error, int64_t cap) {
    pdl_entry();
    __shared__ uint32_t s[kScanChunk];
    __shared__ unsigned long long warp_tot[32];
    __shared__ unsigned long long s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int per = kScanChunk / 1024;
    const int64_t c0 = (int64_t)blockIdx.x * kScanChunk;
    const int n = (int)min((int64_t)kScanChunk, nblocks - c0);
    // the totals of the chunks before this one
    unsigned long long pre = 0;
    for (int c = threadIdx.x; c < (int)blockIdx.x; c += 1024) pre += chunk_tot[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pre += __shfl_xor_sync(0xffffffffu, pre, o);
    if (lane == 0) warp_tot[warp] = pre;
    for (int i = threadIdx.x; i < kScanChunk; i += 1024) s[i] = i < n ? bsum[c0 + i] : 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < 32; ++w) t += warp_tot[w];
        s_carry = t;
    }
    __syncthreads();
    const unsigned long long carry = s_carry;
    const int r0 = threadIdx.x * per;
    unsigned long long run = 0;
#pragma unroll
    for (int i = 0; i < per; ++i) run += s[r0 + i];
    unsigned long long incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    __syncthreads();
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    unsigned long long excl = carry + incl - run, all = 0;
    for (int w = 0; w < 32; ++w) {
        const unsigned long long x = warp_tot[w];
        if (w < warp) excl += x;
        all += x;
    }
#pragma unroll
    for (int i = 0; i < per; ++i) {
        const uint32_t v = s[r0 + i];
        s[r0 + i] = (uint32_t)min(excl, (unsigned long long)0xffffffffu);
        excl += v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += 1024) boff[c0 + i] = s[i];
    if (threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) {
        const unsigned long long tot = carry + all;
        *total_out = (uint32_t)min(tot, (unsigned long long)0xffffffffu);
        if (error && tot > (unsigned long long)cap) atomicOr(error, kErrCapacity);
    }
}

void launch_scan_sums(const uint32_t* bsum, uint32_t* boff, int64_t nblocks, uint32_t* total, uint32_t* error,
                      int64_t cap, unsigned long long* chunk_tot, cudaStream_t stream) {
    const int64_t chunks = (nblocks + kScanChunk - 1) / kScanChunk;
    if (chunks <= 1 || !chunk_tot) {
        launch_k(true, scan_block_sums, 1, 1024, 0, stream, bsum, boff, nblocks, total, error, cap);
        return;
    }
    launch_k(true, scan_chunk_totals, (int)chunks, 1024, 0, stream, bsum, nblocks, chunk_tot);
    launch_k(true, scan_chunks, (int)chunks, 1024, 0, stream, bsum, boff, nblocks,
             (const unsigned long long*)chunk_tot, total, error, cap);
}

__global__ void __launch_bounds__(kPrepThreads)
duplicate_kernel(const uint32_t* __restrict__ touched, const uint4* __restrict__ rect,
                 const float* __restrict__ depth, const uint32_t* __restrict__ boff, int64_t n,
                 int tiles_x, const Ctrl* __restrict__ ctrl, uint64_t* __restrict__ keys,
                 uint32_t* __restrict__ vals) {
    if (ctrl->error & kErrCapacity) return;   // nothing fits: leave the buffers alone
    __shared__ uint32_t s_start[kPrepThreads];   // exclusive offset within the warp's run
    __shared__ uint32_t warp_tot[kPrepThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kPrepThreads + threadIdx.x;
    const uint32_t cnt = (i < n) ? touched[i] : 0u;
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    s_start[threadIdx.x] = incl - cnt;
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    uint32_t warp_base = boff[blockIdx.x];
    for (int w = 0; w < warp; ++w) warp_base += warp_tot[w];
    const uint32_t run = warp_tot[warp];
    const int g0 = warp * 32;   // first Gaussian (block-local) of this warp
    for (uint32_t j = lane; j < run; j += 32) {
        // owner: the last g of the warp with s_start[g] <= j; a Gaussian with a zero
        // count shares its start with the next one, so the last such g owns key j
        int lo = 0, hi = 31;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_start[g0 + mid] <= j) lo = mid; else hi = mid - 1;
        }
        const int64_t gi = (int64_t)blockIdx.x * kPrepThreads + g0 + lo;
        const uint32_t k = j - s_start[g0 + lo];
        const uint64_t tile = fp_tile(fp_unpack(rect[gi]), k, (uint32_t)tiles_x);
        const uint32_t zb = __float_as_uint(depth[gi]);
        keys[warp_base + j] = (tile << 32) | zb;
        vals[warp_base + j] = (uint32_t)gi;
    }
}

void launch_scan_and_duplicate(const Layout& L, char* ws, int64_t n, cudaStream_t stream) {
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.off_ctrl);
    const uint32_t* bsum = reinterpret_cast<const uint32_t*>(ws + L.off_bsum);
    uint32_t* boff = reinterpret_cast<uint32_t*>(ws + L.off_boff);
    launch_scan_sums(bsum, boff, L.prep_blocks, &ctrl->num_keys, &ctrl->error, L.cap,
                     reinterpret_cast<unsigned long long*>(ws + L.off_scan_tot), stream);
    if (n <= 0) return;
    duplicate_kernel<<<(int)L.prep_blocks, kPrepThreads, 0, stream>>>(
        reinterpret_cast<const uint32_t*>(ws + L.off_touched), reinterpret_cast<const uint4*>(ws + L.off_rect),
        reinterpret_cast<const float*>(ws + L.off_depth), boff, n, L.tiles_x, ctrl,
        reinterpret_cast<uint64_t*>(ws + L.off_keys[0]), reinterpret_cast<uint32_t*>(ws + L.off_vals[0]));
}

__global__ void ranges_kernel(const uint64_t* __restrict__ keys, const Ctrl* __restrict__ ctrl,
                              int64_t cap, uint2* __restrict__ ranges) {
    if (ctrl->error) return;
    const int64_t m = min((int64_t)ctrl->num_keys, cap);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = (uint32_t)(keys[j] >> 32);
        if (j == 0 || (uint32_t)(keys[j - 1] >> 32) != t) ranges[t].x = (uint32_t)j;
        if (j == m - 1 || (uint32_t)(keys[j + 1] >> 32) != t) ranges[t].y = (uint32_t)(j + 1);
    }
}

void launch_ranges(const Layout& L, char* ws, cudaStream_t stream) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (L.cap + 255) / 256;
    const int64_t lim = (int64_t)sms * 8;
    const int blocks = (int)(want < 1 ? 1 : (want < lim ? want : lim));
    ranges_kernel<<<blocks, 256, 0, stream>>>(
        reinterpret_cast<const uint64_t*>(ws + L.off_keys[L.sorted_buffer]),
        reinterpret_cast<const Ctrl*>(ws + L.off_ctrl), L.cap, reinterpret_cast<uint2*>(ws + L.off_ranges));
}

}  // namespace vis
