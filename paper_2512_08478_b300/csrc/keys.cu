// K2 -- tile-key duplication, and K4 -- per-tile ranges.
//
// Algorithm 1 appends every surviving splat with an atomic counter, which makes
// the order (and so the tie order of the sort) run-dependent. Here the offsets are
// an exclusive prefix sum of the tiles-touched counts in Gaussian-index order, so
// the key list -- and the sorted result -- is deterministic:
//   1. scan_sums: a single-pass scan of the per-block sums written by the preprocess,
//      which stores the total key count M in the status block (capacity checked);
//   2. duplicate_kernel: each block rescans its 256 counts (warp shuffles), then
//      every warp emits its Gaussians' keys cooperatively, lane j writing key j of
//      the warp's contiguous output run, so stores are coalesced whatever the
//      per-Gaussian counts. key = (tile id << 32) | float bits of the view depth,
//      val = Gaussian index; tiles in the footprint's row-major order (footprint.cuh).
//   3. ranges_kernel: [start, end) of every tile in the sorted keys.
#include "vis_internal.cuh"
#include "footprint.cuh"

namespace vis {

// Exclusive scan of per-block sums in one pass. Each CTA takes the next chunk of kScanPart sums
// from a ticket, so chunks start in order and a CTA only ever waits on running ones. It scans the
// chunk (two sums per thread, warp scans, a scan of the 32 warp totals) and publishes the chunk's
// total. Its first warp then resolves the chunk's offset by decoupled look-back over the
// preceding chunks' words, 32 per round. A word holds a chunk's total or its inclusive prefix,
// flagged in its top two bits, and the walk stops at the nearest inclusive prefix. The chunk
// then writes its offsets. The chunk with the last sum writes the total; a total above `cap`
// (when cap > 0) sets kErrCapacity. A poll of an unpublished word gives up after spin_limit polls
// and sets kErrTimeout; the prefix is then wrong but still published, so no successor waits.
constexpr unsigned long long kScanFlagAgg = 1ull << 62, kScanFlagInc = 2ull << 62;
constexpr unsigned long long kScanValMask = (1ull << 62) - 1;

__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(1024)
scan_sums(const uint32_t* __restrict__ bsum, uint32_t* __restrict__ boff, int64_t nblocks, uint32_t* total_out,
          uint32_t* error, int64_t cap, unsigned long long* lb, uint32_t* ticket, uint32_t spin_limit) {
    static_assert(kScanPart == 2 * 1024, "two sums per thread");
    pdl_entry();
    __shared__ uint32_t s_part;
    __shared__ unsigned long long s_warp[32];
    __shared__ unsigned long long s_prefix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_part = atomicAdd(ticket, 1u);
    __syncthreads();
    const int64_t part = s_part;
    const int64_t i0 = part * kScanPart + 2 * tid;
    const uint32_t v0 = i0 < nblocks ? bsum[i0] : 0u;
    const uint32_t v1 = i0 + 1 < nblocks ? bsum[i0 + 1] : 0u;
    const unsigned long long run = (unsigned long long)v0 + v1;
    unsigned long long incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long wt = s_warp[lane];
        unsigned long long wi = wt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        s_warp[lane] = wi - wt;   // exclusive offset of warp `lane` in the chunk
        const unsigned long long agg = __shfl_sync(0xffffffffu, wi, 31);
        if (lane == 0)
            st_relaxed64(&lb[part], (part == 0 ? kScanFlagInc : kScanFlagAgg) | (agg < kScanValMask ? agg : kScanValMask));
        unsigned long long prefix = 0;
        bool to = false;
        for (int64_t q0 = part - 1; q0 >= 0; q0 -= 32) {
            const int64_t q = q0 - lane;
            unsigned long long w = kScanFlagInc;   // before the first chunk: an inclusive prefix of 0
            if (q >= 0) {
                w = ld_relaxed64(&lb[q]);
                uint32_t spins = 0;
                while ((w >> 62) == 0) {
                    if (++spins > spin_limit) {
                        to = true;
                        w = kScanFlagInc;
                        break;
                    }
                    if (spins > 8) __nanosleep(32);
                    w = ld_relaxed64(&lb[q]);
                }
            }
            const uint32_t inc = __ballot_sync(0xffffffffu, (w >> 62) == 2ull);
            const int stop = inc ? __ffs(inc) - 1 : 31;   // lanes up to the nearest inclusive prefix count
            unsigned long long c = lane <= stop ? (w & kScanValMask) : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            prefix += c;
            if (inc) break;
        }
        const bool any_to = __any_sync(0xffffffffu, to);
        if (lane == 0) {
            const unsigned long long tot = prefix + agg;
            if (part > 0) st_relaxed64(&lb[part], kScanFlagInc | (tot < kScanValMask ? tot : kScanValMask));
            s_prefix = prefix;
            if (any_to && error) atomicOr(error, kErrTimeout);
            if ((part + 1) * kScanPart >= nblocks) {   // the chunk with the last sum
                *total_out = (uint32_t)min(tot, (unsigned long long)0xffffffffu);
                if (cap > 0 && error && tot > (unsigned long long)cap) atomicOr(error, kErrCapacity);
            }
        }
    }
    __syncthreads();
    const unsigned long long excl = s_prefix + s_warp[warp] + incl - run;
    if (i0 < nblocks) boff[i0] = (uint32_t)min(excl, (unsigned long long)0xffffffffu);
    if (i0 + 1 < nblocks) boff[i0 + 1] = (uint32_t)min(excl + v0, (unsigned long long)0xffffffffu);
}

void launch_scan_sums(const uint32_t* bsum, uint32_t* boff, int64_t nblocks, uint32_t* total, uint32_t* error,
                      int64_t cap, unsigned long long* lb, uint32_t* ticket, uint32_t spin_limit,
                      cudaStream_t stream) {
    const int64_t parts = scan_parts(nblocks);
    launch_k(true, scan_sums, (int)(parts < 1 ? 1 : parts), 1024, 0, stream, bsum, boff, nblocks, total, error, cap,
             lb, ticket, spin_limit);
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
                     reinterpret_cast<unsigned long long*>(ws + L.off_scan_lb), &ctrl->scan_ticket[0], L.spin_limit,
                     stream);
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
