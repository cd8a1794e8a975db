// Building blocks of one onesweep-style LSD radix pass (8-bit digit, 256 threads, one
// digit per thread in the scan and look-back phases), shared by the generic pair sort
// and by the tile binning that generates its keys in shared memory.
//
// Per partition: per-warp digit counts ("early counts"), publish the partition's
// per-digit aggregate, resolve its global digit offsets by decoupled look-back over the
// preceding partitions, then rank every key stably inside its warp and reorder the
// partition by digit in shared memory so that the global writes go out in digit runs.
#pragma once
#include "vis_internal.cuh"

namespace vis {

constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1;
constexpr int kLookbackWindow = 16;   // predecessors read per look-back round

static_assert(kSortThreads == kRadix, "one digit per thread");

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// exclusive scan of one value per thread over a 256-thread block; returns total in *tot
__device__ __forceinline__ uint32_t block_exclusive_scan_256(uint32_t v, uint32_t* s_warp, uint32_t* tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t woff = 0, all = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const uint32_t x = s_warp[w];
        if (w < warp) woff += x;
        all += x;
    }
    __syncthreads();
    if (tot) *tot = all;
    return woff + incl - v;
}

// Turn the per-warp counts of digit d (whist[w][d]) into exclusive per-warp offsets and
// return the partition's count of d.
__device__ __forceinline__ uint32_t warp_offsets_of_digit(uint32_t (*whist)[kRadix], uint32_t d) {
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) {
        const uint32_t c = whist[w][d];
        whist[w][d] = cnt;
        cnt += c;
    }
    return cnt;
}

// Publish this partition's count of digit d (partition 0 publishes it as inclusive).
__device__ __forceinline__ void publish_aggregate(uint32_t* lookback, uint32_t part, uint32_t d, uint32_t cnt) {
    st_relaxed(&lookback[(size_t)part * kRadix + d], (part == 0 ? kFlagInc : kFlagAgg) | cnt);
}

// Decoupled look-back for digit d: the count of d over all preceding partitions. A
// window of kLookbackWindow predecessors is read at once, then consumed in order up to
// the first inclusive prefix; only a word not yet published is polled again, at most
// kSpinLimit times (then *timed_out is set and the prefix is incomplete). Publishes this
// partition's inclusive prefix before returning.
__device__ __forceinline__ uint32_t lookback_prefix(uint32_t* lookback, uint32_t part, uint32_t d, uint32_t cnt,
                                                    bool* timed_out) {
    uint32_t prefix = 0;
    *timed_out = false;
    if (part == 0) return 0;
    int64_t q = (int64_t)part - 1;
    bool found = false, to = false;
    while (!found && !to && q >= 0) {
        uint32_t v[kLookbackWindow];
#pragma unroll
        for (int i = 0; i < kLookbackWindow; ++i)
            v[i] = (q - i >= 0) ? ld_relaxed(&lookback[(size_t)(q - i) * kRadix + d]) : kFlagInc;
#pragma unroll
        for (int i = 0; i < kLookbackWindow; ++i) {
            if (found || to || q - i < 0) break;
            uint32_t w = v[i];
            uint32_t spins = 0;
            while ((w & ~kCountMask) == 0) {
                if (++spins > kSpinLimit) { to = true; break; }
                if (spins > 8) __nanosleep(32);
                w = ld_relaxed(&lookback[(size_t)(q - i) * kRadix + d]);
            }
            if (to) break;
            prefix += w & kCountMask;
            if ((w & ~kCountMask) == kFlagInc) found = true;
        }
        q -= kLookbackWindow;
    }
    st_relaxed(&lookback[(size_t)part * kRadix + d], kFlagInc | ((prefix + cnt) & kCountMask));
    *timed_out = to;
    return prefix;
}

// Stable rank of KPT warp-striped keys (digit (key[k] >> shift) & 255, key k valid iff
// bit k of valid_mask) inside the partition: one __match_any_sync per round; the
// group's leader takes the group's slots from the warp's running digit counter wh[]
// (holding the warp's exclusive offset per digit) with a shared atomic, which keeps the
// rounds in program order. Returns partition-local positions
// local_start[digit] + (rank of the key among the partition's keys of its digit).
template <int KPT, typename K>
__device__ __forceinline__ void rank_keys(const K (&key)[KPT], int shift, uint32_t valid_mask, uint32_t* wh,
                                          const uint32_t* local_start, uint32_t (&pos)[KPT]) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
        const bool valid = (valid_mask >> k) & 1u;
        const uint32_t dk = (uint32_t)(key[k] >> shift) & (kRadix - 1);
        const uint32_t peers = __match_any_sync(0xffffffffu, valid ? dk : (kRadix + lane));
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (valid && lane == leader) old = atomicAdd(&wh[dk], (uint32_t)__popc(peers));
        old = __shfl_sync(0xffffffffu, old, leader);
        pos[k] = local_start[dk] + old + __popc(peers & lt);
    }
}

}  // namespace vis
