// Building blocks of one onesweep-style LSD radix pass (8-bit digit, 256 threads, one
// digit per thread in the scan and look-back phases).
//
// Per partition: rank every key stably inside its warp (which also yields the warp's
// digit counts), publish the partition's per-digit aggregate, issue the decoupled
// look-back over the preceding partitions, reorder the partition by digit in shared
// memory while the look-back words are in flight, then resolve the global digit offsets
// and write the digit runs.
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

// Stable rank of KPT warp-striped keys (digit (key[k] >> shift) & 255, key k valid iff
// bit k of valid_mask) inside the partition. Per round, the lanes holding the same digit
// ("peers") are found with one ballot per digit bit (the digit's upper bits are zero when
// nbits < 8); the group's leader (lowest lane) takes the group's slots from the warp's
// private running counter wh[digit] with a plain load and store -- groups of one round
// have distinct digits, and the rounds are ordered by __syncwarp. Returns
// local_start[digit] + wh[digit] on entry + (rank of the key among the warp's keys of its
// digit); wh[digit] grows by the warp's count of the digit.
template <int KPT, typename K>
__device__ __forceinline__ void rank_keys(const K (&key)[KPT], int shift, int nbits, uint32_t valid_mask,
                                          uint32_t* wh, const uint32_t* local_start, uint32_t (&pos)[KPT]) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
        const bool valid = (valid_mask >> k) & 1u;
        const uint32_t dk = (uint32_t)(key[k] >> shift) & (kRadix - 1);
        uint32_t peers = __ballot_sync(0xffffffffu, valid);
        for (int b = 0; b < nbits; ++b) {
            const uint32_t bit = (dk >> b) & 1u;
            const uint32_t bal = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bal : ~bal;
        }
        if (!valid) peers = 1u << lane;
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (valid && lane == leader) {
            old = wh[dk];
            wh[dk] = old + (uint32_t)__popc(peers);
        }
        __syncwarp();
        old = __shfl_sync(0xffffffffu, old, leader);
        pos[k] = local_start[dk] + old + __popc(peers & lt);
    }
}

// 4-byte asynchronous copy global -> shared (completes at cp_async_wait_all).
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Decoupled look-back, split in two so that its loads overlap the ranking:
// lookback_issue reads the window of WIN predecessors of partition `part` for digit d;
// lookback_resolve consumes it in order up to the first inclusive prefix, polling a word
// not yet published at most `limit` times, continues one predecessor at a time past
// the window if needed, publishes this partition's inclusive prefix and returns the
// count of d over all preceding partitions (*timed_out set if a poll gave up).
template <int WIN>
__device__ __forceinline__ void lookback_issue(const uint32_t* lookback, uint32_t part, uint32_t d,
                                               uint32_t (&v)[WIN]) {
    const int64_t q0 = (int64_t)part - 1;
#pragma unroll
    for (int i = 0; i < WIN; ++i)
        v[i] = (q0 - i >= 0) ? ld_relaxed(&lookback[(size_t)(q0 - i) * kRadix + d]) : kFlagInc;
}

__device__ __forceinline__ bool lookback_wait(const uint32_t* lookback, int64_t q, uint32_t d, uint32_t* w,
                                              uint32_t limit) {
    uint32_t spins = 0;
    while ((*w & ~kCountMask) == 0) {
        if (++spins > limit) return false;
        if (spins > 8) __nanosleep(32);
        *w = ld_relaxed(&lookback[(size_t)q * kRadix + d]);
    }
    return true;
}

template <int WIN>
__device__ __forceinline__ uint32_t lookback_resolve(uint32_t* lookback, uint32_t part, uint32_t d, uint32_t cnt,
                                                     const uint32_t (&v)[WIN], uint32_t limit,
                                                     bool* timed_out) {
    *timed_out = false;
    if (part == 0) return 0;
    uint32_t prefix = 0;
    bool found = false, to = false;
    const int64_t q0 = (int64_t)part - 1;
#pragma unroll
    for (int i = 0; i < WIN; ++i) {
        if (found || to || q0 - i < 0) break;
        uint32_t w = v[i];
        if (!lookback_wait(lookback, q0 - i, d, &w, limit)) { to = true; break; }
        prefix += w & kCountMask;
        if ((w & ~kCountMask) == kFlagInc) found = true;
    }
    for (int64_t q = q0 - WIN; !found && !to && q >= 0; --q) {
        uint32_t w = ld_relaxed(&lookback[(size_t)q * kRadix + d]);
        if (!lookback_wait(lookback, q, d, &w, limit)) { to = true; break; }
        prefix += w & kCountMask;
        if ((w & ~kCountMask) == kFlagInc) found = true;
    }
    st_relaxed(&lookback[(size_t)part * kRadix + d], kFlagInc | ((prefix + cnt) & kCountMask));
    *timed_out = to;
    return prefix;
}

}  // namespace vis
