// Building blocks of one onesweep-style LSD radix pass: 256 threads, a digit of DBITS = 8,
// 10 or 11 bits, so that in the scan and look-back phases each thread owns 1, 4 or 8
// consecutive digits.
//
// Per partition: rank every key stably inside its warp (which also yields the warp's
// digit counts), publish the partition's per-digit aggregate, issue the decoupled
// look-back over the preceding partitions, reorder the partition by digit in shared
// memory while the look-back words are in flight, then resolve the global digit offsets
// and write the digit runs.
#pragma once
#include <type_traits>

#include "vis_internal.cuh"

namespace vis {

constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1;
// Group words (one row of D per group of WIN consecutive partitions, after the partitions'
// rows): every partition of the group adds its digit count plus one arrival, in one atomic,
// so a word whose arrivals reach WIN holds the group's complete count (at most WIN x 4096).
constexpr int kGroupArriveShift = 26;
constexpr uint32_t kGroupArrive = 1u << kGroupArriveShift;
constexpr uint32_t kGroupCountMask = kGroupArrive - 1;
constexpr int kGroupRound = 4;   // group words read per round of the look-back's group walk

static_assert(kSortThreads == 256, "the scan phase assumes 8 warps");

// Per digit width: D digits, DPT of them per thread, and the type of the per-warp digit
// counters (a warp counts at most 32 x 16 = 512 keys of one digit, so 16 bits suffice and
// halve the shared memory of the wide digits).
template <int DBITS>
struct RadixCfg {
    static constexpr int D = 1 << DBITS;
    static constexpr int DPT = D > kSortThreads ? D / kSortThreads : 1;
    using Counter = typename std::conditional<(D > kSortThreads), uint16_t, uint32_t>::type;
    static_assert(D >= kSortThreads, "at least one digit per thread");
};

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Stable rank of KPT warp-striped keys (digit (key[k] >> shift) & (D - 1), with nbits
// significant bits; key k valid iff bit k of valid_mask) among the warp's keys of the same
// digit. Per round, the lanes holding the same digit ("peers") are found with one ballot per
// digit bit; the group's leader (lowest lane) takes the group's slots from the warp's
// private running counter wh[digit] with a plain load and store -- groups of one round
// have distinct digits, and the rounds are ordered by __syncwarp. Returns wh[digit] on
// entry + (rank of the key among the warp's keys of its digit in this round); wh[digit]
// grows by the warp's count of the digit.
template <int KPT, int DBITS, typename K, typename Counter>
__device__ __forceinline__ void rank_keys(const K (&key)[KPT], int shift, int nbits, uint32_t valid_mask,
                                          Counter* wh, uint32_t (&pos)[KPT]) {
    constexpr uint32_t kMask = (1u << DBITS) - 1;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
        const bool valid = (valid_mask >> k) & 1u;
        const uint32_t dk = (uint32_t)(key[k] >> shift) & kMask;
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
            wh[dk] = (Counter)(old + (uint32_t)__popc(peers));
        }
        __syncwarp();
        old = __shfl_sync(0xffffffffu, old, leader);
        pos[k] = old + __popc(peers & lt);
    }
}

// 4-byte asynchronous copy global -> shared (completes at cp_async_wait_all).
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Decoupled look-back over the words lookback[q * D + d] of the partitions q preceding
// `part`, in two levels. The partitions form groups of WIN (group g: partitions g WIN ..
// g WIN + WIN - 1); besides its own word every partition adds its count to its group's word
// groups[g * D + d] (group_add). lookback_issue reads this partition's predecessors within
// its own group (at most WIN - 1) while the reordering runs; lookback_resolve consumes them in
// order up to the first inclusive prefix, then walks whole groups back, kGroupRound groups per
// round with their loads in flight together: a group counts by its last partition's inclusive
// prefix if published (and the walk stops there), else by its complete group count. A word
// not yet published is polled at most `limit` times. The walk covers WIN partitions per
// group word, so a partition far from the last published inclusive prefix (all partitions
// of a single wave start together) waits a few rounds, not one per WIN partitions. It then
// publishes this partition's inclusive prefix and returns the count of d over all preceding
// partitions (*timed_out set if a poll gave up; the prefix is then wrong, but still
// published, so that no successor waits on this partition).
template <int WIN, int D>
__device__ __forceinline__ void lookback_issue(const uint32_t* lookback, uint32_t part, uint32_t d,
                                               uint32_t (&v)[WIN]) {
    const int64_t q0 = (int64_t)part - 1, gstart = (int64_t)(part / WIN) * WIN;
#pragma unroll
    for (int i = 0; i < WIN; ++i)
        v[i] = (q0 - i >= gstart) ? ld_relaxed(&lookback[(size_t)(q0 - i) * D + d]) : kFlagInc;
}

template <int WIN, int D>
__device__ __forceinline__ void group_add(uint32_t* groups, uint32_t part, uint32_t d, uint32_t cnt) {
    atomicAdd(&groups[(size_t)(part / WIN) * D + d], cnt + kGroupArrive);
}

__device__ __forceinline__ bool lookback_wait(const uint32_t* word, uint32_t* w, uint32_t limit) {
    uint32_t spins = 0;
    while ((*w & ~kCountMask) == 0) {
        if (++spins > limit) return false;
        if (spins > 8) __nanosleep(32);
        *w = ld_relaxed(word);
    }
    return true;
}

// Wait until group g's last partition has published its inclusive prefix (*lw) or all WIN
// partitions of the group have added their counts (*gw); false if `limit` polls pass.
template <int WIN>
__device__ __forceinline__ bool group_wait(const uint32_t* last_word, const uint32_t* group_word, uint32_t* lw,
                                           uint32_t* gw, uint32_t limit) {
    uint32_t spins = 0;
    while ((*lw & ~kCountMask) != kFlagInc && (*gw >> kGroupArriveShift) != (uint32_t)WIN) {
        if (++spins > limit) return false;
        if (spins > 8) __nanosleep(32);
        *lw = ld_relaxed(last_word);
        *gw = ld_relaxed(group_word);
    }
    return true;
}

template <int WIN, int D>
__device__ __forceinline__ uint32_t lookback_resolve(uint32_t* lookback, const uint32_t* groups, uint32_t part,
                                                     uint32_t d, uint32_t cnt, const uint32_t (&v)[WIN],
                                                     uint32_t limit, bool* timed_out) {
    *timed_out = false;
    if (part == 0) return 0;
    uint32_t prefix = 0;
    bool found = false, to = false;
    const int64_t q0 = (int64_t)part - 1, gstart = (int64_t)(part / WIN) * WIN;
    // this partition's predecessors in its own group
#pragma unroll
    for (int i = 0; i < WIN; ++i) {
        if (found || to || q0 - i < gstart) break;
        uint32_t w = v[i];
        if (!lookback_wait(&lookback[(size_t)(q0 - i) * D + d], &w, limit)) { to = true; break; }
        prefix += w & kCountMask;
        if ((w & ~kCountMask) == kFlagInc) found = true;
    }
    // the whole groups before it, kGroupRound groups per round
    for (int64_t gb = (int64_t)(part / WIN) - 1; !found && !to && gb >= 0; gb -= kGroupRound) {
        uint32_t lw[kGroupRound], gw[kGroupRound];
#pragma unroll
        for (int i = 0; i < kGroupRound; ++i) {
            const bool ok = gb - i >= 0;
            lw[i] = ok ? ld_relaxed(&lookback[(size_t)((gb - i) * WIN + WIN - 1) * D + d]) : 0u;
            gw[i] = ok ? ld_relaxed(&groups[(size_t)(gb - i) * D + d]) : 0u;
        }
#pragma unroll
        for (int i = 0; i < kGroupRound; ++i) {
            if (found || to || gb - i < 0) break;
            const int64_t g = gb - i;
            if (!group_wait<WIN>(&lookback[(size_t)(g * WIN + WIN - 1) * D + d], &groups[(size_t)g * D + d], &lw[i],
                                 &gw[i], limit)) {
                to = true;
                break;
            }
            if ((lw[i] & ~kCountMask) == kFlagInc) {
                prefix += lw[i] & kCountMask;
                found = true;
            } else {
                prefix += gw[i] & kGroupCountMask;
            }
        }
    }
    st_relaxed(&lookback[(size_t)part * D + d], kFlagInc | ((prefix + cnt) & kCountMask));
    *timed_out = to;
    return prefix;
}

}  // namespace vis
