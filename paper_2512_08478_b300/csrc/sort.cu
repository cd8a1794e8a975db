// K3 -- stable LSD radix sort of (key, value) pairs, onesweep style.
//
// Algorithm 1 sorts the splats on the GPU with a radix sort (section 3.4, "GPU
// sorting and rasterization"); here the keys are 64-bit (tile id << 32 | float bits
// of the view depth) with the Gaussian index as payload, so one stable sort yields
// the (tile, depth, index) order the compositor walks; the depth-first order sorts
// 32-bit depth keys, then 16- or 32-bit tile ids.
//
//  - sort_histogram: one read of all keys builds the digit histograms of every
//    pass at once (shared-memory counters, one global atomic per bin per CTA).
//  - sort_pass (one launch per digit of DBITS = 8, 10 or 11 bits): a CTA takes the next
//    partition of 256 x KPT keys from an atomic ticket (so partitions start in order and
//    the look-back below always makes progress), ranks its keys stably per warp with
//    ballots, publishes its per-digit counts, and resolves its global offsets by
//    decoupled look-back over the preceding partitions' published counts. The keys are
//    then reordered by digit in shared memory and written out in runs, so global stores
//    are coalesced within each digit run. Wider digits need fewer passes but publish and
//    read D = 2^DBITS look-back words per partition (4 D bytes against 4096 keys).
//  - Spin waits on a predecessor are bounded (spin_limit polls); on expiry the
//    CTA records kErrTimeout, publishes anyway so nobody waits on it, and writes
//    nothing out of range (every destination is checked against the key count).
#include <mutex>
#include <type_traits>

#include "onesweep.cuh"

namespace vis {

// Digit histograms of `passes` digits of DBITS bits (pass p: digit (key >> DBITS p)),
// hist[p * D + digit]; dynamic shared memory of passes * D words.
template <typename K, int DBITS>
__global__ void __launch_bounds__(1024)
sort_histogram(const K* __restrict__ keys, const uint32_t* __restrict__ num_keys, int64_t cap, int passes,
               uint32_t* __restrict__ hist, const uint32_t* __restrict__ error) {
    constexpr int D = 1 << DBITS;
    pdl_entry();
    extern __shared__ uint32_t sh[];
    for (int i = threadIdx.x; i < passes * D; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    if (*error) return;
    const int64_t m = min((int64_t)*num_keys, cap);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        const K k = keys[j];
        for (int p = 0; p < passes; ++p)
            atomicAdd(&sh[p * D + (uint32_t)((k >> (DBITS * p)) & (D - 1))], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * D; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

template <typename K, int KPT, int DBITS>
struct SortSmem {
    using Cfg = RadixCfg<DBITS>;
    K keys[kSortThreads * KPT];          // reordered by digit
    uint32_t vals[kSortThreads * KPT];   // reordered by digit
    uint32_t vin[kSortThreads * KPT];    // values in input order (asynchronous copies)
    typename Cfg::Counter whist[kSortThreads / 32][Cfg::D];
    uint32_t digit_off[Cfg::D];
    uint32_t local_start[Cfg::D];
    uint32_t scan_a[8], scan_b[8];
    uint32_t part;
    uint32_t bad;
};

// CTAs per SM the register budget is set for: three (80-85 registers, no spills) for 8- and
// 10-bit digits and for the 16-bit tile keys (with the persistent passes measured 1-3% faster
// on the tile keys than four CTAs at 64 registers, which spill), four for the short 32-bit
// partitions, two for the 11-bit digits, whose shared memory (~96 KB) admits no more.
template <typename K, int KPT, int DBITS>
struct SortOcc {
    static constexpr int value = DBITS == 11 ? 2 : (KPT <= 8 && sizeof(K) == 4) ? 4 : 3;
};
// Look-back window (predecessors read per round) by key type and digit width.
template <typename K, int DBITS>
struct SortWin {
    static constexpr int value = DBITS > 8 ? 4 : (sizeof(K) == 2 ? 8 : 16);
};

// Per partition (warp-striped: warp w owns keys [w*32*KPT, (w+1)*32*KPT)):
//   keys -> registers, values -> shared memory by asynchronous copies;
//   stable ranking inside each warp (rank_keys, warp counters from zero): the rank of
//   every key among its warp's keys of the same digit, and the warp's digit counts;
//   per-digit partition counts (each thread its DPT consecutive digits), published at
//   once for the successors; exclusive scans of the counts and of the pass's global digit
//   histogram; the look-back windows are issued; the keys and values are reordered by
//   digit in shared memory; the look-back is resolved -> global digit offsets; digit runs
//   are written out.
// All indexing inside the partition is 32-bit and relative to its base. keys_out may be
// null (last pass of a sort whose keys are not needed). nbits: significant bits of this
// pass's digit (DBITS, fewer for the top digit of a narrow key).
template <typename K, int KPT, int DBITS>
__global__ void __launch_bounds__(kSortThreads, SortOcc<K, KPT, DBITS>::value)
sort_pass(const K* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
          K* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
          const uint32_t* __restrict__ num_keys, int64_t cap, int shift, int nbits,
          const uint32_t* __restrict__ hist_pass, uint32_t* __restrict__ lookback,
          uint32_t* __restrict__ part_counter, uint32_t* __restrict__ error, uint32_t spin_limit) {
    using Cfg = RadixCfg<DBITS>;
    using Counter = typename Cfg::Counter;
    constexpr int D = Cfg::D, DPT = Cfg::DPT, WIN = SortWin<K, DBITS>::value;
    static_assert(WIN == lookback_group((int)sizeof(K), DBITS), "look-back groups are one window wide");
    pdl_entry();
    constexpr int PART = kSortThreads * KPT;
    // the pass's look-back region: a row of D words per partition of the capacity, then a row
    // per group of WIN partitions
    uint32_t* groups = lookback + (size_t)((cap + PART - 1) / PART) * D;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem<K, KPT, DBITS>& S = *reinterpret_cast<SortSmem<K, KPT, DBITS>*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (ld_relaxed(error) & kErrCapacity) return;
    const int64_t m = min((int64_t)*num_keys, cap);
    const int wofs = warp * (32 * KPT) + lane;
    K key[KPT];
    uint32_t vmask = 0;
    // Take the next partition (ticket) and start loading it: keys to registers, values to
    // shared memory by asynchronous copies; false if no partition is left. Requires whist and
    // vin free (a barrier since their last use).
    auto take_and_load = [&](uint32_t& part, int& n_in) -> bool {
        if (tid == 0) {
            S.part = atomicAdd(part_counter, 1u);
            S.bad = 0;
        }
        for (int i = tid; i < (kSortThreads / 32) * D; i += kSortThreads) (&S.whist[0][0])[i] = 0;
        __syncthreads();
        part = S.part;
        const int64_t base = (int64_t)part * PART;
        if (base >= m) return false;
        n_in = (m - base) < (int64_t)PART ? (int)(m - base) : PART;
        const K* kin = keys_in + base;
        const uint32_t* vin = vals_in + base;
        vmask = 0;
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
            const int idx = wofs + k * 32;
            if (idx < n_in) {
                key[k] = kin[idx];
                vmask |= 1u << k;
                cp_async4(&S.vin[idx], vin + idx);
            } else {
                key[k] = 0;
            }
        }
        cp_async_commit();
        return true;
    };
    // persistent: the grid holds about one wave of CTAs, each takes partitions (tickets in
    // order) until none is left; a CTA waits only on lower tickets, all taken by running CTAs.
    // The next partition's loads are issued before this one's look-back is resolved, so that
    // they are in flight during the wait and the write-out.
    // Publish a ranked partition's per-digit aggregate (the warp counts summed; the warp
    // counters hold the counts until the next barrier-separated step turns them into offsets).
    // A digit that no key of the pass has (zero in the global histogram, which every partition
    // reads) has no look-back chain: nobody publishes or reads its words.
    auto publish = [&](uint32_t p) {
#pragma unroll
        for (int j = 0; j < DPT; ++j) {
            const uint32_t d = (uint32_t)tid * DPT + j;
            if (hist_pass[d] == 0) continue;
            uint32_t c = 0;
#pragma unroll
            for (int w = 0; w < kSortThreads / 32; ++w) c += S.whist[w][d];
            st_relaxed(&lookback[(size_t)p * D + d], (p == 0 ? kFlagInc : kFlagAgg) | c);
            group_add<WIN, D>(groups, p, d, c);
        }
    };
    Counter* wh = S.whist[warp];
    uint32_t part;
    int n_in;
    if (!take_and_load(part, n_in)) return;
    // ---- stable ranking inside the warp; the warp counters end as the warp's digit counts ----
    uint32_t pos[KPT];
    rank_keys<KPT, DBITS, K, Counter>(key, shift, nbits, vmask, wh, pos);
    __syncthreads();
    publish(part);
    for (;;) {

    // ---- per-digit counts and warp offsets (the aggregate is published); scans; issue the look-back ----
    const uint32_t d0 = (uint32_t)tid * DPT;   // this thread's digits d0 .. d0 + DPT - 1
    uint32_t cnt[DPT], h[DPT];
    uint32_t ta = 0, tb = 0;
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
        const uint32_t d = d0 + j;
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) {
            const uint32_t x = S.whist[w][d];
            S.whist[w][d] = (Counter)c;   // exclusive offset of warp w within digit d
            c += x;
        }
        cnt[j] = c;
        h[j] = hist_pass[d];
        ta += c;
        tb += h[j];
    }
    uint32_t ia = ta, ib = tb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t xa = __shfl_up_sync(0xffffffffu, ia, o), xb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) { ia += xa; ib += xb; }
    }
    if (lane == 31) { S.scan_a[warp] = ia; S.scan_b[warp] = ib; }
    uint32_t lbw[DPT][WIN];
#pragma unroll
    for (int j = 0; j < DPT; ++j)
        if (h[j] != 0) lookback_issue<WIN, D>(lookback, part, d0 + j, lbw[j]);
    __syncthreads();
    uint32_t ls = ia - ta, gs = ib - tb;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w)
        if (w < warp) { ls += S.scan_a[w]; gs += S.scan_b[w]; }
    uint32_t lsd[DPT], gsd[DPT];
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
        lsd[j] = ls;
        gsd[j] = gs;
        S.local_start[d0 + j] = ls;
        ls += cnt[j];
        gs += h[j];
    }
    __syncthreads();

    // ---- reorder by digit: partition position = digit start + warp offset + rank ----
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
        const uint32_t dk = (uint32_t)(key[k] >> shift) & (D - 1);
        pos[k] += S.local_start[dk] + (uint32_t)wh[dk];
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k)
        if ((vmask >> k) & 1u) S.keys[pos[k]] = key[k];
    cp_async_wait_all();   // this thread's own values (same striped slots)
#pragma unroll
    for (int k = 0; k < KPT; ++k)
        if ((vmask >> k) & 1u) S.vals[pos[k]] = S.vin[wofs + k * 32];
    __syncthreads();   // whist and vin are free: start the next partition's loads
    uint32_t next_part;
    int next_n;
    const bool more = take_and_load(next_part, next_n);
    // rank the next partition now, while this one's look-back words arrive, and publish its
    // aggregate at once for the partitions behind it
    if (more) {
        rank_keys<KPT, DBITS, K, Counter>(key, shift, nbits, vmask, wh, pos);
        __syncthreads();
        publish(next_part);
    }

    // ---- resolve the look-back: global digit offsets ----
    bool timed_out = false;
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
        bool to = false;
        const uint32_t prefix =
            h[j] != 0 ? lookback_resolve<WIN, D>(lookback, groups, part, d0 + j, cnt[j], lbw[j], spin_limit, &to) : 0u;
        timed_out = timed_out || to;
        S.digit_off[d0 + j] = gsd[j] + prefix - lsd[j];
    }
    if (timed_out) {
        atomicOr(error, kErrTimeout);
        S.bad = 1;
    }
    __syncthreads();
    if (S.bad) {   // give up: wait for the next partition's copies to this CTA's shared memory
        cp_async_wait_all();
        return;
    }

    // ---- write out in digit runs (destinations are modular: digit_off may wrap) ----
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
        const int i = tid + k * kSortThreads;
        if (i < n_in) {
            const K kk = S.keys[i];
            const uint32_t dest = S.digit_off[(uint32_t)(kk >> shift) & (D - 1)] + (uint32_t)i;
            if (dest < (uint32_t)m) {
                if (keys_out) keys_out[dest] = kk;
                vals_out[dest] = S.vals[i];
            }
        }
    }
    if (!more) return;
    __syncthreads();   // the next partition reuses keys, vals and digit_off; its warp counts are in
    part = next_part;
    n_in = next_n;
    }
}

__global__ void set_u32_kernel(uint32_t* ptr, uint32_t value) { *ptr = value; }

void launch_set_u32(uint32_t* ptr, uint32_t value, cudaStream_t stream) {
    set_u32_kernel<<<1, 1, 0, stream>>>(ptr, value);
}

static int sm_count() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// CTAs of a persistent pass: one wave at `occ` CTAs per SM, at most one per partition.
static int pass_grid(int64_t parts, int occ) {
    const int64_t wave = (int64_t)sm_count() * occ;
    return (int)(parts < wave ? parts : wave);
}

template <typename K, int KPT, int DBITS>
static void sort_generic_impl(const K* keys_in, const uint32_t* vals_in, K* keys_a, uint32_t* vals_a, K* keys_b,
                              uint32_t* vals_b, int64_t cap, const uint32_t* num_keys_dev, int passes, uint32_t* hist,
                              uint32_t* lookback, uint32_t* part_counters, uint32_t* error, cudaStream_t stream,
                              StageMark mark, int mark_index, int last_bits, uint32_t spin_limit,
                              bool last_keys) {
    constexpr int D = 1 << DBITS;
    static std::atomic<uint64_t> attr_dev{0};   // devices whose attributes are set
    static std::mutex attr_mu;
    const size_t smem = sizeof(SortSmem<K, KPT, DBITS>);
    const size_t hsmem = sizeof(uint32_t) * kMaxPasses * D;
    set_up_per_device(attr_dev, attr_mu, [&] {
        return cudaFuncSetAttribute(sort_pass<K, KPT, DBITS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem) == cudaSuccess &&
               cudaFuncSetAttribute(sort_histogram<K, DBITS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)hsmem) == cudaSuccess;
    });
    const int64_t parts = (cap + (int64_t)kSortThreads * KPT - 1) / ((int64_t)kSortThreads * KPT);
    const int grid = pass_grid(parts, SortOcc<K, KPT, DBITS>::value);
    // two CTAs of 1024 threads per SM: each flushes its shared histograms with one global
    // atomic per non-zero bin, so fewer, larger CTAs halve the atomics on the same words
    // (against four CTAs of 256: 1M depth sort 0.087 -> 0.083 ms, 6M 0.251 -> 0.238 ms)
    const int64_t hb = (cap + 1023) / 1024, hlim = (int64_t)sm_count() * 2;
    const int hist_blocks = (int)(hb < hlim ? hb : hlim);
    launch_k(true, sort_histogram<K, DBITS>, hist_blocks, 1024, sizeof(uint32_t) * passes * D, stream, keys_in,
             (const uint32_t*)num_keys_dev, cap, passes, hist, (const uint32_t*)error);
    if (mark) mark(mark_index, stream);
    const K* src_k = keys_in;
    const uint32_t* src_v = vals_in;
    for (int p = 0; p < passes; ++p) {
        const bool to_a = ((passes - 1 - p) % 2) == 0;
        K* dk = (p == passes - 1 && !last_keys) ? nullptr : (to_a ? keys_a : keys_b);
        uint32_t* dv = to_a ? vals_a : vals_b;
        const int nbits = (p == passes - 1 && last_bits > 0 && last_bits < DBITS) ? last_bits : DBITS;
        launch_k(true, sort_pass<K, KPT, DBITS>, grid, kSortThreads, smem, stream, src_k, src_v, dk, dv,
                 (const uint32_t*)num_keys_dev, cap, DBITS * p, nbits, (const uint32_t*)(hist + (size_t)p * D),
                 lookback + (size_t)p * lookback_rows(parts, SortWin<K, DBITS>::value) * D, &part_counters[p], error,
                 spin_limit);
        src_k = dk;
        src_v = dv;
    }
}

// kpt: keys per thread of the passes (0: SortKPT<K>; 8 is also built for 32-bit keys of
// 8-bit digits); digit_bits 8, or 10 / 11 for 32-bit keys
template <typename K>
void launch_sort_generic(const K* keys_in, const uint32_t* vals_in, K* keys_a, uint32_t* vals_a, K* keys_b,
                         uint32_t* vals_b, int64_t cap, const uint32_t* num_keys_dev, int passes, uint32_t* hist,
                         uint32_t* lookback, uint32_t* part_counters, uint32_t* error, cudaStream_t stream,
                         StageMark mark, int mark_index, int last_bits, int kpt, uint32_t spin_limit,
                         int digit_bits, bool last_keys) {
    if (cap <= 0 || passes <= 0) return;
    constexpr bool k32 = std::is_same<K, uint32_t>::value;
#define VIS_SORT_IMPL(KPT_, DB_)                                                                                   \
    sort_generic_impl<K, KPT_, DB_>(keys_in, vals_in, keys_a, vals_a, keys_b, vals_b, cap, num_keys_dev, passes, \
                                    hist, lookback, part_counters, error, stream, mark, mark_index, last_bits,     \
                                    spin_limit, last_keys)
    if constexpr (k32) {
        if (digit_bits == 11) VIS_SORT_IMPL(16, 11);
        else if (digit_bits == 10) VIS_SORT_IMPL(16, 10);
        else if (kpt == 8) VIS_SORT_IMPL(8, 8);
        else VIS_SORT_IMPL(16, 8);
    } else {
        VIS_SORT_IMPL(SortKPT<K>::value, 8);
    }
#undef VIS_SORT_IMPL
}

// One pass of sort_pass over m <= cap keys (read from *num_keys_dev) with digit
// (key >> shift) & 255 and the digit histogram hist_pass; keys_out may be null.
template <typename K>
void launch_sort_pass(const K* keys_in, const uint32_t* vals_in, K* keys_out, uint32_t* vals_out, int64_t cap,
                      const uint32_t* num_keys_dev, int shift, int nbits, const uint32_t* hist_pass,
                      uint32_t* lookback, uint32_t* part_counter, uint32_t* error, cudaStream_t stream,
                      uint32_t spin_limit) {
    if (cap <= 0) return;
    static std::atomic<uint64_t> attr_dev{0};   // devices whose attributes are set
    static std::mutex attr_mu;
    constexpr int KPT = SortKPT<K>::value;
    const size_t smem = sizeof(SortSmem<K, KPT, 8>);
    set_up_per_device(attr_dev, attr_mu, [&] {
        return cudaFuncSetAttribute(sort_pass<K, KPT, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
               cudaSuccess;
    });
    launch_k(true, sort_pass<K, KPT, 8>, pass_grid(sort_parts<K>(cap), SortOcc<K, KPT, 8>::value), kSortThreads,
             smem, stream, keys_in, vals_in,
             keys_out, vals_out, (const uint32_t*)num_keys_dev, cap, shift, nbits, (const uint32_t*)hist_pass,
             lookback, part_counter, error, spin_limit);
}

template void launch_sort_pass<uint16_t>(const uint16_t*, const uint32_t*, uint16_t*, uint32_t*, int64_t,
                                         const uint32_t*, int, int, const uint32_t*, uint32_t*, uint32_t*,
                                         uint32_t*, cudaStream_t, uint32_t);

template void launch_sort_generic<uint64_t>(const uint64_t*, const uint32_t*, uint64_t*, uint32_t*, uint64_t*,
                                            uint32_t*, int64_t, const uint32_t*, int, uint32_t*, uint32_t*,
                                            uint32_t*, uint32_t*, cudaStream_t, StageMark, int, int, int, uint32_t,
                                            int, bool);
template void launch_sort_generic<uint32_t>(const uint32_t*, const uint32_t*, uint32_t*, uint32_t*, uint32_t*,
                                            uint32_t*, int64_t, const uint32_t*, int, uint32_t*, uint32_t*,
                                            uint32_t*, uint32_t*, cudaStream_t, StageMark, int, int, int, uint32_t,
                                            int, bool);

void launch_sort(const Layout& L, char* ws, cudaStream_t stream, StageMark mark, int mark_index) {
    uint64_t* k0 = reinterpret_cast<uint64_t*>(ws + L.off_keys[0]);
    uint64_t* k1 = reinterpret_cast<uint64_t*>(ws + L.off_keys[1]);
    uint32_t* v0 = reinterpret_cast<uint32_t*>(ws + L.off_vals[0]);
    uint32_t* v1 = reinterpret_cast<uint32_t*>(ws + L.off_vals[1]);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.off_ctrl);
    // the result lands in buffer (passes & 1); see Layout::sorted_buffer
    uint64_t* ka = (L.passes & 1) ? k1 : k0;
    uint32_t* va = (L.passes & 1) ? v1 : v0;
    uint64_t* kb = (L.passes & 1) ? k0 : k1;
    uint32_t* vb = (L.passes & 1) ? v0 : v1;
    launch_sort_generic<uint64_t>(k0, v0, ka, va, kb, vb, L.cap, &ctrl->num_keys, L.passes,
                                  reinterpret_cast<uint32_t*>(ws + L.off_hist),
                                  reinterpret_cast<uint32_t*>(ws + L.off_lookback), ctrl->part_counter,
                                  &ctrl->error, stream, mark, mark_index, L.key_bits - kRadixBits * (L.passes - 1), 0,
                                  L.spin_limit, kRadixBits);
}

}  // namespace vis
