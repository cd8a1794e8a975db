// vis_sort_pairs_noalloc -- the radix sort of vis_sort_pairs for callers that cannot
// allocate device memory.
//
// Some callers are not allowed to call cudaMalloc at the point where they sort: a
// real-time frame loop with a fixed memory budget, a plug-in running inside a host
// application that owns every device allocation, or code that must not risk the
// implicit device synchronisation an allocation can cause. They cannot provide the
// workspace vis_sort_pairs asks for, so this entry point takes its scratch (status
// block, digit histograms, look-back words and one ping-pong key/value buffer) from
// a fixed array in device memory that is part of the library image. The caller
// still passes the input and output arrays.
//
// The array is file-scope and static, so every GPU that loads the library holds
// VIS_SORT_NOALLOC_SCRATCH_BYTES of it until the process exits, and every call
// shares it. In host code the array's name is only a host-side stand-in, never a
// device address: the first call on each device (with that device current) looks
// the real address up with cudaGetSymbolAddress and caches it per device (so a device
// reset after that first call is not supported: the module may be reloaded elsewhere).
// A device-side error of the sort (a look-back wait that ran out) lands in the status
// word at the start of the array; vis_sort_noalloc_check() reads it.
#include <cstdio>
#include <mutex>

#include "vis_internal.cuh"

namespace {

constexpr int64_t kMaxKeys = VIS_SORT_NOALLOC_MAX_KEYS;
constexpr int64_t kMaxParts = vis::sort_parts<uint64_t>(kMaxKeys);
constexpr size_t kOffCtrl = 0;
constexpr size_t kOffHist = 256;
constexpr size_t kOffLookback = kOffHist + sizeof(uint32_t) * vis::kMaxPasses * vis::kRadix;
constexpr int64_t kMaxRows = kMaxParts + (kMaxParts + vis::lookback_group(8, 8) - 1) / vis::lookback_group(8, 8);
constexpr size_t kLookbackBytes = sizeof(uint32_t) * vis::kMaxPasses * kMaxRows * vis::kRadix;
constexpr size_t kOffKeys = (kOffLookback + kLookbackBytes + 255) / 256 * 256;   // cleared below this
constexpr size_t kOffVals = kOffKeys + sizeof(uint64_t) * kMaxKeys;
constexpr size_t kScratchBytes = kOffVals + sizeof(uint32_t) * kMaxKeys;
static_assert(kScratchBytes == VIS_SORT_NOALLOC_SCRATCH_BYTES, "header states the scratch size");
static_assert(sizeof(vis::Ctrl) <= kOffHist, "status block fits");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

namespace {

vis_status fail_na(vis_status s, const char* msg) {
    vis::set_last_error(msg);
    return s;
}

// Device address of g_sort_scratch on the current device (looked up once per device).
vis_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_na(VIS_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail_na(VIS_ERR_UNSUPPORTED, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess || p == nullptr)
            return fail_na(VIS_ERR_CUDA, "cudaGetSymbolAddress of the static sort scratch failed");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return VIS_OK;
}

bool aligned16_na(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" vis_status vis_sort_pairs_noalloc(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                                             uint32_t* vals_out, int64_t m, int key_bits, void* stream_) {
    if (m < 0 || m > kMaxKeys) {
        char buf[160];
        snprintf(buf, sizeof(buf), "m = %lld exceeds the %lld-key limit of the static sort scratch "
                 "(use vis_sort_pairs with a caller workspace)", (long long)m, (long long)kMaxKeys);
        return fail_na(VIS_ERR_INVALID_ARG, buf);
    }
    if (key_bits < 1 || key_bits > 64) return fail_na(VIS_ERR_INVALID_ARG, "key_bits must be in [1, 64]");
    if (m == 0) { vis::set_last_error(""); return VIS_OK; }
    const void* ptrs[4] = {keys_in, vals_in, keys_out, vals_out};
    for (int k = 0; k < 4; ++k)
        if (!ptrs[k] || !aligned16_na(ptrs[k])) return fail_na(VIS_ERR_INVALID_ARG, "sort buffer null or misaligned");
    if ((const void*)keys_in == (const void*)keys_out || (const void*)vals_in == (const void*)vals_out)
        return fail_na(VIS_ERR_INVALID_ARG, "sort input and output must not alias");
    void* base = nullptr;
    vis_status st = scratch_address(&base);
    if (st) return st;
    char* w = static_cast<char*>(base);
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    // the array keeps the previous call's contents: clear the status block, the histograms and
    // the look-back words that this sort's passes read (passes x partitions x digits)
    const int passes = (key_bits + vis::kRadixBits - 1) / vis::kRadixBits;
    const size_t used = kOffLookback + sizeof(uint32_t) * (size_t)passes *
                                           (size_t)vis::lookback_rows(vis::sort_parts<uint64_t>(m),
                                                                      vis::lookback_group(8, 8)) *
                                           vis::kRadix;
    cudaError_t e = cudaMemsetAsync(w, 0, used, stream);
    if (e != cudaSuccess) return fail_na(VIS_ERR_CUDA, cudaGetErrorString(e));
    vis::Ctrl* ctrl = reinterpret_cast<vis::Ctrl*>(w + kOffCtrl);
    vis::launch_set_u32(&ctrl->num_keys, (uint32_t)m, stream);
    vis::launch_sort_generic<uint64_t>(keys_in, vals_in, keys_out, vals_out,
                                       reinterpret_cast<uint64_t*>(w + kOffKeys), reinterpret_cast<uint32_t*>(w + kOffVals),
                                       m, &ctrl->num_keys, passes, reinterpret_cast<uint32_t*>(w + kOffHist),
                                       reinterpret_cast<uint32_t*>(w + kOffLookback), ctrl->part_counter, &ctrl->error,
                                       stream, nullptr, 0, key_bits - vis::kRadixBits * (passes - 1));
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_na(VIS_ERR_CUDA, cudaGetErrorString(e));
    vis::set_last_error("");
    return VIS_OK;
}

extern "C" vis_status vis_sort_noalloc_check(void* stream_) {
    void* base = nullptr;
    vis_status st = scratch_address(&base);
    if (st) return st;
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream_));
    if (e != cudaSuccess) return fail_na(VIS_ERR_CUDA, cudaGetErrorString(e));
    uint32_t word[2] = {0, 0};   // num_keys, error (the head of the status block)
    e = cudaMemcpy(word, base, sizeof(word), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_na(VIS_ERR_CUDA, cudaGetErrorString(e));
    if (word[1] & vis::kErrTimeout) return fail_na(VIS_ERR_TIMEOUT, "a look-back wait of the sort timed out");
    vis::set_last_error("");
    return VIS_OK;
}
