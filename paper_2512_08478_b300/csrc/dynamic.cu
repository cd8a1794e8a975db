// The per-frame update kernel of a dynamic scene (the formulas: dynamic.cuh). Elementwise and
// bandwidth-bound: 40 B read and 16 B written per Gaussian.
#include "dynamic.cuh"

namespace vis {

__global__ void __launch_bounds__(256)
dynamic_update_kernel(const float* __restrict__ means0, const float* __restrict__ velocity,
                      const float* __restrict__ logits0, const float* __restrict__ amp,
                      const float* __restrict__ freq, const float* __restrict__ phase, float t, int64_t n,
                      float* __restrict__ means_out, float* __restrict__ logits_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
#pragma unroll
        for (int k = 0; k < 3; ++k) means_out[3 * i + k] = dyn_mean(means0[3 * i + k], velocity[3 * i + k], t);
        logits_out[i] = dyn_logit(logits0[i], amp[i], freq[i], phase[i], t);
    }
}

void launch_dynamic_update(const float* means0, const float* velocity, const float* logits0, const float* amp,
                           const float* freq, const float* phase, float t, int64_t n, float* means_out,
                           float* logits_out, cudaStream_t stream) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256, lim = (int64_t)sms * 16;
    const int blocks = (int)(want < lim ? want : lim);
    dynamic_update_kernel<<<blocks, 256, 0, stream>>>(means0, velocity, logits0, amp, freq, phase, t, n, means_out,
                                                      logits_out);
}

}  // namespace vis
