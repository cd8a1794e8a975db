// K5 -- tile compositor (section 3.2 Eqs. 2-3, front to back).
//
// One CTA per TILE x TILE tile, one thread per pixel. The tile's range of the
// sorted (tile, depth, index) list is walked in chunks of TILE^2 splats: each
// thread gathers one splat record (3 x float4) into shared memory, then every
// thread composites the whole chunk for its pixel from shared memory (broadcast
// reads). A pixel is done when T (1 - alpha) would fall below t_stop (that splat
// excluded); the CTA leaves as soon as all its pixels are done.
// Outputs: planar rgb = C + T bg, alpha = 1 - T, and for the adjoint the final T
// and 1 + the sorted position of the last composited splat.
#include "splat_eval.cuh"

namespace vis {

template <int TILE>
__global__ void __launch_bounds__(TILE * TILE)
composite_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                 const float4* __restrict__ rec, int W, int H, int tiles_x, float bg0, float bg1,
                 float bg2, float alpha_min, float alpha_max, float t_stop, const Ctrl* __restrict__ ctrl,
                 float* __restrict__ out_rgb, float* __restrict__ out_alpha, float* __restrict__ t_final,
                 int32_t* __restrict__ last_out) {
    constexpr int NT = TILE * TILE;
    __shared__ float4 s_a[NT], s_b[NT], s_c[NT];
    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int px = tx * TILE + (threadIdx.x % TILE), py = ty * TILE + (threadIdx.x / TILE);
    const bool inside = px < W && py < H;
    const size_t pix = (size_t)py * W + px;
    const size_t HW = (size_t)H * W;
    if (ctrl->error) {   // keys were not produced: make the failure visible
        if (inside) {
            const float nan = __int_as_float(0x7fc00000);
            out_rgb[pix] = nan; out_rgb[HW + pix] = nan; out_rgb[2 * HW + pix] = nan;
            out_alpha[pix] = nan; t_final[pix] = nan; last_out[pix] = 0;
        }
        return;
    }
    const float pcx = (float)px + 0.5f, pcy = (float)py + 0.5f;
    const uint2 r = ranges[tile];
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    int32_t last = 0;
    bool done = !inside;
    for (uint32_t base = r.x; base < r.y; base += NT) {
        if (__syncthreads_count(done) == NT) break;
        const uint32_t j = base + threadIdx.x;
        if (j < r.y) {
            const uint32_t g = vals[j];
            s_a[threadIdx.x] = rec[3 * (size_t)g + 0];
            s_b[threadIdx.x] = rec[3 * (size_t)g + 1];
            s_c[threadIdx.x] = rec[3 * (size_t)g + 2];
        }
        __syncthreads();
        const int cnt = (int)umin((uint32_t)NT, r.y - base);
        if (!done) {
            for (int k = 0; k < cnt; ++k) {
                const PairEval e = eval_pair(pcx, pcy, s_a[k], s_b[k]);
                if (e.q > 9.f) continue;
                const float4 c = s_c[k];
                const float alpha = fminf(alpha_max, __fmul_rn(c.x, gauss_of_q(e.q)));
                if (alpha < alpha_min) continue;
                const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
                if (Tn < t_stop) { done = true; break; }
                const float w = __fmul_rn(alpha, T);
                C0 = __fmaf_rn(c.y, w, C0);
                C1 = __fmaf_rn(c.z, w, C1);
                C2 = __fmaf_rn(c.w, w, C2);
                T = Tn;
                last = (int32_t)(base + k + 1);
            }
        }
    }
    if (inside) {
        out_rgb[pix] = __fmaf_rn(T, bg0, C0);
        out_rgb[HW + pix] = __fmaf_rn(T, bg1, C1);
        out_rgb[2 * HW + pix] = __fmaf_rn(T, bg2, C2);
        out_alpha[pix] = 1.f - T;
        t_final[pix] = T;
        last_out[pix] = last;
    }
}

void launch_composite(const Layout& L, char* ws, float bg0, float bg1, float bg2, float alpha_min,
                      float alpha_max, float t_stop, float* out_rgb, float* out_alpha,
                      cudaStream_t stream) {
    const uint2* ranges = reinterpret_cast<const uint2*>(ws + L.off_ranges);
    const uint32_t* vals = reinterpret_cast<const uint32_t*>(ws + L.off_vals[L.sorted_buffer]);
    const float4* rec = reinterpret_cast<const float4*>(ws + L.off_rec);
    const Ctrl* ctrl = reinterpret_cast<const Ctrl*>(ws + L.off_ctrl);
    float* tfin = reinterpret_cast<float*>(ws + L.off_tfinal);
    int32_t* last = reinterpret_cast<int32_t*>(ws + L.off_last);
    const int blocks = (int)L.ntiles;
    if (blocks <= 0) return;
#define VIS_LAUNCH_COMPOSITE(TS)                                                                      \
    composite_kernel<TS><<<blocks, TS * TS, 0, stream>>>(ranges, vals, rec, L.W, L.H, L.tiles_x, bg0, \
                                                         bg1, bg2, alpha_min, alpha_max, t_stop,      \
                                                         ctrl, out_rgb, out_alpha, tfin, last)
    if (L.tile == 8) VIS_LAUNCH_COMPOSITE(8);
    else if (L.tile == 32) VIS_LAUNCH_COMPOSITE(32);
    else VIS_LAUNCH_COMPOSITE(16);
#undef VIS_LAUNCH_COMPOSITE
}

}  // namespace vis
