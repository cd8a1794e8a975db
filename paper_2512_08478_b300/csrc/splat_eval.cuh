// Per (pixel, splat) evaluation shared by the compositor and its adjoint, written
// with explicit rounding intrinsics so both kernels take bit-identical decisions.
//
// Splat record in the workspace (3 x float4 per Gaussian, written by the preprocess):
//   r0 = (u_hi, v_hi, u_lo, v_lo)   pixel-space centre in float-float
//   r1 = (f1x, f1y, f2x, f2y)       scaled whitening rows: q' = (d.f1)^2 + (d.f2)^2
//                                   = c d^T S^-1 d with c = log2(e)/2, so that the
//                                   Gaussian factor of Eq. 2 is exp(-q/2) = 2^-q'
//   r2 = (opacity, r, g, b)
// For one tile the compositor stages each splat once (StagedSplat) with its centre
// relative to the tile centre and one threshold that folds the 3-sigma cut (q <= 9)
// and the alpha_min skip (opacity 2^-q' >= alpha_min) into q' <= thr.
#pragma once
#include "vis_internal.cuh"

namespace vis {

struct StagedSplat {
    float4 a;   // (du, dv, f1x, f1y): centre relative to the tile centre
    float4 b;   // (f2x, f2y, thr, opacity)
    float4 c;   // (r, g, b, unused)
};

// qcut = 9 c (the 3-sigma cut in q' units), alpha_min as in the options.
__device__ __forceinline__ StagedSplat stage_splat(const float4* __restrict__ rec, uint32_t g, float xc, float yc,
                                                   float qcut, float alpha_min) {
    const float4 r0 = rec[3 * (size_t)g + 0];
    const float4 r1 = rec[3 * (size_t)g + 1];
    const float4 r2 = rec[3 * (size_t)g + 2];
    StagedSplat s;
    s.a = make_float4(__fadd_rn(__fsub_rn(r0.x, xc), r0.z), __fadd_rn(__fsub_rn(r0.y, yc), r0.w), r1.x, r1.y);
    const float thr = fminf(qcut, __log2f(__fdiv_rn(r2.x, alpha_min)));
    s.b = make_float4(r1.z, r1.w, thr, r2.x);
    s.c = make_float4(r2.y, r2.z, r2.w, 0.f);
    return s;
}

// Bit w set iff the pixel centres of warp block w may hold a pixel with q'(d) <= thr: the
// block's rectangle of pixel centres meets both the exact axis-aligned box of the ellipse
// {d : q'(d) <= thr} and its oriented box, the two slabs |d.f_k| <= sqrt(thr) along the
// whitening rows (q' = (d.f1)^2 + (d.f2)^2, so every point of the ellipse lies in both).
// Both tests are padded for float rounding, so no block with such a pixel is dropped.
// Blocks are 8 px wide and BH px tall, BX per row of the CTA's square, NW in all; the square
// starts at (ox, oy) pixels from the tile's corner (a CTA covering part of its tile);
// coordinates are relative to the tile centre (half = TILE / 2).
template <int NW, int BX, int BH>
__device__ __forceinline__ uint32_t warp_block_mask(const StagedSplat& s, float half, float ox = 0.f, float oy = 0.f) {
    // half extents sqrt(thr (Q'^-1)_xx), sqrt(thr (Q'^-1)_yy) with Q' = F^T F, F = [f1; f2]
    const float det = fabsf(__fmaf_rn(s.a.z, s.b.y, -__fmul_rn(s.a.w, s.b.x)));
    const float rt = sqrtf(fmaxf(s.b.z, 0.f));
    const float ext = rt / det;
    const float rx = ext * sqrtf(__fmaf_rn(s.a.w, s.a.w, __fmul_rn(s.b.y, s.b.y))) * 1.0001f + 1e-3f;
    const float ry = ext * sqrtf(__fmaf_rn(s.a.z, s.a.z, __fmul_rn(s.b.x, s.b.x))) * 1.0001f + 1e-3f;
    // slab half-widths of a block in the f1, f2 directions, and the padded slab bound
    constexpr float hx = 3.5f, hy = 0.5f * BH - 0.5f;
    const float e1 = fabsf(s.a.z) * hx + fabsf(s.a.w) * hy;
    const float e2 = fabsf(s.b.x) * hx + fabsf(s.b.y) * hy;
    const float bound = rt * 1.0001f + 1e-4f;
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const float mx = ox + (float)((w % BX) * 8) + 4.f - half;
        const float my = oy + (float)((w / BX) * BH) + 0.5f * BH - half;
        const float dx = mx - s.a.x, dy = my - s.a.y;
        const float ox = fabsf(dx) - 3.5f, oy = fabsf(dy) - (0.5f * BH - 0.5f);
        const float p1 = fabsf(__fmaf_rn(dy, s.a.w, __fmul_rn(dx, s.a.z))) - e1;
        const float p2 = fabsf(__fmaf_rn(dy, s.b.y, __fmul_rn(dx, s.b.x))) - e2;
        if (ox <= rx && oy <= ry && p1 <= bound && p2 <= bound) m |= 1u << w;
    }
    return m;
}

struct PairEval {
    float dx, dy, p1, p2, q;
};

// (lx, ly): pixel centre relative to the tile centre; q is q' (scaled).
__device__ __forceinline__ PairEval eval_pair(float lx, float ly, float4 a, float4 b) {
    PairEval e;
    e.dx = __fsub_rn(lx, a.x);
    e.dy = __fsub_rn(ly, a.y);
    e.p1 = __fmaf_rn(e.dy, a.w, __fmul_rn(e.dx, a.z));
    e.p2 = __fmaf_rn(e.dy, b.y, __fmul_rn(e.dx, b.x));
    e.q = __fmaf_rn(e.p2, e.p2, __fmul_rn(e.p1, e.p1));
    return e;
}

// Gaussian factor of Eq. 2 from the scaled Mahalanobis distance: 2^-q' = exp(-q/2)
// (one ex2 instruction; relative error ~2^-22 over the range used, q' <= 6.5)
__device__ __forceinline__ float gauss_of_qs(float qs) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-qs));
    return y;
}

}  // namespace vis
