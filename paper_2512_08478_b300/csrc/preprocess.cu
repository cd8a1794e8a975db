// K1 -- per-Gaussian preprocess (section 3.2 Eq. 1; Algorithm 1, Preprocess).
//
// One thread per Gaussian. Reads the caller's fp32 SoA attributes once and writes
// a 48-byte splat record, the view depth, the tile footprint (footprint.cuh) and the
// number of tiles touched; each block also writes the sum of its tiles-touched counts
// (or of its survivors) for the offset scan.
//
// Numerics. The camera transform and the perspective division are carried in
// float-float (error-free transforms) so that the pixel centre (u, v) is exact to
// ~1e-7 px even 1000 px from the principal point. The 2D covariance is formed as
// S = A A^T + dil I with A = J W R_q diag(s); its determinant as
// |A_0 x A_1|^2 + dil tr(A A^T) + dil^2 (no cancellation), and the splat is stored
// in whitened form: q' = (d.f1)^2 + (d.f2)^2 with f_k = sqrt(c) e_k / sqrt(lambda_k),
// (lambda_k, e_k) the eigenpairs of S and c = log2(e)/2. This is c d^T S^-1 d (Eq. 2's
// exponent in base 2) and stays well conditioned for needle-shaped splats, where the
// conic form (a, b, c) loses digits.
//
// Pre-packed scenes (PACKED: Algorithm 1's pre-pack, section 3.4's FP16 layout) give the
// mean, the opacity, the covariance's upper triangle and the SH coefficients as fp16 pairs.
// Their covariance arrives unfactored, so det S is formed from Sigma's cofactors
// (screen_cov_packed) rather than from S's rounded entries, which would cost eps cond(S).
#include <cuda_fp16.h>

#include "vis_internal.cuh"
#include "footprint.cuh"
#include "dynamic.cuh"

namespace vis {

__device__ __forceinline__ float half_lo(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu))); }
__device__ __forceinline__ float half_hi(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }

// S = T Sigma T^T + dil I for T = [T0; T1] (2x3) and Sigma = (xx, xy, xz, yy, yz, zz). The
// entries are plain float sums; det(T Sigma T^T) is taken as (T0 x T1)^T adj(Sigma) (T0 x T1)
// (the Cauchy-Binet form for a 2x3 T), with the cross product and Sigma's cofactors from
// Kahan's accurate a b - c d, so Sigma's large entries never cancel against each other:
// det S keeps ~1e-5 relative accuracy where s00 s11 - s01^2 in float loses eps cond(S).
__device__ __forceinline__ void screen_cov_packed(const float T0[3], const float T1[3], const float sg[6], float dil,
                                                  float& s00, float& s01, float& s11, float& det) {
    const float xx = sg[0], xy = sg[1], xz = sg[2], yy = sg[3], yz = sg[4], zz = sg[5];
    const float b00 = T0[0] * xx + T0[1] * xy + T0[2] * xz;   // (T0 Sigma)
    const float b01 = T0[0] * xy + T0[1] * yy + T0[2] * yz;
    const float b02 = T0[0] * xz + T0[1] * yz + T0[2] * zz;
    const float b10 = T1[0] * xx + T1[1] * xy + T1[2] * xz;   // (T1 Sigma)
    const float b11 = T1[0] * xy + T1[1] * yy + T1[2] * yz;
    const float b12 = T1[0] * xz + T1[1] * yz + T1[2] * zz;
    const float a00 = b00 * T0[0] + b01 * T0[1] + b02 * T0[2];
    const float a01 = b00 * T1[0] + b01 * T1[1] + b02 * T1[2];
    const float a11 = b10 * T1[0] + b11 * T1[1] + b12 * T1[2];
    const float c0 = diff_of_products(T0[1], T1[2], T0[2], T1[1]);
    const float c1 = diff_of_products(T0[2], T1[0], T0[0], T1[2]);
    const float c2 = diff_of_products(T0[0], T1[1], T0[1], T1[0]);
    const float A00 = diff_of_products(yy, zz, yz, yz), A11 = diff_of_products(xx, zz, xz, xz);
    const float A22 = diff_of_products(xx, yy, xy, xy), A01 = diff_of_products(xz, yz, xy, zz);
    const float A02 = diff_of_products(xy, yz, xz, yy), A12 = diff_of_products(xy, xz, xx, yz);
    const float q = c0 * c0 * A00 + c1 * c1 * A11 + c2 * c2 * A22 +
                    2.f * (c0 * c1 * A01 + c0 * c2 * A02 + c1 * c2 * A12);
    s00 = a00 + dil; s11 = a11 + dil; s01 = a01;
    det = q + dil * (a00 + a11) + dil * dil;
}

// One block of the preprocess: Gaussians local_block * 256 + threadIdx.x of the scene of p.
// ZCULL: a depth-tested render's occlusion cull against p.tile_zmax. `item` goes into the
// footprint's last word (the image of a fused batch; 0 otherwise).
template <bool FOLDED, bool PACKED, bool ZCULL>
__device__ __forceinline__ void preprocess_block(const PrepParams& p, int local_block, uint32_t item,
                                                 float4* __restrict__ rec, float* __restrict__ depth_out,
                                                 uint4* __restrict__ rect_out, uint32_t* __restrict__ touched_out,
                                                 uint32_t* __restrict__ block_sums) {
    // i: the Gaussian in the scene's arrays; gi: its slot in the workspace (a multi-scene
    // render places scene k at index_offset = the sum of the earlier scenes' padded sizes)
    const int i = local_block * kPrepThreads + threadIdx.x;
    const int gi = (int)p.index_offset + i;   // slots number at most 2^31 - 1
    __shared__ float s_trim[7][kPrepThreads];
    uint32_t touched = 0;
    if (p.dyn_flags && local_block == 0 && threadIdx.x == 0) *p.dyn_flags = kFlagNoAdjoint;
    if (i < p.n) {
        // --- camera-space position in float-float: p = R mu + t ---
        float mx, my, mz, opac;
        uint32_t cw0 = 0, cw1 = 0, cw2 = 0;   // packed covariance words
        if (PACKED) {
            // the covariance words go out with the position (one round trip fewer for the
            // Gaussians in front; 12 B more for the culled ones)
            cw0 = __ldg(p.pk_cov + 3 * (size_t)i);
            cw1 = __ldg(p.pk_cov + 3 * (size_t)i + 1);
            cw2 = __ldg(p.pk_cov + 3 * (size_t)i + 2);
            const uint2 w = __ldg(p.pk_pos + i);
            mx = half_lo(w.x); my = half_hi(w.x); mz = half_lo(w.y); opac = half_hi(w.y);
        } else {
            mx = __ldg(p.means + 3 * i + 0);
            my = __ldg(p.means + 3 * i + 1);
            mz = __ldg(p.means + 3 * i + 2);
            float logit = __ldg(p.logits + i);
            if (p.dyn_velocity) {   // a dynamic frame: frame 0's attributes updated as they are read
                mx = dyn_mean(mx, __ldg(p.dyn_velocity + 3 * i + 0), p.dyn_t);
                my = dyn_mean(my, __ldg(p.dyn_velocity + 3 * i + 1), p.dyn_t);
                mz = dyn_mean(mz, __ldg(p.dyn_velocity + 3 * i + 2), p.dyn_t);
                logit = dyn_logit(logit, __ldg(p.dyn_amp + i), __ldg(p.dyn_freq + i), __ldg(p.dyn_phase + i), p.dyn_t);
            }
            opac = 1.f / (1.f + __expf(-logit));
            // quaternion and log-scales are read after the cull test: start them towards L2
            asm volatile("prefetch.global.L2 [%0];" ::"l"(p.quats + 4 * (size_t)i));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(p.log_scales + 3 * (size_t)i));
        }
        float2 pc[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            float2 acc = make_float2(p.t[r], FOLDED ? p.t_lo[r] : 0.f);
            acc = ff_add(acc, two_prod(p.R[3 * r + 0], mx));
            acc = ff_add(acc, two_prod(p.R[3 * r + 1], my));
            acc = ff_add(acc, two_prod(p.R[3 * r + 2], mz));
            if (FOLDED) {
                acc.y = __fmaf_rn(p.R_lo[3 * r + 0], mx, acc.y);
                acc.y = __fmaf_rn(p.R_lo[3 * r + 1], my, acc.y);
                acc.y = __fmaf_rn(p.R_lo[3 * r + 2], mz, acc.y);
                acc = fast_two_sum(acc.x, acc.y);
            }
            pc[r] = acc;
        }
        const float z = pc[2].x;
        depth_out[gi] = z;
        bool ok = (z > p.near_z) && (opac >= p.alpha_min);

        uint32_t x0 = 0, x1 = 0, y0 = 0, y1 = 0, trims = 0;
        if (ok) {
            // --- pixel centre u = fx x/z + cx (float-float) ---
            const float2 rx = ff_div(pc[0], pc[2]);
            const float2 ry = ff_div(pc[1], pc[2]);
            if (fabsf(rx.x) <= p.limx && fabsf(ry.x) <= p.limy) {
                // centre inside the (guard-widened) frustum: the splat will very likely need its
                // colour row at the end; start it towards L2 now
                const char* row = PACKED ? reinterpret_cast<const char*>(p.pk_col + (size_t)i * p.col_words)
                                         : reinterpret_cast<const char*>(p.sh + (size_t)i * 3 * (p.deg + 1) * (p.deg + 1));
                const int bytes = PACKED ? 4 * p.col_words : 12 * (p.deg + 1) * (p.deg + 1);
                asm volatile("prefetch.global.L2 [%0];" ::"l"(row));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(row + bytes - 4));
            }
            float2 u, v;
            {
                float2 a = two_prod(p.fx, rx.x);
                a.y = __fmaf_rn(p.fx, rx.y, a.y);
                float2 s = two_sum(a.x, p.cx);
                u = fast_two_sum(s.x, __fadd_rn(s.y, a.y));
                float2 b = two_prod(p.fy, ry.x);
                b.y = __fmaf_rn(p.fy, ry.y, b.y);
                float2 s2 = two_sum(b.x, p.cy);
                v = fast_two_sum(s2.x, __fadd_rn(s2.y, b.y));
            }
            // --- EWA Jacobian at the camera-space mean, with the x/z, y/z guard ---
            const float zi = 1.f / z;
            const float tx = fminf(p.limx, fmaxf(-p.limx, rx.x));
            const float ty = fminf(p.limy, fmaxf(-p.limy, ry.x));
            const float J00 = p.fx * zi, J02 = -p.fx * tx * zi;
            const float J11 = p.fy * zi, J12 = -p.fy * ty * zi;
            // T = J W (2x3), W = camera rotation
            float T0[3], T1[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                T0[c] = J00 * p.R[c] + J02 * p.R[6 + c];
                T1[c] = J11 * p.R[3 + c] + J12 * p.R[6 + c];
            }
            float s00, s11, s01, det;
            if (PACKED) {
                const float sg[6] = {half_lo(cw0), half_hi(cw0), half_lo(cw1), half_hi(cw1), half_lo(cw2), half_hi(cw2)};
                screen_cov_packed(T0, T1, sg, p.dilation, s00, s01, s11, det);
            } else {
                // --- covariance factor M = R_q diag(s) ---
                const float4 q4 = __ldg(reinterpret_cast<const float4*>(p.quats) + i);
                float qw = q4.x, qx = q4.y, qy = q4.z, qz = q4.w;
                const float qn2 = qw * qw + qx * qx + qy * qy + qz * qz;
                if (qn2 < 1e-24f) { qw = 1.f; qx = qy = qz = 0.f; }
                else { const float inv = rsqrtf(qn2); qw *= inv; qx *= inv; qy *= inv; qz *= inv; }
                const float Rq[9] = {
                    1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
                    2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
                    2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
                const float s0 = __expf(__ldg(p.log_scales + 3 * i + 0));
                const float s1 = __expf(__ldg(p.log_scales + 3 * i + 1));
                const float s2 = __expf(__ldg(p.log_scales + 3 * i + 2));
                // A = T M: rows A0, A1 (3 each); M[:, k] = Rq[:, k] s_k
                float A0[3], A1[3];
                const float sk[3] = {s0, s1, s2};
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float m0 = Rq[0 + k] * sk[k], m1 = Rq[3 + k] * sk[k], m2 = Rq[6 + k] * sk[k];
                    A0[k] = T0[0] * m0 + T0[1] * m1 + T0[2] * m2;
                    A1[k] = T1[0] * m0 + T1[1] * m1 + T1[2] * m2;
                }
                const float a00 = A0[0] * A0[0] + A0[1] * A0[1] + A0[2] * A0[2];
                const float a11 = A1[0] * A1[0] + A1[1] * A1[1] + A1[2] * A1[2];
                const float a01 = A0[0] * A1[0] + A0[1] * A1[1] + A0[2] * A1[2];
                const float c0 = diff_of_products(A0[1], A1[2], A0[2], A1[1]);
                const float c1 = diff_of_products(A0[2], A1[0], A0[0], A1[2]);
                const float c2 = diff_of_products(A0[0], A1[1], A0[1], A1[0]);
                const float dil = p.dilation;
                s00 = a00 + dil; s11 = a11 + dil; s01 = a01;
                det = (c0 * c0 + c1 * c1 + c2 * c2) + dil * (a00 + a11) + dil * dil;
            }
            if (det > 0.f) {
                const float m = 0.5f * (s00 + s11);
                const float h = 0.5f * (s00 - s11);
                const float disc = h * h + s01 * s01;
                const float rt = sqrtf(disc);
                const float lam1 = m + rt;                 // largest eigenvalue
                const float lam2 = det / lam1;             // smallest, without cancellation
                float ex, ey;
                if (h >= 0.f) { ex = h + rt; ey = s01; } else { ex = s01; ey = rt - h; }
                const float en2 = ex * ex + ey * ey;
                if (en2 > 0.f) { const float inv = rsqrtf(en2); ex *= inv; ey *= inv; }
                else { ex = 1.f; ey = 0.f; }
                const float i1 = rsqrtf(lam1) * p.wscale, i2 = rsqrtf(lam2) * p.wscale;
                const float T = (float)p.tile;
                const float ftx = (float)p.tiles_x, fty = (float)p.tiles_y;
                float fx0, fx1, fy0, fy1;
                if (p.tight_extent) {
                    // tight box of the region a pixel can take the splat from: q <= min(9, 2 ln(o / alpha_min))
                    // (the 3-sigma cut and the alpha_min skip), padded for float rounding
                    const float qthr = fminf(9.f, 2.f * logf(opac / p.alpha_min)) * 1.0002f;
                    const float rx = sqrtf(qthr * s00) * 1.0001f + 0.01f;
                    const float ry = sqrtf(qthr * s11) * 1.0001f + 0.01f;
                    // pixel px is reachable iff |px + 0.5 - u| <= rx
                    fx0 = floorf((u.x - rx - 0.5f) / T); fx1 = floorf((u.x + rx - 0.5f) / T) + 1.f;
                    fy0 = floorf((v.x - ry - 0.5f) / T); fy1 = floorf((v.x + ry - 0.5f) / T) + 1.f;
                } else {
                    // conservative square of radius ceil(3 sqrt(lambda_max)) plus one pixel
                    const float lam_ext = m + sqrtf(fmaxf(0.1f, disc));
                    const float radius = ceilf(3.f * sqrtf(lam_ext));
                    fx0 = floorf((u.x - radius - 1.f) / T); fx1 = floorf((u.x + radius + 1.f) / T) + 1.f;
                    fy0 = floorf((v.x - radius - 1.f) / T); fy1 = floorf((v.x + radius + 1.f) / T) + 1.f;
                }
                // clamp in float before converting (u may be far off screen)
                const int ix0 = (int)fminf(ftx, fmaxf(0.f, fx0));
                const int ix1 = (int)fminf(ftx, fmaxf(0.f, fx1));
                const int iy0 = (int)fminf(fty, fmaxf(0.f, fy0));
                const int iy1 = (int)fminf(fty, fmaxf(0.f, fy1));
                touched = (ix1 > ix0 && iy1 > iy0) ? (uint32_t)((ix1 - ix0) * (iy1 - iy0)) : 0u;
                if (ZCULL && touched > 0 && touched <= 64) {
                    // behind the depth buffer in every tile it reaches: no pixel would take it
                    float zm = __int_as_float(0xff800000);
                    for (int ty = iy0; ty < iy1; ++ty)
                        for (int tx = ix0; tx < ix1; ++tx) zm = fmaxf(zm, __ldg(p.tile_zmax + ty * p.tiles_x + tx));
                    if (z > zm) touched = 0;
                }
                // the outer-row trims below need these after the colour; they wait in shared
                // memory rather than in registers across the SH evaluation
                s_trim[0][threadIdx.x] = s00; s_trim[1][threadIdx.x] = s11; s_trim[2][threadIdx.x] = s01;
                s_trim[3][threadIdx.x] = det; s_trim[4][threadIdx.x] = opac;
                s_trim[5][threadIdx.x] = u.x; s_trim[6][threadIdx.x] = v.x;
                if (touched > 0) {
                    x0 = ix0; x1 = ix1; y0 = iy0; y1 = iy1;
                    // --- colour from SH at dir = normalize(mu - camera centre) ---
                    float dx = mx - p.cam_pos[0], dy = my - p.cam_pos[1], dz = mz - p.cam_pos[2];
                    const float dinv = rsqrtf(dx * dx + dy * dy + dz * dz);
                    dx *= dinv; dy *= dinv; dz *= dinv;
                    const int K = (p.deg + 1) * (p.deg + 1);
                    float Y[16];
                    Y[0] = p.shc[9];
                    if (p.deg >= 1) {
                        Y[1] = -p.shc[1] * dy; Y[2] = p.shc[0] * dz; Y[3] = -p.shc[1] * dx;
                    }
                    if (p.deg >= 2) {
                        const float xx = dx * dx, yy = dy * dy, zz = dz * dz;
                        Y[4] = 2.f * p.shc[4] * dx * dy;
                        Y[5] = -p.shc[3] * dy * dz;
                        Y[6] = p.shc[2] * (3.f * zz - 1.f);
                        Y[7] = -p.shc[3] * dx * dz;
                        Y[8] = p.shc[4] * (xx - yy);
                        if (p.deg >= 3) {
                            Y[9] = -p.shc[8] * (3.f * xx * dy - yy * dy);
                            Y[10] = 2.f * p.shc[7] * dx * dy * dz;
                            Y[11] = -p.shc[6] * (5.f * zz - 1.f) * dy;
                            Y[12] = p.shc[5] * (5.f * zz * dz - 3.f * dz);
                            Y[13] = -p.shc[6] * (5.f * zz - 1.f) * dx;
                            Y[14] = p.shc[7] * dz * (xx - yy);
                            Y[15] = -p.shc[8] * (xx * dx - 3.f * dx * yy);
                        }
                    }
                    float col[3] = {0.5f, 0.5f, 0.5f};
                    const float* shi = p.sh + (size_t)i * K * 3;
                    if (PACKED) {
                        const uint32_t* ci = p.pk_col + (size_t)i * p.col_words;
                        if (p.deg == 3) {   // 24 words = six 16-byte loads
                            const uint4* c4 = reinterpret_cast<const uint4*>(ci);
                            float buf[48];
#pragma unroll
                            for (int k = 0; k < 6; ++k) {
                                const uint4 w = __ldg(c4 + k);
                                buf[8 * k + 0] = half_lo(w.x); buf[8 * k + 1] = half_hi(w.x);
                                buf[8 * k + 2] = half_lo(w.y); buf[8 * k + 3] = half_hi(w.y);
                                buf[8 * k + 4] = half_lo(w.z); buf[8 * k + 5] = half_hi(w.z);
                                buf[8 * k + 6] = half_lo(w.w); buf[8 * k + 7] = half_hi(w.w);
                            }
#pragma unroll
                            for (int k = 0; k < 16; ++k) {
                                col[0] += buf[3 * k] * Y[k]; col[1] += buf[3 * k + 1] * Y[k];
                                col[2] += buf[3 * k + 2] * Y[k];
                            }
                        } else {
                            for (int k = 0; k < K; ++k) {
#pragma unroll
                                for (int c = 0; c < 3; ++c) {
                                    const int h = 3 * k + c;
                                    const uint32_t w = __ldg(ci + (h >> 1));
                                    col[c] += ((h & 1) ? half_hi(w) : half_lo(w)) * Y[k];
                                }
                            }
                        }
                    } else if (p.deg == 3) {
                        const float4* s4 = reinterpret_cast<const float4*>(shi);
                        float buf[48];
#pragma unroll
                        for (int k = 0; k < 12; ++k) {
                            const float4 w = __ldg(s4 + k);
                            buf[4 * k] = w.x; buf[4 * k + 1] = w.y; buf[4 * k + 2] = w.z; buf[4 * k + 3] = w.w;
                        }
#pragma unroll
                        for (int k = 0; k < 16; ++k) {
                            col[0] += buf[3 * k] * Y[k]; col[1] += buf[3 * k + 1] * Y[k]; col[2] += buf[3 * k + 2] * Y[k];
                        }
                    } else {
                        for (int k = 0; k < K; ++k) {
                            col[0] += __ldg(shi + 3 * k) * Y[k];
                            col[1] += __ldg(shi + 3 * k + 1) * Y[k];
                            col[2] += __ldg(shi + 3 * k + 2) * Y[k];
                        }
                    }
                    rec[3 * (size_t)gi + 0] = make_float4(u.x, v.x, u.y, v.y);
                    rec[3 * (size_t)gi + 1] = make_float4(ex * i1, ey * i1, -ey * i2, ex * i2);
                    rec[3 * (size_t)gi + 2] = make_float4(opac, fmaxf(col[0], 0.f), fmaxf(col[1], 0.f),
                                                         fmaxf(col[2], 0.f));
                }
                if (touched > 0 && p.tight_extent == 2 && ix1 - ix0 > 1) {
                    // exact outer rows: narrow the box's top and bottom rows to the tiles their
                    // band of pixel centres of the ellipse d^T S^-1 d <= qthr reaches. For dy
                    // fixed the ellipse spans dx = (s01/s11) dy +- sqrt((det/s11)(qthr - dy^2/s11));
                    // over a band of dy its leftmost (rightmost) point is at dy = -+ s01 sqrt(qthr/s00)
                    // clamped to the band. Padded like the box for float rounding.
                    const float s00 = s_trim[0][threadIdx.x], s11 = s_trim[1][threadIdx.x];
                    const float s01 = s_trim[2][threadIdx.x], det = s_trim[3][threadIdx.x];
                    const float opac = s_trim[4][threadIdx.x], ux = s_trim[5][threadIdx.x];
                    const float vx = s_trim[6][threadIdx.x];
                    const float qthr = fminf(9.f, 2.f * logf(opac / p.alpha_min)) * 1.0002f;
                    const float inv11 = 1.f / s11;
                    const float kx = s01 * inv11, hwf = det * inv11;
                    const float yext = sqrtf(qthr * s11) * 1.0001f + 0.01f;
                    const float dyl = -s01 * sqrtf(qthr / s00);
                    const float pad = 1e-4f * sqrtf(qthr * s00) + 0.02f;
                    const float fW = (float)(ix1 - ix0);
                    const int rows = iy1 - iy0;
                    uint32_t lr[4] = {0u, 0u, 0u, 0u};
#pragma unroll 1
                    for (int e = 0; e < (rows > 1 ? 2 : 1); ++e) {
                        const int ty = e == 0 ? iy0 : iy1 - 1;
                        const float ya = (float)(ty * p.tile) + 0.5f - vx - 0.02f;
                        const float yb = (float)(ty * p.tile + p.tile) - 0.5f - vx + 0.02f;
                        float fl = fW, fr = 0.f;   // a row the ellipse misses keeps no tile
                        if (ya <= yext && yb >= -yext) {
                            const float lo = fmaxf(ya, -yext), hi = fminf(yb, yext);
                            const float dL = fminf(fmaxf(dyl, lo), hi), dR = fminf(fmaxf(-dyl, lo), hi);
                            const float xmin = kx * dL - sqrtf(fmaxf(0.f, hwf * (qthr - dL * dL * inv11))) - pad;
                            const float xmax = kx * dR + sqrtf(fmaxf(0.f, hwf * (qthr - dR * dR * inv11))) + pad;
                            const float ta = floorf((ux + xmin - 0.5f) / T), tb = floorf((ux + xmax - 0.5f) / T);
                            fl = fminf(fmaxf(0.f, ta - (float)ix0), fW);
                            fr = fminf(fmaxf(0.f, (float)(ix1 - 1) - tb), fW - fl);
                        }
                        lr[2 * e] = (uint32_t)fminf(fl, 255.f);
                        lr[2 * e + 1] = (uint32_t)fminf(fr, 255.f);
                    }
                    trims = fp_pack_trims(lr[0], lr[1], lr[2], lr[3]);
                    const Footprint f = {(uint32_t)ix0, (uint32_t)ix1, (uint32_t)iy0, (uint32_t)iy1, trims};
                    touched = fp_count(f);   // the count every copy enumerator agrees with
                }
            }
        }
        if (touched == 0) { x0 = x1 = y0 = y1 = 0; trims = 0; }
        else { y0 += p.canvas_row0; y1 += p.canvas_row0; }   // a batch image's rows in its canvas
        rect_out[gi] = make_uint4(x0 | (x1 << 16), y0 | (y1 << 16), trims, item);
        touched_out[gi] = touched;
    } else if (i < p.n_pad) {   // padding slots of a multi-scene render or a batch: no copies
        rect_out[gi] = make_uint4(0u, 0u, 0u, item);
        touched_out[gi] = 0u;
    }
    // block sum of tiles touched (for the offset scan of the index-order duplication) or, for
    // the depth-first sorts, of survivors (for their compaction)
    __shared__ uint32_t warp_sums[kPrepThreads / 32];
    uint32_t s = p.count_survivors ? (touched > 0 ? 1u : 0u) : touched;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < kPrepThreads / 32; ++w) tot += warp_sums[w];
        block_sums[p.index_offset / kPrepThreads + local_block] = tot;
    }
}

template <bool FOLDED, bool PACKED, bool ZCULL>
__global__ void __launch_bounds__(kPrepThreads, 5)
preprocess_kernel(PrepParams p, float4* __restrict__ rec, float* __restrict__ depth_out,
                  uint4* __restrict__ rect_out, uint32_t* __restrict__ touched_out,
                  uint32_t* __restrict__ block_sums) {
    preprocess_block<FOLDED, PACKED, ZCULL>(p, (int)blockIdx.x, 0u, rec, depth_out, rect_out, touched_out,
                                            block_sums);
}

// The preprocess of a fused batch: one launch over the work list of every (asset, camera)
// item. Block b belongs to the item whose first block blk0[item] is the last <= b; the
// item's parameters (scene arrays, camera, image size, workspace slots) are read into
// shared memory and the block runs as block b - blk0[item] of that item's preprocess. This
// file is compiled without floating-point contraction (every a * b + c not written as an
// fma is a rounded product and a rounded sum), so that the arithmetic cannot depend on
// where the parameters live: a batch's images are bit for bit those of plain renders.
static_assert(sizeof(PrepParams) % 4 == 0, "parameters copied as words");
template <bool PACKED>
__global__ void __launch_bounds__(kPrepThreads, 5)
preprocess_batch_kernel(const PrepParams* __restrict__ items, const uint32_t* __restrict__ blk0, int n_items,
                        float4* __restrict__ rec, float* __restrict__ depth_out, uint4* __restrict__ rect_out,
                        uint32_t* __restrict__ touched_out, uint32_t* __restrict__ block_sums) {
    pdl_entry();
    __shared__ PrepParams sp;
    __shared__ int s_item;
    const uint32_t b = blockIdx.x;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n_items - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (blk0[mid] <= b) lo = mid; else hi = mid - 1;
        }
        s_item = lo;
    }
    __syncthreads();
    const int item = s_item;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(items + item);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sp);
    for (int k = threadIdx.x; k < (int)(sizeof(PrepParams) / 4); k += kPrepThreads) dst[k] = src[k];
    __syncthreads();
    preprocess_block<false, PACKED, false>(sp, (int)(b - blk0[item]), sp.batch_image, rec, depth_out, rect_out,
                                           touched_out, block_sums);
}

void launch_preprocess_batch(const PrepParams* items, const uint32_t* blk0, int n_items, int64_t blocks,
                             bool packed, const Layout& L, char* ws, cudaStream_t stream) {
    if (n_items <= 0 || blocks <= 0) return;
    launch_k(false, packed ? preprocess_batch_kernel<true> : preprocess_batch_kernel<false>, (unsigned)blocks,
             kPrepThreads, 0, stream, items, blk0, n_items, reinterpret_cast<float4*>(ws + L.off_rec),
             reinterpret_cast<float*>(ws + L.off_depth), reinterpret_cast<uint4*>(ws + L.off_rect),
             reinterpret_cast<uint32_t*>(ws + L.off_touched), reinterpret_cast<uint32_t*>(ws + L.off_bsum));
}

void launch_preprocess(const PrepParams& p, const Layout& L, char* ws, cudaStream_t stream) {
    if (p.n_pad <= 0) return;
    const int blocks = (p.n_pad + kPrepThreads - 1) / kPrepThreads;
    bool folded = false;
    for (int k = 0; k < 9; ++k) folded |= p.R_lo[k] != 0.f;
    for (int k = 0; k < 3; ++k) folded |= p.t_lo[k] != 0.f;
    const bool packed = p.pk_pos != nullptr;
    auto kernel = p.tile_zmax
        ? (packed ? (folded ? preprocess_kernel<true, true, true> : preprocess_kernel<false, true, true>)
                  : (folded ? preprocess_kernel<true, false, true> : preprocess_kernel<false, false, true>))
        : (packed ? (folded ? preprocess_kernel<true, true, false> : preprocess_kernel<false, true, false>)
                  : (folded ? preprocess_kernel<true, false, false> : preprocess_kernel<false, false, false>));
    kernel<<<blocks, kPrepThreads, 0, stream>>>(
        p, reinterpret_cast<float4*>(ws + L.off_rec), reinterpret_cast<float*>(ws + L.off_depth),
        reinterpret_cast<uint4*>(ws + L.off_rect), reinterpret_cast<uint32_t*>(ws + L.off_touched),
        reinterpret_cast<uint32_t*>(ws + L.off_bsum));
}

// Largest depth-buffer value of every tile (one warp per tile; NaN counts as +inf: it rejects
// nothing), for the preprocess's occlusion cull.
__global__ void __launch_bounds__(256)
tile_zmax_kernel(const float* __restrict__ zlim, int W, int H, int tile, int tiles_x, int ntiles,
                 float* __restrict__ zmax) {
    const int t = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (t >= ntiles) return;
    const int tx = t % tiles_x, ty = t / tiles_x;
    float m = __int_as_float(0xff800000);
    for (int k = lane; k < tile * tile; k += 32) {
        const int x = tx * tile + k % tile, y = ty * tile + k / tile;
        if (x < W && y < H) {
            const float v = __ldg(zlim + (size_t)y * W + x);
            m = fmaxf(m, isnan(v) ? __int_as_float(0x7f800000) : v);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) zmax[t] = m;
}

void launch_tile_zmax(const Layout& L, char* ws, const float* zlim, cudaStream_t stream) {
    const int nt = (int)L.ntiles;
    tile_zmax_kernel<<<(nt + 7) / 8, 256, 0, stream>>>(zlim, L.W, L.H, L.tile, L.tiles_x, nt,
                                                       reinterpret_cast<float*>(ws + L.off_zmax));
}

// Pre-pack (Algorithm 1, once per scene): Sigma = M M^T with M = R_q diag(exp(log_s)),
// alpha = sigmoid(logit); mean, alpha, Sigma's upper triangle and the SH coefficients rounded
// to fp16 (nearest even) and packed two per uint32, low half first.
__global__ void __launch_bounds__(256)
pack_kernel(const float* __restrict__ means, const float* __restrict__ log_scales, const float* __restrict__ quats,
            const float* __restrict__ logits, const float* __restrict__ sh, int deg, int64_t n,
            uint2* __restrict__ pos, uint32_t* __restrict__ cov, uint32_t* __restrict__ col) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    auto pk = [](float lo, float hi) {
        return (uint32_t)__half_as_ushort(__float2half_rn(lo)) | ((uint32_t)__half_as_ushort(__float2half_rn(hi)) << 16);
    };
    const float alpha = 1.f / (1.f + expf(-logits[i]));
    pos[i] = make_uint2(pk(means[3 * i], means[3 * i + 1]), pk(means[3 * i + 2], alpha));
    float qw = quats[4 * i], qx = quats[4 * i + 1], qy = quats[4 * i + 2], qz = quats[4 * i + 3];
    const float qn2 = qw * qw + qx * qx + qy * qy + qz * qz;
    if (qn2 < 1e-24f) { qw = 1.f; qx = qy = qz = 0.f; }
    else { const float inv = 1.f / sqrtf(qn2); qw *= inv; qx *= inv; qy *= inv; qz *= inv; }
    const float Rq[9] = {
        1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
        2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
        2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
    float s2[3];
    for (int k = 0; k < 3; ++k) { const float sk = expf(log_scales[3 * i + k]); s2[k] = sk * sk; }
    float S[6];   // xx, xy, xz, yy, yz, zz
    const int ra[6] = {0, 0, 0, 1, 1, 2}, rb[6] = {0, 1, 2, 1, 2, 2};
    for (int e = 0; e < 6; ++e) {
        float acc = 0.f;
        for (int k = 0; k < 3; ++k) acc = __fmaf_rn(Rq[3 * ra[e] + k] * s2[k], Rq[3 * rb[e] + k], acc);
        S[e] = acc;
    }
    cov[3 * i] = pk(S[0], S[1]);
    cov[3 * i + 1] = pk(S[2], S[3]);
    cov[3 * i + 2] = pk(S[4], S[5]);
    const int K3 = 3 * (deg + 1) * (deg + 1), W = packed_col_words(deg);
    const float* shi = sh + i * K3;
    uint32_t* ci = col + i * W;
    for (int w = 0; w < W; ++w) {
        const int h = 2 * w;
        ci[w] = pk(h < K3 ? shi[h] : 0.f, h + 1 < K3 ? shi[h + 1] : 0.f);
    }
}

void launch_pack(const float* means, const float* log_scales, const float* quats, const float* logits,
                 const float* sh, int deg, int64_t n, uint2* pos, uint32_t* cov, uint32_t* col, cudaStream_t stream) {
    if (n <= 0) return;
    pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(means, log_scales, quats, logits, sh, deg, n, pos,
                                                                 cov, col);
}

}  // namespace vis
