// K7 -- adjoint of the render (section 3.2: the splatting formulation is
// differentiable in every Gaussian parameter).
//
// K7a composite_backward_kernel: one CTA per tile, one thread per pixel, each warp an
// 8 x 4 pixel block, walking the tile's sorted range back to front in shared-memory
// chunks -- per warp only the splats whose 3-sigma box meets its block -- starting
// from the final transmittance and the last contributor the forward stored. Per-splat
// alphas are recomputed (with the forward's exact arithmetic, so every skip and cut
// decision is the same) rather than stored; T before each splat is recovered as
// T / (1 - alpha). With S the colour behind a splat, normalised by the
// transmittance after it (S <- rgb a + (1 - a) S walking backwards):
//   dC/drgb = a T,  dC/da = T (rgb - S) - T_final bg / (1 - a),  dA/da = T_final / (1 - a).
// The nine screen-space gradients of a splat (u, v, conic a/b/c, opacity, rgb) are
// summed over the warp with shuffles and added to global memory by one lane.
//
// K7b preprocess_backward_kernel: one thread per Gaussian chains those through
// conic = S^-1, S = A A^T + dil I with A = J W R_q diag(s), the projection, the
// quaternion normalisation, exp, sigmoid and the SH basis.
#include "splat_eval.cuh"

namespace vis {

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums eight per-lane values over the warp with 9 shuffles (recursive halving: each
// exchange step hands half of the remaining values to the partner lane). On return,
// lanes with (lane & 3) == 0 hold the total of value index
// 4 bit4(lane) + 2 bit3(lane) + bit2(lane); the index is returned in *which.
__device__ __forceinline__ float warp_sum8_transposed(const float v[8], int lane, int* which) {
    const bool u4 = lane & 16, u3 = lane & 8, u2 = lane & 4;
    float w[4], x[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = u4 ? v[i] : v[i + 4];
        const float keep = u4 ? v[i + 4] : v[i];
        w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = u3 ? w[i] : w[i + 2];
        const float keep = u3 ? w[i + 2] : w[i];
        x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float y = (u2 ? x[1] : x[0]) + __shfl_xor_sync(0xffffffffu, u2 ? x[0] : x[1], 4);
    y += __shfl_xor_sync(0xffffffffu, y, 2);
    y += __shfl_xor_sync(0xffffffffu, y, 1);
    *which = (u4 ? 4 : 0) + (u3 ? 2 : 0) + (u2 ? 1 : 0);
    return y;
}

// The warp's nine gradient terms of one splat summed over the warp and added to dst[0..8]
// (one lane per value; zero sums are skipped).
__device__ __forceinline__ void warp_add_gradients(const float g[9], int lane, float* dst) {
    int which;
    const float t8 = warp_sum8_transposed(g, lane, &which);
    const float t9 = warp_sum(g[8]);
    if ((lane & 3) == 0 && t8 != 0.f) atomicAdd(dst + which, t8);
    if (lane == 1 && t9 != 0.f) atomicAdd(dst + 8, t9);
}

template <int TILE, int SUB, int PPT, bool DEPTH>
__global__ void __launch_bounds__(SUB * SUB / PPT)
composite_backward_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                          const float4* __restrict__ rec, int W, int H, int tiles_x, float bg0,
                          float bg1, float bg2, float alpha_min, float alpha_max, float qcut, float inv_scale,
                          const float* __restrict__ t_final, const int32_t* __restrict__ last_in,
                          const float* __restrict__ d_rgb, const float* __restrict__ d_alpha,
                          float* __restrict__ g2, const float* __restrict__ depth,
                          const float* __restrict__ zlim, Ctrl* __restrict__ ctrl,
                          const uint32_t* __restrict__ order) {
    if (ctrl->flags & kFlagNoAdjoint) {   // a dynamic frame: its attributes were never stored
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ctrl->error, kErrNoAdjoint);
        return;
    }
    if (ctrl->error) return;   // the forward produced no valid lists: leave the gradients at zero
    // a CTA takes one SUB x SUB square of its tile (the whole tile's list), as the forward does
    static_assert(TILE % SUB == 0, "the squares tile the tile");
    constexpr int NSUB = (TILE / SUB) * (TILE / SUB);
    constexpr int NT = SUB * SUB / PPT;       // threads; each owns PPT vertically adjacent pixels
    constexpr int NW = NT / 32;               // warps; each owns an 8 x (4 PPT) pixel block
    constexpr int BX = SUB / 8, BH = 4 * PPT;
    constexpr int CH = NT < 256 ? NT : 256;   // splats staged per chunk
    static_assert(NW == BX * (SUB / BH), "warp blocks tile the square");
    // staged splats, NS float4 slots each: PPT 1 -> (du, dv, f1x, f1y), (f2x, f2y, thr, opacity),
    // (r, g, b, depth); PPT 2 -> packed pairs for the f32x2 instructions (see the pair walk)
    constexpr int NS = PPT == 1 ? 3 : 6;
    __shared__ float4 s_st[NS][CH];
    __shared__ uint32_t s_g[CH], s_mask[CH];
    __shared__ uint16_t s_list[NW][CH];
    const int tile = order ? (int)order[blockIdx.x / NSUB] : (int)(blockIdx.x / NSUB);   // longest first if ordered
    const int sub = (int)(blockIdx.x % NSUB);
    const int sx = (sub % (TILE / SUB)) * SUB, sy = (sub / (TILE / SUB)) * SUB;   // the square in the tile
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int bx = warp % BX, by = warp / BX;
    const int px = tx * TILE + sx + bx * 8 + (lane & 7);
    const size_t HW = (size_t)H * W;
    const float half = 0.5f * TILE;
    const float xc = (float)(tx * TILE) + half, yc = (float)(ty * TILE) + half;
    const float lx = (float)px + 0.5f - xc;
    const uint2 r = ranges[tile];

    // per pixel: the walk state (T, S), the incoming gradients and the terms constant
    // along the walk
    bool inside[PPT];
    float ly[PPT], T[PPT], TN[PPT], gC0[PPT], gC1[PPT], gC2[PPT], gA[PPT], dl[PPT];
    float aterm[PPT], S0[PPT], S1[PPT], S2[PPT];
    int32_t last[PPT];
    int32_t my_last = 0;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int py = ty * TILE + sy + by * BH + (lane >> 3) * PPT + q;
        inside[q] = px < W && py < H;
        const size_t pix = (size_t)py * W + px;
        ly[q] = (float)py + 0.5f - yc;
        T[q] = TN[q] = 1.f; gC0[q] = gC1[q] = gC2[q] = gA[q] = 0.f; last[q] = 0;
        dl[q] = (DEPTH && inside[q]) ? zlim[pix] : __int_as_float(0x7f800000);   // depth limit
        if (inside[q]) {
            TN[q] = t_final[pix];
            T[q] = TN[q];
            last[q] = last_in[pix];
            gC0[q] = d_rgb[pix]; gC1[q] = d_rgb[HW + pix]; gC2[q] = d_rgb[2 * HW + pix];
            gA[q] = d_alpha[pix];
        }
        aterm[q] = (gA[q] - (bg0 * gC0[q] + bg1 * gC1[q] + bg2 * gC2[q])) * TN[q];   // (gA - bg.gC) T_final
        S0[q] = S1[q] = S2[q] = 0.f;
        my_last = max(my_last, last[q]);
    }

    // block-wide maximum of `last` bounds the walk
    __shared__ int32_t s_max_last;
    if (threadIdx.x == 0) s_max_last = 0;
    __syncthreads();
    atomicMax(&s_max_last, my_last);
    __syncthreads();
    const uint32_t end = (uint32_t)max((int32_t)r.x, s_max_last);

    for (int64_t top = end; top > (int64_t)r.x; top -= CH) {
        const int64_t lo = max((int64_t)r.x, top - CH);
        const int cnt = (int)(top - lo);
        __syncthreads();
        if (threadIdx.x < cnt) {
            const int t = threadIdx.x;
            const uint32_t g = vals[lo + t];
            const StagedSplat st = stage_splat(rec, g, xc, yc, qcut, alpha_min);
            const float z = DEPTH ? depth[g] : 0.f;
            s_g[t] = g;
            if constexpr (PPT == 1) {
                s_st[0][t] = st.a;
                s_st[1][t] = st.b;
                s_st[2][t] = make_float4(st.c.x, st.c.y, st.c.z, z);
            } else {
                s_st[0][t] = make_float4(-st.a.x, -st.a.x, -st.a.y, -st.a.y);
                s_st[1][t] = make_float4(st.a.z, st.a.z, st.b.x, st.b.x);
                s_st[2][t] = make_float4(st.a.w, st.a.w, st.b.y, st.b.y);
                s_st[3][t] = make_float4(st.b.z, z, st.b.w, st.b.w);
                s_st[4][t] = make_float4(st.c.x, st.c.x, st.c.y, st.c.y);
                s_st[5][t] = make_float4(st.c.z, st.c.z, 0.f, 0.f);
            }
            s_mask[t] = warp_block_mask<NW, BX, BH>(st, half, (float)sx, (float)sy);
        }
        __syncthreads();
        // this warp's list of splats whose 3-sigma box meets its block, in depth order
        int nlist = 0;
        for (int g0 = 0; g0 < cnt; g0 += 32) {
            const int k = g0 + lane;
            const bool in = k < cnt && ((s_mask[k] >> warp) & 1u);
            const uint32_t bal = __ballot_sync(0xffffffffu, in);
            if (in) s_list[warp][nlist + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)k;
            nlist += __popc(bal);
        }
        __syncwarp();
        if constexpr (PPT == 1) {
        for (int i = nlist - 1; i >= 0; --i) {     // back to front
            const int k = s_list[warp][i];
            const int64_t pos = lo + k;   // sorted position of this splat
            const float4 a = s_st[0][k], b = s_st[1][k], c = s_st[2][k];
            // this thread's gradient terms
            float g[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool contrib = false;
            const int q = 0;
            if (inside[q] && pos < (int64_t)last[q]) {
                const PairEval e = eval_pair(lx, ly[q], a, b);
                // the forward's decisions: 3-sigma cut and alpha_min (and the depth test)
                if (e.q <= b.z && (!DEPTH || c.w <= dl[q])) {
                    contrib = true;
                    const float G = gauss_of_qs(e.q);
                    const float raw = __fmul_rn(b.w, G);
                    const float alpha = fminf(alpha_max, raw);
                    const float om = __fsub_rn(1.f, alpha);
                    // 1 / (1 - alpha) with alpha <= alpha_max < 1: one approximate reciprocal
                    // (relative error ~1e-7 per splat, far inside the gradients' tolerance)
                    float inv_om;
                    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv_om) : "f"(om));
                    T[q] = T[q] * inv_om;                      // T before this splat
                    const float w = alpha * T[q];
                    g[6] = gC0[q] * w; g[7] = gC1[q] * w; g[8] = gC2[q] * w;
                    float ga = T[q] * ((c.x - S0[q]) * gC0[q] + (c.y - S1[q]) * gC1[q] + (c.z - S2[q]) * gC2[q]);
                    ga += aterm[q] * inv_om;
                    S0[q] = c.x * alpha + om * S0[q];
                    S1[q] = c.y * alpha + om * S1[q];
                    S2[q] = c.z * alpha + om * S2[q];
                    if (raw <= alpha_max) {   // clamp inactive
                        g[5] = ga * G;
                        // G = exp(-q/2) in the unscaled q = d^T S^-1 d: dL/dq = -ga opacity G / 2
                        const float gq = -0.5f * ga * raw;
                        // dq/dd = 2 S^-1 d = 2 (f1 p1 + f2 p2) / c for the scaled rows f, p, and
                        // d = pixel - (u, v): dL/du = -2 gq (f1 p1 + f2 p2)_x / c
                        const float gu = -2.f * inv_scale * gq;
                        g[0] = gu * (a.z * e.p1 + b.x * e.p2);
                        g[1] = gu * (a.w * e.p1 + b.y * e.p2);
                        const float gdx = gq * e.dx;
                        g[2] = gdx * e.dx;
                        g[3] = 2.f * gdx * e.dy;
                        g[4] = gq * e.dy * e.dy;
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) warp_add_gradients(g, lane, g2 + 9 * (size_t)s_g[k]);
        }
        } else {
        // Two vertically adjacent pixels per thread: the same arithmetic for both with packed
        // f32x2 instructions (the forward's decisions exactly as the forward takes them: q' is
        // the one-pixel rounding), branch-free over the pair -- a pixel that does not take the
        // splat gets alpha = 0 (T, S unchanged: 1 - 0 = 1 and reciprocal 1) and a zero term.
        // S is carried negated (nS = -S) so that c - S and the S update are pair adds and FMAs.
        const float2 lx2 = make_float2(lx, lx), ly2 = make_float2(ly[0], ly[PPT - 1]);
        const float2 one2 = make_float2(1.f, 1.f);
        float2 T2 = make_float2(T[0], T[PPT - 1]);
        float2 nR = make_float2(-S0[0], -S0[PPT - 1]), nG = make_float2(-S1[0], -S1[PPT - 1]),
               nB = make_float2(-S2[0], -S2[PPT - 1]);
        const float2 gR = make_float2(gC0[0], gC0[PPT - 1]), gG = make_float2(gC1[0], gC1[PPT - 1]),
                     gB = make_float2(gC2[0], gC2[PPT - 1]), at2 = make_float2(aterm[0], aterm[PPT - 1]);
        const float2 is2 = make_float2(inv_scale, inv_scale);
        for (int i = nlist - 1; i >= 0; --i) {     // back to front
            const int k = s_list[warp][i];
            const int64_t pos = lo + k;   // sorted position of this splat
            const float4 q0 = s_st[0][k], q1 = s_st[1][k], q2 = s_st[2][k], q3 = s_st[3][k];
            const float2 dx = __fadd2_rn(lx2, make_float2(q0.x, q0.y));
            const float2 dy = __fadd2_rn(ly2, make_float2(q0.z, q0.w));
            const float2 f1x = make_float2(q1.x, q1.y), f2x = make_float2(q1.z, q1.w);
            const float2 f1y = make_float2(q2.x, q2.y), f2y = make_float2(q2.z, q2.w);
            const float2 p1 = __ffma2_rn(dy, f1y, __fmul2_rn(dx, f1x));
            const float2 p2 = __ffma2_rn(dy, f2y, __fmul2_rn(dx, f2x));
            const float2 qq = __ffma2_rn(p2, p2, __fmul2_rn(p1, p1));
            const bool h0 = inside[0] && pos < (int64_t)last[0] && qq.x <= q3.x && (!DEPTH || q3.y <= dl[0]);
            const bool h1 = inside[PPT - 1] && pos < (int64_t)last[PPT - 1] && qq.y <= q3.x &&
                            (!DEPTH || q3.y <= dl[PPT - 1]);
            if (!__any_sync(0xffffffffu, h0 || h1)) continue;
            const float2 G = make_float2(gauss_of_qs(qq.x), gauss_of_qs(qq.y));
            const float2 raw = __fmul2_rn(make_float2(q3.z, q3.w), G);
            // -alpha (0 for a pixel that does not take the splat)
            const float2 na = make_float2(h0 ? fmaxf(-alpha_max, -raw.x) : 0.f, h1 ? fmaxf(-alpha_max, -raw.y) : 0.f);
            const float2 om = __fadd2_rn(one2, na);
            float r0, r1;
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(om.x));
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r1) : "f"(om.y));
            const float2 inv_om = make_float2(h0 ? r0 : 1.f, h1 ? r1 : 1.f);
            T2 = __fmul2_rn(T2, inv_om);                  // T before this splat
            const float2 nw = __fmul2_rn(na, T2);         // -alpha T
            const float4 k0 = s_st[4][k], k1 = s_st[5][k];
            const float2 cR = make_float2(k0.x, k0.y), cG = make_float2(k0.z, k0.w), cB = make_float2(k1.x, k1.y);
            // sum over the colours of (c - S) dL/dC, then the pixel's dL/dalpha
            const float2 e = __ffma2_rn(__fadd2_rn(cB, nB), gB,
                                        __ffma2_rn(__fadd2_rn(cG, nG), gG, __fmul2_rn(__fadd2_rn(cR, nR), gR)));
            const float2 ga = __ffma2_rn(at2, inv_om, __fmul2_rn(T2, e));
            nR = __ffma2_rn(cR, na, __fmul2_rn(om, nR));   // -S <- om (-S) - c alpha
            nG = __ffma2_rn(cG, na, __fmul2_rn(om, nG));
            nB = __ffma2_rn(cB, na, __fmul2_rn(om, nB));
            // clamp inactive and taking the splat: the conic, centre and opacity terms
            const float2 gam = make_float2(h0 && raw.x <= alpha_max ? ga.x : 0.f,
                                           h1 && raw.y <= alpha_max ? ga.y : 0.f);
            const float2 gr = __fmul2_rn(gam, raw);      // -2 dL/dq
            const float2 gu = __fmul2_rn(gr, is2);       // -2 inv_scale dL/dq
            const float2 qx = __ffma2_rn(f1x, p1, __fmul2_rn(f2x, p2));
            const float2 qy = __ffma2_rn(f1y, p1, __fmul2_rn(f2y, p2));
            const float2 t0 = __fmul2_rn(gu, qx), t1 = __fmul2_rn(gu, qy);
            const float2 gdx = __fmul2_rn(gr, dx), gdy = __fmul2_rn(gr, dy);
            const float2 t2 = __fmul2_rn(gdx, dx), t3 = __fmul2_rn(gdx, dy), t4 = __fmul2_rn(gdy, dy);
            const float2 t5 = __fmul2_rn(gam, G);
            const float2 t6 = __fmul2_rn(gR, nw), t7 = __fmul2_rn(gG, nw), t8 = __fmul2_rn(gB, nw);
            float g[9];
            g[0] = t0.x + t0.y;
            g[1] = t1.x + t1.y;
            g[2] = -0.5f * (t2.x + t2.y);
            g[3] = -(t3.x + t3.y);
            g[4] = -0.5f * (t4.x + t4.y);
            g[5] = t5.x + t5.y;
            g[6] = -(t6.x + t6.y);
            g[7] = -(t7.x + t7.y);
            g[8] = -(t8.x + t8.y);
            warp_add_gradients(g, lane, g2 + 9 * (size_t)s_g[k]);
        }
        T[0] = T2.x; T[PPT - 1] = T2.y;
        S0[0] = -nR.x; S0[PPT - 1] = -nR.y;
        S1[0] = -nG.x; S1[PPT - 1] = -nG.y;
        S2[0] = -nB.x; S2[PPT - 1] = -nB.y;
        }
    }
}

template <int DEG>
__global__ void __launch_bounds__(kPrepThreads)
preprocess_backward_kernel(PrepParams p, const float* __restrict__ g2, const uint32_t* __restrict__ touched,
                           float* __restrict__ d_means, float* __restrict__ d_log_scales,
                           float* __restrict__ d_quats, float* __restrict__ d_logits, float* __restrict__ d_sh) {
    pdl_entry();
    // i: the Gaussian in the scene's arrays; gi: its workspace slot (multi-scene renders)
    const int i = blockIdx.x * kPrepThreads + threadIdx.x;
    if (i >= p.n) return;
    const int64_t gi = p.index_offset + i;
    constexpr int K = (DEG + 1) * (DEG + 1);
    float* dsh = d_sh + (size_t)i * K * 3;
    if (touched[gi] == 0) {
        for (int k = 0; k < 3; ++k) { d_means[3 * i + k] = 0.f; d_log_scales[3 * i + k] = 0.f; }
        for (int k = 0; k < 4; ++k) d_quats[4 * i + k] = 0.f;
        d_logits[i] = 0.f;
        for (int k = 0; k < 3 * K; ++k) dsh[k] = 0.f;
        return;
    }
    float gg[9];
#pragma unroll
    for (int f = 0; f < 9; ++f) gg[f] = g2[9 * (size_t)gi + f];
    const float mx = p.means[3 * i], my = p.means[3 * i + 1], mz = p.means[3 * i + 2];

    // ---- colour: rgb_c = max(0, sum_k sh_kc Y_k(dir) + 0.5) ----
    float vx = mx - p.cam_pos[0], vy = my - p.cam_pos[1], vz = mz - p.cam_pos[2];
    const float vinv = rsqrtf(vx * vx + vy * vy + vz * vz);
    const float x = vx * vinv, y = vy * vinv, z = vz * vinv;
    const float* c = p.shc;
    float Y[16], Yx[16], Yy[16], Yz[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) { Y[k] = 0.f; Yx[k] = 0.f; Yy[k] = 0.f; Yz[k] = 0.f; }
    Y[0] = c[9];
    if (DEG >= 1) {
        Y[1] = -c[1] * y; Yy[1] = -c[1];
        Y[2] = c[0] * z;  Yz[2] = c[0];
        Y[3] = -c[1] * x; Yx[3] = -c[1];
    }
    if (DEG >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = 2.f * c[4] * x * y;       Yx[4] = 2.f * c[4] * y;  Yy[4] = 2.f * c[4] * x;
        Y[5] = -c[3] * y * z;            Yy[5] = -c[3] * z;       Yz[5] = -c[3] * y;
        Y[6] = c[2] * (3.f * zz - 1.f);  Yz[6] = 6.f * c[2] * z;
        Y[7] = -c[3] * x * z;            Yx[7] = -c[3] * z;       Yz[7] = -c[3] * x;
        Y[8] = c[4] * (xx - yy);         Yx[8] = 2.f * c[4] * x;  Yy[8] = -2.f * c[4] * y;
        if (DEG >= 3) {
            Y[9] = -c[8] * (3.f * xx * y - yy * y);
            Yx[9] = -6.f * c[8] * x * y;     Yy[9] = -c[8] * (3.f * xx - 3.f * yy);
            Y[10] = 2.f * c[7] * x * y * z;
            Yx[10] = 2.f * c[7] * y * z;     Yy[10] = 2.f * c[7] * x * z;  Yz[10] = 2.f * c[7] * x * y;
            Y[11] = -c[6] * (5.f * zz - 1.f) * y;
            Yy[11] = -c[6] * (5.f * zz - 1.f); Yz[11] = -10.f * c[6] * z * y;
            Y[12] = c[5] * (5.f * zz * z - 3.f * z);
            Yz[12] = c[5] * (15.f * zz - 3.f);
            Y[13] = -c[6] * (5.f * zz - 1.f) * x;
            Yx[13] = -c[6] * (5.f * zz - 1.f); Yz[13] = -10.f * c[6] * z * x;
            Y[14] = c[7] * z * (xx - yy);
            Yx[14] = 2.f * c[7] * x * z;     Yy[14] = -2.f * c[7] * y * z;  Yz[14] = c[7] * (xx - yy);
            Y[15] = -c[8] * (xx * x - 3.f * x * yy);
            Yx[15] = -c[8] * (3.f * xx - 3.f * yy); Yy[15] = 6.f * c[8] * x * y;
        }
    }
    const float* shi = p.sh + (size_t)i * K * 3;
    float shv[3 * K];
    if (K * 3 % 4 == 0) {   // 16-byte rows (degrees 1 and 3): vector loads
#pragma unroll
        for (int k = 0; k < 3 * K / 4; ++k) {
            const float4 w4 = __ldg(reinterpret_cast<const float4*>(shi) + k);
            shv[4 * k] = w4.x; shv[4 * k + 1] = w4.y; shv[4 * k + 2] = w4.z; shv[4 * k + 3] = w4.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 3 * K; ++k) shv[k] = __ldg(shi + k);
    }
    float gdx = 0.f, gdy = 0.f, gdz = 0.f;
    float dshv[3 * K];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float col = 0.5f;
#pragma unroll
        for (int k = 0; k < K; ++k) col += shv[3 * k + ch] * Y[k];
        const float gch = (col < 0.f) ? 0.f : gg[6 + ch];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            dshv[3 * k + ch] = gch * Y[k];
            const float sv = shv[3 * k + ch] * gch;
            gdx += sv * Yx[k]; gdy += sv * Yy[k]; gdz += sv * Yz[k];
        }
    }
    if (K * 3 % 4 == 0) {
#pragma unroll
        for (int k = 0; k < 3 * K / 4; ++k)
            reinterpret_cast<float4*>(dsh)[k] = make_float4(dshv[4 * k], dshv[4 * k + 1], dshv[4 * k + 2], dshv[4 * k + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < 3 * K; ++k) dsh[k] = dshv[k];
    }
    const float dd = gdx * x + gdy * y + gdz * z;
    float gmx = (gdx - x * dd) * vinv, gmy = (gdy - y * dd) * vinv, gmz = (gdz - z * dd) * vinv;

    // ---- opacity ----
    const float opac = 1.f / (1.f + __expf(-p.logits[i]));
    d_logits[i] = gg[5] * opac * (1.f - opac);

    // ---- camera-space position (float is enough for gradients) ----
    float pc[3];
#pragma unroll
    for (int rr = 0; rr < 3; ++rr) pc[rr] = p.R[3 * rr] * mx + p.R[3 * rr + 1] * my + p.R[3 * rr + 2] * mz + p.t[rr];
    const float zc = pc[2], zi = 1.f / zc;
    const float rx = pc[0] * zi, ry = pc[1] * zi;
    float gp0 = gg[0] * p.fx * zi, gp1 = gg[1] * p.fy * zi;
    float gp2 = -(gg[0] * p.fx * rx + gg[1] * p.fy * ry) * zi;

    // ---- recompute A = J W M and S ----
    const float4 q4 = *reinterpret_cast<const float4*>(p.quats + 4 * (size_t)i);
    const float qn2 = q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w;
    const bool qdeg = qn2 < 1e-24f;
    const float qinv = qdeg ? 0.f : rsqrtf(qn2);
    const float qw = qdeg ? 1.f : q4.x * qinv, qx = q4.y * qinv, qy = q4.z * qinv, qz = q4.w * qinv;
    const float Rq[9] = {
        1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
        2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
        2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
    const float sk[3] = {__expf(p.log_scales[3 * i]), __expf(p.log_scales[3 * i + 1]),
                         __expf(p.log_scales[3 * i + 2])};
    const bool clx = rx > p.limx || rx < -p.limx, cly = ry > p.limy || ry < -p.limy;
    const float txc = fminf(p.limx, fmaxf(-p.limx, rx)), tyc = fminf(p.limy, fmaxf(-p.limy, ry));
    const float J00 = p.fx * zi, J02 = -p.fx * txc * zi, J11 = p.fy * zi, J12 = -p.fy * tyc * zi;
    float Tm[2][3];
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
        Tm[0][cc] = J00 * p.R[cc] + J02 * p.R[6 + cc];
        Tm[1][cc] = J11 * p.R[3 + cc] + J12 * p.R[6 + cc];
    }
    float M[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) M[a][k] = Rq[3 * a + k] * sk[k];
    float A[2][3];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int k = 0; k < 3; ++k) A[rr][k] = Tm[rr][0] * M[0][k] + Tm[rr][1] * M[1][k] + Tm[rr][2] * M[2][k];
    const float s00 = A[0][0] * A[0][0] + A[0][1] * A[0][1] + A[0][2] * A[0][2] + p.dilation;
    const float s11 = A[1][0] * A[1][0] + A[1][1] * A[1][1] + A[1][2] * A[1][2] + p.dilation;
    const float s01 = A[0][0] * A[1][0] + A[0][1] * A[1][1] + A[0][2] * A[1][2];
    const float det = s00 * s11 - s01 * s01;
    const float idet = 1.f / det;
    const float Qa = s11 * idet, Qb = -s01 * idet, Qc = s00 * idet;

    // ---- conic -> S: G_S = -Q Gbar Q, Gbar = [[ga, gb/2], [gb/2, gc]] ----
    const float Gb00 = gg[2], Gb01 = 0.5f * gg[3], Gb11 = gg[4];
    const float QG00 = Qa * Gb00 + Qb * Gb01, QG01 = Qa * Gb01 + Qb * Gb11;
    const float QG10 = Qb * Gb00 + Qc * Gb01, QG11 = Qb * Gb01 + Qc * Gb11;
    const float GS00 = -(QG00 * Qa + QG01 * Qb);
    const float GS01 = -(QG00 * Qb + QG01 * Qc);
    const float GS11 = -(QG10 * Qb + QG11 * Qc);
    // ---- S = A A^T + dil I: dL/dA = 2 G_S A ----
    float gA_[2][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        gA_[0][k] = 2.f * (GS00 * A[0][k] + GS01 * A[1][k]);
        gA_[1][k] = 2.f * (GS01 * A[0][k] + GS11 * A[1][k]);
    }
    // ---- A = T M: dL/dT = dL/dA M^T, dL/dM = T^T dL/dA ----
    float gT[2][3], gM[3][3];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int a = 0; a < 3; ++a) gT[rr][a] = gA_[rr][0] * M[a][0] + gA_[rr][1] * M[a][1] + gA_[rr][2] * M[a][2];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) gM[a][k] = Tm[0][a] * gA_[0][k] + Tm[1][a] * gA_[1][k];
    // ---- T = J W: dL/dJ = dL/dT W^T (only J00, J02, J11, J12 are non-zero) ----
    const float gJ00 = gT[0][0] * p.R[0] + gT[0][1] * p.R[1] + gT[0][2] * p.R[2];
    const float gJ02 = gT[0][0] * p.R[6] + gT[0][1] * p.R[7] + gT[0][2] * p.R[8];
    const float gJ11 = gT[1][0] * p.R[3] + gT[1][1] * p.R[4] + gT[1][2] * p.R[5];
    const float gJ12 = gT[1][0] * p.R[6] + gT[1][1] * p.R[7] + gT[1][2] * p.R[8];
    const float zi2 = zi * zi;
    gp2 += -gJ00 * p.fx * zi2 - gJ11 * p.fy * zi2 + gJ02 * p.fx * txc * zi2 + gJ12 * p.fy * tyc * zi2;
    if (!clx) { gp0 += -gJ02 * p.fx * zi2; gp2 += gJ02 * p.fx * rx * zi2; }
    if (!cly) { gp1 += -gJ12 * p.fy * zi2; gp2 += gJ12 * p.fy * ry * zi2; }
    // ---- p = R mu + t ----
    gmx += p.R[0] * gp0 + p.R[3] * gp1 + p.R[6] * gp2;
    gmy += p.R[1] * gp0 + p.R[4] * gp1 + p.R[7] * gp2;
    gmz += p.R[2] * gp0 + p.R[5] * gp1 + p.R[8] * gp2;
    d_means[3 * i] = gmx; d_means[3 * i + 1] = gmy; d_means[3 * i + 2] = gmz;
    // ---- M = Rq diag(s) ----
    float gR[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float gs = gM[0][k] * Rq[k] + gM[1][k] * Rq[3 + k] + gM[2][k] * Rq[6 + k];
        d_log_scales[3 * i + k] = gs * sk[k];
#pragma unroll
        for (int a = 0; a < 3; ++a) gR[3 * a + k] = gM[a][k] * sk[k];
    }
    // ---- Rq(qhat) -> qhat -> q ----
    float gw = -2.f * qz * gR[1] + 2.f * qy * gR[2] + 2.f * qz * gR[3] - 2.f * qx * gR[5] - 2.f * qy * gR[6] + 2.f * qx * gR[7];
    float gx = 2.f * qy * gR[1] + 2.f * qz * gR[2] + 2.f * qy * gR[3] - 4.f * qx * gR[4] - 2.f * qw * gR[5] + 2.f * qz * gR[6] + 2.f * qw * gR[7] - 4.f * qx * gR[8];
    float gy = -4.f * qy * gR[0] + 2.f * qx * gR[1] + 2.f * qw * gR[2] + 2.f * qx * gR[3] + 2.f * qz * gR[5] - 2.f * qw * gR[6] + 2.f * qz * gR[7] - 4.f * qy * gR[8];
    float gz = -4.f * qz * gR[0] - 2.f * qw * gR[1] + 2.f * qx * gR[2] + 2.f * qw * gR[3] - 4.f * qz * gR[4] + 2.f * qy * gR[5] + 2.f * qx * gR[6] + 2.f * qy * gR[7];
    if (qdeg) { gw = gx = gy = gz = 0.f; }
    const float dq = gw * qw + gx * qx + gy * qy + gz * qz;
    d_quats[4 * i + 0] = (gw - qw * dq) * qinv;
    d_quats[4 * i + 1] = (gx - qx * dq) * qinv;
    d_quats[4 * i + 2] = (gy - qy * dq) * qinv;
    d_quats[4 * i + 3] = (gz - qz * dq) * qinv;
}

void launch_composite_backward(const Layout& L, char* ws, const float bg[3], float alpha_min, float alpha_max,
                               int ppt, const float* d_rgb, const float* d_alpha, const float* zlim,
                               cudaStream_t stream) {
    float* g2 = reinterpret_cast<float*>(ws + L.off_g2);
    cudaMemsetAsync(g2, 0, sizeof(float) * 9 * (size_t)L.n, stream);
    const uint2* ranges = reinterpret_cast<const uint2*>(ws + L.off_ranges);
    const uint32_t* vals = reinterpret_cast<const uint32_t*>(ws + L.off_vals[L.sorted_buffer]);
    const float4* rec = reinterpret_cast<const float4*>(ws + L.off_rec);
    const float* tfin = reinterpret_cast<const float*>(ws + L.off_tfinal);
    const int32_t* last = reinterpret_cast<const int32_t*>(ws + L.off_last);
    const int blocks = (int)L.ntiles;
    const QScale qs = q_scale();
    const float* depth = reinterpret_cast<const float*>(ws + L.off_depth);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.off_ctrl);
    const uint32_t* order = L.tile_fused ? reinterpret_cast<const uint32_t*>(ws + L.off_order) : nullptr;
    // 16 x 16 squares at most per CTA, as the forward compositor
#define VIS_LAUNCH_BWD_D(TS, PP, DT)                                                                           \
    composite_backward_kernel<TS, (TS < 16 ? TS : 16), PP, DT>                                                 \
        <<<blocks * (TS / (TS < 16 ? TS : 16)) * (TS / (TS < 16 ? TS : 16)), (TS < 16 ? TS : 16) * (TS < 16 ? TS : 16) / PP, \
           0, stream>>>(ranges, vals, rec, L.W, L.H, L.tiles_x, bg[0], bg[1], bg[2], alpha_min, alpha_max, qs.qcut, \
                        qs.inv_scale, tfin, last, d_rgb, d_alpha, g2, depth, zlim, ctrl, order)
#define VIS_LAUNCH_BWD(TS, PP)                       \
    do {                                             \
        if (zlim) VIS_LAUNCH_BWD_D(TS, PP, true);    \
        else VIS_LAUNCH_BWD_D(TS, PP, false);        \
    } while (0)
    if (blocks > 0) {
        const bool two = ppt == 2;
        if (L.tile == 8) { if (two) VIS_LAUNCH_BWD(8, 2); else VIS_LAUNCH_BWD(8, 1); }
        else if (L.tile == 32) { if (two) VIS_LAUNCH_BWD(32, 2); else VIS_LAUNCH_BWD(32, 1); }
        else { if (two) VIS_LAUNCH_BWD(16, 2); else VIS_LAUNCH_BWD(16, 1); }
    }
#undef VIS_LAUNCH_BWD_D
#undef VIS_LAUNCH_BWD
}

void launch_preprocess_backward(const PrepParams& p, const Layout& L, const char* ws, float* d_means,
                                float* d_log_scales, float* d_quats, float* d_logits, float* d_sh,
                                cudaStream_t stream) {
    const float* g2 = reinterpret_cast<const float*>(ws + L.off_g2);
    if (p.n > 0) {
        const uint32_t* touched = reinterpret_cast<const uint32_t*>(ws + L.off_touched);
        const int blocks = (p.n + kPrepThreads - 1) / kPrepThreads;
#define VIS_LAUNCH_PBWD(D)                                                                                \
    launch_k(true, preprocess_backward_kernel<D>, blocks, kPrepThreads, 0, stream, p, g2, touched, d_means,      \
             d_log_scales, d_quats, d_logits, d_sh)
        if (p.deg == 0) VIS_LAUNCH_PBWD(0);
        else if (p.deg == 1) VIS_LAUNCH_PBWD(1);
        else if (p.deg == 2) VIS_LAUNCH_PBWD(2);
        else VIS_LAUNCH_PBWD(3);
#undef VIS_LAUNCH_PBWD
    }
}

}  // namespace vis
