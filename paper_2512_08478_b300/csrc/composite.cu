// K5 -- tile compositor (section 3.2 Eqs. 2-3, front to back).
//
// One CTA per SUB x SUB square of a TILE x TILE tile (the whole tile up to 16 pixels, a
// quarter of a 32-pixel tile); each thread owns PPT vertically adjacent pixels and each warp
// an 8 x (4 PPT) pixel block. With PPT = 2 the two pixels are evaluated and
// composited together with packed f32x2 arithmetic (one instruction for both pixels' add,
// multiply or FMA), rounded exactly as the one-pixel code, so the image does not depend on PPT.
// The tile's range of the sorted (tile, depth, index) list is walked in chunks of
// CH splats: each thread stages splats (gather of the 48-byte record by index)
// into shared memory -- centre relative to the tile centre, scaled whitening rows,
// and one threshold for the 3-sigma cut and the alpha_min skip -- then every
// warp builds (ballot compaction) the list of staged splats whose exact 3-sigma
// bounding box meets its pixel block, and composites only those for its pixels,
// from shared memory (broadcast reads).
// A splat that misses costs two shared loads and ~10 FP32 operations; only hits
// evaluate 2^-q'. A pixel is done when T (1 - alpha) would fall below t_stop
// (that splat excluded); the CTA leaves as soon as all its pixels are done.
// Outputs: planar rgb = C + T bg, alpha = 1 - T, and for the adjoint the final T
// and 1 + the sorted position of the last composited splat.
// DEPTH: depth-buffer-aware compositing (section 3.4's depth test against a caller's
// buffer, without writing it): a splat whose view depth exceeds the pixel's value in
// zlim [H,W] is not composited at that pixel. A warp block's list leaves out the splats
// deeper than all of its pixels' limits, and since a tile's list is in depth order the tile
// stops at the first chunk that ends beyond every limit in the tile (behind a wall nothing
// is walked).
#include "splat_eval.cuh"

namespace vis {

struct PixAcc {
    float T, C0, C1, C2;
    int32_t last;
    bool done;
};

// Composite one staged splat into one pixel; returns false when the pixel stops.
// The colour weight alpha T of Eq. 3 is taken as the drop in transmittance, T - T (1 - alpha):
// the same quantity, and the weights of a pixel then add up to 1 - T to within one rounding each.
__device__ __forceinline__ void composite_hit(PixAcc& P, float q, const float4& b, const float4& c, float alpha_max,
                                              float t_stop, int32_t pos1) {
    const float alpha = fminf(alpha_max, __fmul_rn(b.w, gauss_of_qs(q)));
    const float Tn = __fmul_rn(P.T, __fsub_rn(1.f, alpha));
    if (Tn < t_stop) { P.done = true; return; }
    const float w = __fsub_rn(P.T, Tn);
    P.C0 = __fmaf_rn(c.x, w, P.C0);
    P.C1 = __fmaf_rn(c.y, w, P.C1);
    P.C2 = __fmaf_rn(c.z, w, P.C2);
    P.T = Tn;
    P.last = pos1;
}

template <int TILE, int SUB, int PPT, bool STATS, bool DEPTH, bool BATCH>
__global__ void __launch_bounds__(SUB * SUB / PPT)
composite_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                 const float4* __restrict__ rec, int W, int H, int tiles_x, float bg0, float bg1,
                 float bg2, float alpha_min, float alpha_max, float t_stop, float qcut,
                 Ctrl* __restrict__ ctrl, float* __restrict__ out_rgb, float* __restrict__ out_alpha,
                 float* __restrict__ t_final, int32_t* __restrict__ last_out,
                 const float* __restrict__ depth, const float* __restrict__ zlim,
                 const BatchImage* __restrict__ images, int n_images, const uint32_t* __restrict__ order) {
    pdl_entry();
    // a CTA composites one SUB x SUB square of its TILE x TILE tile (the tile's whole list,
    // each warp its own block of the square): NSUB CTAs per tile
    static_assert(TILE % SUB == 0, "the squares tile the tile");
    constexpr int NSUB = (TILE / SUB) * (TILE / SUB);
    constexpr int NT = SUB * SUB / PPT;     // threads
    constexpr int NW = NT / 32;             // warps; each owns an 8 x (4 PPT) pixel block
    constexpr int BX = SUB / 8;             // blocks per row of the square
    constexpr int BH = 4 * PPT;             // block height in pixels
    // splats staged per chunk: one per thread, up to 256 (512 for a 512-thread square of
    // two pixels per thread: half the chunk barriers)
    constexpr int CHMAX = PPT == 2 ? 512 : 256;
    constexpr int CH = NT < CHMAX ? NT : CHMAX;
    static_assert(NW == BX * (SUB / BH), "warp blocks tile the square");
    // staged splats, NS float4 slots each: PPT 1 -> (du, dv, f1x, f1y), (f2x, f2y, thr, opacity),
    // (r, g, b, depth); PPT 2 -> the same values laid out as packed pairs for the f32x2
    // instructions (see the pair walk below)
    constexpr int NS = PPT == 1 ? 3 : 6;
    __shared__ float4 s_st[NS][CH];
    __shared__ uint32_t s_mask[CH];
    __shared__ uint16_t s_list[NW][CH];
    __shared__ float s_wmax[NW];   // DEPTH: largest depth limit of each warp block's live pixels
    // the tile's index in `ranges`: CTAs take the tiles longest first when an order is given
    const uint32_t gtile = order ? order[blockIdx.x / NSUB] : blockIdx.x / NSUB;
    const int sub = (int)(blockIdx.x % NSUB);
    const int sx = (sub % (TILE / SUB)) * SUB, sy = (sub / (TILE / SUB)) * SUB;   // the square in the tile
    int tile = (int)gtile;
    if (BATCH) {
        // a batch group's canvas (tiles_x tiles wide) stacks its images' tile rows: find this
        // tile's image (the last whose first tile is <= gtile) and take its size and outputs; a
        // canvas tile right of a narrower image has no pixels
        int lo = 0, hi = n_images - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (images[mid].tile0 <= gtile) lo = mid; else hi = mid - 1;
        }
        const BatchImage im = images[lo];
        const int t = (int)(gtile - im.tile0), cx = t % tiles_x, cy = t / tiles_x;
        if (cx >= im.tiles_x) return;
        tile = cy * im.tiles_x + cx;
        W = im.W; H = im.H; tiles_x = im.tiles_x;
        out_rgb = im.out_rgb; out_alpha = im.out_alpha;
    }
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int bx = warp % BX, by = warp / BX;
    const int col = sx + bx * 8 + (lane & 7), row0 = sy + by * BH + (lane >> 3) * PPT;
    const int px = tx * TILE + col;
    const float half = 0.5f * TILE;
    const float xc = (float)(tx * TILE) + half, yc = (float)(ty * TILE) + half;
    const float lx = (float)px + 0.5f - xc;
    const size_t HW = (size_t)H * W;
    if (ctrl->error) {   // keys were not produced: make the failure visible
        const float nan = __int_as_float(0x7fc00000);
        for (int r = 0; r < PPT; ++r) {
            const int py = ty * TILE + row0 + r;
            if (px < W && py < H) {
                const size_t pix = (size_t)py * W + px;
                out_rgb[pix] = nan; out_rgb[HW + pix] = nan; out_rgb[2 * HW + pix] = nan;
                out_alpha[pix] = nan;
                if (!BATCH) { t_final[pix] = nan; last_out[pix] = 0; }
            }
        }
        return;
    }
    PixAcc P[PPT];
    float ly[PPT];
    float dl[PPT];   // depth limits (DEPTH only)
    unsigned long long n_tests = 0, n_hits = 0;
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
        const int py = ty * TILE + row0 + r;
        P[r].T = 1.f; P[r].C0 = P[r].C1 = P[r].C2 = 0.f; P[r].last = 0;
        P[r].done = !(px < W && py < H);
        ly[r] = (float)py + 0.5f - yc;
        dl[r] = (DEPTH && !P[r].done) ? zlim[(size_t)py * W + px] : __int_as_float(0x7f800000);
    }
    // PPT 2: the two pixels' state as packed pairs (x: row0, y: row0 + 1)
    float2 T2 = make_float2(1.f, 1.f), Cr = make_float2(0.f, 0.f), Cg = Cr, Cb = Cr;
    const float2 lx2 = make_float2(lx, lx), ly2 = make_float2(ly[0], ly[PPT - 1]), one2 = T2;
    if (DEPTH) {   // a NaN limit rejects nothing (no comparison holds): it counts as +inf here
        float m = __int_as_float(0xff800000);
#pragma unroll
        for (int r = 0; r < PPT; ++r)
            if (!P[r].done) m = fmaxf(m, isnan(dl[r]) ? __int_as_float(0x7f800000) : dl[r]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s_wmax[warp] = m;
    }
    const uint2 rg = ranges[gtile];
    for (uint32_t base = rg.x; base < rg.y; base += CH) {
        bool all_done = true;
#pragma unroll
        for (int r = 0; r < PPT; ++r) all_done = all_done && P[r].done;
        if (__syncthreads_count(all_done) == NT) break;
        for (int t = threadIdx.x; t < CH && base + t < rg.y; t += NT) {
            const uint32_t g = vals[base + t];
            const StagedSplat s = stage_splat(rec, g, xc, yc, qcut, alpha_min);
            const float z = DEPTH ? depth[g] : 0.f;
            if constexpr (PPT == 1) {
                s_st[0][t] = s.a;
                s_st[1][t] = s.b;
                s_st[2][t] = make_float4(s.c.x, s.c.y, s.c.z, z);
            } else {
                // negated centre and colour, so that a pair add and a pair FMA give dx, dy and
                // C + c w exactly as the single-pixel arithmetic does
                s_st[0][t] = make_float4(-s.a.x, -s.a.x, -s.a.y, -s.a.y);
                s_st[1][t] = make_float4(s.a.z, s.a.z, s.b.x, s.b.x);
                s_st[2][t] = make_float4(s.a.w, s.a.w, s.b.y, s.b.y);
                s_st[3][t] = make_float4(s.b.z, z, s.b.w, s.b.w);
                s_st[4][t] = make_float4(-s.c.x, -s.c.x, -s.c.y, -s.c.y);
                s_st[5][t] = make_float4(-s.c.z, -s.c.z, 0.f, 0.f);
            }
            uint32_t m = warp_block_mask<NW, BX, BH>(s, half, (float)sx, (float)sy);
            if (DEPTH) {
#pragma unroll
                for (int w = 0; w < NW; ++w)
                    if (!(z <= s_wmax[w])) m &= ~(1u << w);
            }
            s_mask[t] = m;
        }
        __syncthreads();
        const int cnt = (int)umin((uint32_t)CH, rg.y - base);
        bool beyond = false;   // DEPTH: this chunk ends deeper than every limit in the tile
        if (DEPTH) {
            float tmax = s_wmax[0];
#pragma unroll
            for (int w = 1; w < NW; ++w) tmax = fmaxf(tmax, s_wmax[w]);
            beyond = !((PPT == 1 ? s_st[2][cnt - 1].w : s_st[3][cnt - 1].y) <= tmax);
        }
        // this warp's list of splats whose 3-sigma box meets its pixel block, in depth order
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
            if (!all_done) {
                for (int i = 0; i < nlist; ++i) {
                    const int k = s_list[warp][i];
                    const float4 a = s_st[0][k], b = s_st[1][k];
                    const int32_t pos1 = (int32_t)(base + k + 1);
                    const PairEval e = eval_pair(lx, ly[0], a, b);
                    if (STATS) ++n_tests;
                    if (e.q > b.z) continue;
                    const float4 c = s_st[2][k];
                    if (DEPTH && c.w > dl[0]) continue;
                    composite_hit(P[0], e.q, b, c, alpha_max, t_stop, pos1);
                    if (STATS && !P[0].done) ++n_hits;
                    if (P[0].done) break;
                }
            }
        } else if (__any_sync(0xffffffffu, !all_done)) {
            // Two vertically adjacent pixels per thread, evaluated together with the packed
            // f32x2 instructions: per staged splat the eval_pair arithmetic (dx, dy, the two
            // whitened projections, q') and the composite_hit update (alpha, T, C) for both
            // pixels, each lane of a pair rounded exactly as the single-pixel code rounds it.
            // The update is branch-free: a pixel that does not take the splat gets w = 0 and
            // keeps T. The warp walks its list together and leaves once none of its pixels is live.
            bool live0 = !P[0].done, live1 = !P[PPT - 1].done;
            int lk0 = -1, lk1 = -1;   // chunk slot of each pixel's last composited splat
            const float2 mone2 = make_float2(-1.f, -1.f);
            for (int i = 0; i < nlist; ++i) {
                const int k = s_list[warp][i];
                const float4 q0 = s_st[0][k], q1 = s_st[1][k], q2 = s_st[2][k], q3 = s_st[3][k];
                const float2 dx = __fadd2_rn(lx2, make_float2(q0.x, q0.y));
                const float2 dy = __fadd2_rn(ly2, make_float2(q0.z, q0.w));
                const float2 t1 = __fmul2_rn(dx, make_float2(q1.x, q1.y));
                const float2 t2 = __fmul2_rn(dx, make_float2(q1.z, q1.w));
                const float2 p1 = __ffma2_rn(dy, make_float2(q2.x, q2.y), t1);
                const float2 p2 = __ffma2_rn(dy, make_float2(q2.z, q2.w), t2);
                const float2 q = __ffma2_rn(p2, p2, __fmul2_rn(p1, p1));
                bool h0 = live0 && q.x <= q3.x, h1 = live1 && q.y <= q3.x;
                if (DEPTH) { h0 = h0 && q3.y <= dl[0]; h1 = h1 && q3.y <= dl[1]; }
                if (STATS) n_tests += (live0 ? 1 : 0) + (live1 ? 1 : 0);
                // -alpha = max(-alpha_max, -(opacity 2^-q'))
                const float2 a = __fmul2_rn(make_float2(q3.z, q3.w), make_float2(gauss_of_qs(q.x), gauss_of_qs(q.y)));
                const float2 na = make_float2(fmaxf(-alpha_max, -a.x), fmaxf(-alpha_max, -a.y));
                const float2 Tn = __fmul2_rn(T2, __fadd2_rn(one2, na));
                const bool s0 = h0 && Tn.x < t_stop, s1 = h1 && Tn.y < t_stop;   // stops, splat excluded
                const bool c0 = h0 && !s0, c1 = h1 && !s1;                       // composited
                const float2 T2n = make_float2(c0 ? Tn.x : T2.x, c1 ? Tn.y : T2.y);
                // -(T - T'): the negated weight of the one-pixel code (one rounding, exact
                // negation), and +0 for a pixel that keeps T
                const float2 nw = __ffma2_rn(T2, mone2, T2n);
                const float4 k0 = s_st[4][k], k1 = s_st[5][k];
                Cr = __ffma2_rn(make_float2(k0.x, k0.y), nw, Cr);
                Cg = __ffma2_rn(make_float2(k0.z, k0.w), nw, Cg);
                Cb = __ffma2_rn(make_float2(k1.x, k1.y), nw, Cb);
                T2 = T2n;
                if (c0) lk0 = k;
                if (c1) lk1 = k;
                if (STATS) n_hits += (c0 ? 1 : 0) + (c1 ? 1 : 0);
                live0 = live0 && !s0;
                live1 = live1 && !s1;
                if (!__any_sync(0xffffffffu, live0 || live1)) break;
            }
            if (lk0 >= 0) P[0].last = (int32_t)(base + lk0 + 1);
            if (lk1 >= 0) P[PPT - 1].last = (int32_t)(base + lk1 + 1);
            P[0].done = !live0;
            P[PPT - 1].done = !live1;
        }
        if (DEPTH && beyond) break;   // every later splat of the tile is deeper still
    }
    if (STATS) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            n_tests += __shfl_xor_sync(0xffffffffu, n_tests, o);
            n_hits += __shfl_xor_sync(0xffffffffu, n_hits, o);
        }
        if (lane == 0) {
            atomicAdd(&ctrl->pair_tests, n_tests);
            atomicAdd(&ctrl->hits, n_hits);
        }
    }
    if constexpr (PPT == 2) {
        P[0].T = T2.x; P[0].C0 = Cr.x; P[0].C1 = Cg.x; P[0].C2 = Cb.x;
        P[PPT - 1].T = T2.y; P[PPT - 1].C0 = Cr.y; P[PPT - 1].C1 = Cg.y; P[PPT - 1].C2 = Cb.y;
    }
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
        const int py = ty * TILE + row0 + r;
        if (px < W && py < H) {
            const size_t pix = (size_t)py * W + px;
            out_rgb[pix] = __fmaf_rn(P[r].T, bg0, P[r].C0);
            out_rgb[HW + pix] = __fmaf_rn(P[r].T, bg1, P[r].C1);
            out_rgb[2 * HW + pix] = __fmaf_rn(P[r].T, bg2, P[r].C2);
            out_alpha[pix] = 1.f - P[r].T;
            if (!BATCH) {   // the adjoint's inputs (a batch is forward only)
                t_final[pix] = P[r].T;
                last_out[pix] = P[r].last;
            }
        }
    }
}

// Edge of the square a compositor CTA covers: 16 pixels at most, so that a 32-pixel tile (whose
// sort lists half the copies of 16-pixel tiles) is composited by four CTAs of four warps, each
// walking the whole tile's list, instead of one CTA of sixteen warps (which fit two to an SM
// and wait on each other at every chunk).
constexpr int kCompositeSub = 16;
constexpr int sub_of(int tile) { return tile < kCompositeSub ? tile : kCompositeSub; }

void launch_composite(const Layout& L, char* ws, float bg0, float bg1, float bg2, float alpha_min,
                      float alpha_max, float t_stop, int ppt, bool stats, float* out_rgb, float* out_alpha,
                      const float* zlim, cudaStream_t stream) {
    const uint2* ranges = reinterpret_cast<const uint2*>(ws + L.off_ranges);
    const uint32_t* vals = reinterpret_cast<const uint32_t*>(ws + L.off_vals[L.sorted_buffer]);
    const float4* rec = reinterpret_cast<const float4*>(ws + L.off_rec);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.off_ctrl);
    float* tfin = reinterpret_cast<float*>(ws + L.off_tfinal);
    int32_t* last = reinterpret_cast<int32_t*>(ws + L.off_last);
    const int blocks = (int)L.ntiles;
    if (blocks <= 0) return;
    const float qcut = q_scale().qcut;
    const float* depth = reinterpret_cast<const float*>(ws + L.off_depth);
    const uint32_t* order = L.tile_fused ? reinterpret_cast<const uint32_t*>(ws + L.off_order) : nullptr;
    // a 32-pixel tile is composited by four CTAs of 16 x 16 pixels (kCompositeSub)
#define VIS_LAUNCH_COMPOSITE_S(TS, PP, ST, DT)                                                                 \
    launch_k(true, composite_kernel<TS, sub_of(TS), PP, ST, DT, false>, blocks * (TS / sub_of(TS)) * (TS / sub_of(TS)), \
             sub_of(TS) * sub_of(TS) / PP, 0, stream, ranges, vals, rec, L.W, L.H, L.tiles_x, bg0, bg1, bg2,       \
             alpha_min, alpha_max, t_stop, qcut, ctrl, out_rgb, out_alpha, tfin, last, depth, zlim,               \
             (const BatchImage*)nullptr, 0, order)
#define VIS_LAUNCH_COMPOSITE(TS, PP)                          \
    do {                                                      \
        if (zlim) VIS_LAUNCH_COMPOSITE_S(TS, PP, false, true);   \
        else if (stats) VIS_LAUNCH_COMPOSITE_S(TS, PP, true, false); \
        else VIS_LAUNCH_COMPOSITE_S(TS, PP, false, false);       \
    } while (0)
    const bool two = ppt == 2;
    if (L.tile == 8) { if (two) VIS_LAUNCH_COMPOSITE(8, 2); else VIS_LAUNCH_COMPOSITE(8, 1); }
    else if (L.tile == 32) { if (two) VIS_LAUNCH_COMPOSITE(32, 2); else VIS_LAUNCH_COMPOSITE(32, 1); }
    else { if (two) VIS_LAUNCH_COMPOSITE(16, 2); else VIS_LAUNCH_COMPOSITE(16, 1); }
#undef VIS_LAUNCH_COMPOSITE
#undef VIS_LAUNCH_COMPOSITE_S
}

void launch_composite_batch(const Layout& L, char* ws, const BatchImage* images, int n_images, int64_t total_tiles,
                            float bg0, float bg1, float bg2, float alpha_min, float alpha_max, float t_stop, int ppt,
                            cudaStream_t stream) {
    const uint2* ranges = reinterpret_cast<const uint2*>(ws + L.off_ranges);
    const uint32_t* vals = reinterpret_cast<const uint32_t*>(ws + L.off_vals[L.sorted_buffer]);
    const float4* rec = reinterpret_cast<const float4*>(ws + L.off_rec);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.off_ctrl);
    if (total_tiles <= 0) return;
    const int blocks = (int)total_tiles;
    const float qcut = q_scale().qcut;
    const float* depth = reinterpret_cast<const float*>(ws + L.off_depth);
    const uint32_t* order = L.tile_fused ? reinterpret_cast<const uint32_t*>(ws + L.off_order) : nullptr;
#define VIS_LAUNCH_COMPOSITE_B(TS, PP)                                                                          \
    launch_k(true, composite_kernel<TS, sub_of(TS), PP, false, false, true>,                                     \
             blocks * (TS / sub_of(TS)) * (TS / sub_of(TS)), sub_of(TS) * sub_of(TS) / PP, 0, stream, ranges, vals, \
             rec, 0, 0, L.tiles_x, bg0, bg1, bg2, alpha_min, alpha_max, t_stop, qcut, ctrl, (float*)nullptr,       \
             (float*)nullptr, (float*)nullptr, (int32_t*)nullptr, depth, (const float*)nullptr, images, n_images,  \
             order)
    const bool two = ppt == 2;
    if (L.tile == 8) { if (two) VIS_LAUNCH_COMPOSITE_B(8, 2); else VIS_LAUNCH_COMPOSITE_B(8, 1); }
    else if (L.tile == 32) { if (two) VIS_LAUNCH_COMPOSITE_B(32, 2); else VIS_LAUNCH_COMPOSITE_B(32, 1); }
    else { if (two) VIS_LAUNCH_COMPOSITE_B(16, 2); else VIS_LAUNCH_COMPOSITE_B(16, 1); }
#undef VIS_LAUNCH_COMPOSITE_B
}

}  // namespace vis
