// A splat's tile footprint: the tiles it is listed in (its "copies").
//
// Stored per Gaussian as a uint4: x = x0 | x1 << 16, y = y0 | y1 << 16 (the tile box,
// upper bounds exclusive), z = trims, w = 0. The box is [x0, x1) x [y0, y1); the trims
// narrow its top row (y0) and its bottom row (y1 - 1) to the tiles the splat's ellipse
// actually reaches: z = Lt | Rt << 8 | Lb << 16 | Rb << 24, the numbers of tiles dropped at
// the left and right ends of the top (t) and bottom (b) rows, with L + R <= x1 - x0 (a row
// may end up empty). A one-row box uses the top trims only; the middle rows keep the box's
// full width. The copies are enumerated row by row (top to bottom), left to right; every
// kernel that counts, lists or bins copies uses these helpers, so all sort modes list
// exactly the same (tile, splat) pairs.
#pragma once
#include <cstdint>

namespace vis {

struct Footprint {
    uint32_t x0, x1, y0, y1, trims;
};

__host__ __device__ __forceinline__ Footprint fp_unpack(uint4 r) {
    Footprint f;
    f.x0 = r.x & 0xffffu; f.x1 = r.x >> 16;
    f.y0 = r.y & 0xffffu; f.y1 = r.y >> 16;
    f.trims = r.z;
    return f;
}

__host__ __device__ __forceinline__ uint32_t fp_pack_trims(uint32_t lt, uint32_t rt, uint32_t lb, uint32_t rb) {
    return (lt & 0xffu) | (rt & 0xffu) << 8 | (lb & 0xffu) << 16 | (rb & 0xffu) << 24;
}

// width of the top and bottom rows
__host__ __device__ __forceinline__ uint32_t fp_top_width(const Footprint& f) {
    return (f.x1 - f.x0) - (f.trims & 0xffu) - ((f.trims >> 8) & 0xffu);
}
__host__ __device__ __forceinline__ uint32_t fp_bottom_width(const Footprint& f) {
    return (f.x1 - f.x0) - ((f.trims >> 16) & 0xffu) - (f.trims >> 24);
}

// number of copies
__host__ __device__ __forceinline__ uint32_t fp_count(const Footprint& f) {
    if (f.x1 <= f.x0 || f.y1 <= f.y0) return 0;
    const uint32_t rows = f.y1 - f.y0;
    if (rows == 1) return fp_top_width(f);
    return fp_top_width(f) + (rows - 2) * (f.x1 - f.x0) + fp_bottom_width(f);
}

// tile (row-major id) of copy k, 0 <= k < fp_count(f)
__host__ __device__ __forceinline__ uint32_t fp_tile(const Footprint& f, uint32_t k, uint32_t tiles_x) {
    const uint32_t W = f.x1 - f.x0, wt = fp_top_width(f);
    if (k < wt) return f.y0 * tiles_x + f.x0 + (f.trims & 0xffu) + k;
    k -= wt;
    const uint32_t mid = (f.y1 - f.y0 - 2) * W;   // rows >= 2 here
    if (k < mid) {
        const uint32_t r = k / W;
        return (f.y0 + 1 + r) * tiles_x + f.x0 + (k - r * W);
    }
    k -= mid;
    return (f.y1 - 1) * tiles_x + f.x0 + ((f.trims >> 16) & 0xffu) + k;
}

#ifdef __CUDACC__
// add v to a 2D difference array over a tiles_x x tiles_y grid for the tile rectangle
// [x0, x1) x [y0, y1); corners at x1 == tiles_x or y1 == tiles_y only affect tiles outside
// the grid
__device__ __forceinline__ void diff_rect(int* diff, uint32_t x0, uint32_t x1, uint32_t y0, uint32_t y1, int v,
                                          uint32_t tiles_x, uint32_t tiles_y) {
    atomicAdd(&diff[y0 * tiles_x + x0], v);
    if (x1 < tiles_x) atomicAdd(&diff[y0 * tiles_x + x1], -v);
    if (y1 < tiles_y) {
        atomicAdd(&diff[y1 * tiles_x + x0], -v);
        if (x1 < tiles_x) atomicAdd(&diff[y1 * tiles_x + x1], v);
    }
}

// add one footprint (its box, then its trimmed row ends taken out again) to a 2D difference
// array, so that the array's 2D prefix sums count every copy once
__device__ __forceinline__ void fp_add_to_diff(int* diff, const Footprint& f, uint32_t tiles_x, uint32_t tiles_y) {
    if (f.x1 <= f.x0 || f.y1 <= f.y0) return;
    diff_rect(diff, f.x0, f.x1, f.y0, f.y1, 1, tiles_x, tiles_y);
    if (f.trims) {
        const uint32_t lt = f.trims & 0xffu, rt = (f.trims >> 8) & 0xffu;
        const uint32_t lb = (f.trims >> 16) & 0xffu, rb = f.trims >> 24;
        if (lt) diff_rect(diff, f.x0, f.x0 + lt, f.y0, f.y0 + 1, -1, tiles_x, tiles_y);
        if (rt) diff_rect(diff, f.x1 - rt, f.x1, f.y0, f.y0 + 1, -1, tiles_x, tiles_y);
        if (f.y1 - f.y0 > 1) {
            if (lb) diff_rect(diff, f.x0, f.x0 + lb, f.y1 - 1, f.y1, -1, tiles_x, tiles_y);
            if (rb) diff_rect(diff, f.x1 - rb, f.x1, f.y1 - 1, f.y1, -1, tiles_x, tiles_y);
        }
    }
}
#endif

}  // namespace vis
