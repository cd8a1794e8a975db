// Per (pixel, splat) evaluation shared by the compositor and its adjoint, written
// with explicit rounding intrinsics so both kernels take bit-identical decisions.
//
// Record layout (3 x float4 per Gaussian):
//   a = (u_hi, v_hi, u_lo, v_lo)   pixel-space centre in float-float
//   b = (f1x, f1y, f2x, f2y)       whitening rows: q = (d.f1)^2 + (d.f2)^2 = d^T S^-1 d
//   c = (opacity, r, g, b)
// d = pixel centre - (u, v). Eq. 2: w = opacity * exp(-q/2), cut at q > 9 (3 sigma).
#pragma once
#include "vis_internal.cuh"

namespace vis {

struct PairEval {
    float dx, dy, p1, p2, q;
};

__device__ __forceinline__ PairEval eval_pair(float pcx, float pcy, float4 a, float4 b) {
    PairEval e;
    e.dx = __fsub_rn(__fsub_rn(pcx, a.x), a.z);
    e.dy = __fsub_rn(__fsub_rn(pcy, a.y), a.w);
    e.p1 = __fmaf_rn(e.dy, b.y, __fmul_rn(e.dx, b.x));
    e.p2 = __fmaf_rn(e.dy, b.w, __fmul_rn(e.dx, b.z));
    e.q = __fmaf_rn(e.p2, e.p2, __fmul_rn(e.p1, e.p1));
    return e;
}

// Gaussian factor G = exp(-q/2)
__device__ __forceinline__ float gauss_of_q(float q) { return __expf(__fmul_rn(-0.5f, q)); }

}  // namespace vis
