// The per-frame update of a dynamic scene, standing in for the paper's per-frame Gaussian
// generator (section 3.3: a model produces the Gaussians of each frame, which the renderer
// then preprocesses and re-sorts globally; section 4 shows that re-sorting every frame is
// what avoids lazy-sort artifacts):
//   mu_t    = mu_0 + t v
//   logit_t = logit_0 + A sin(2 pi f t + phi)
// Shared by the update kernel (dynamic.cu) and by the preprocess of vis_render_dynamic, which
// applies it to the frame-0 attributes as it loads them. Both files are compiled without
// floating-point contraction, so the two round every value identically.
#pragma once
#include "vis_internal.cuh"

namespace vis {

constexpr float kInvPi = (float)(1.0 / 3.14159265358979323846);

__device__ __forceinline__ float dyn_mean(float m0, float v, float t) { return __fmaf_rn(t, v, m0); }

// sin(2 pi f t + phi) as sinpi(2 f t + phi / pi): the same angle, with an exact range reduction
// (no large-argument path, so no local-memory table in the kernels that inline it)
__device__ __forceinline__ float dyn_logit(float l0, float amp, float freq, float phase, float t) {
    const float x = __fmaf_rn(__fmul_rn(2.f, freq), t, __fmul_rn(phase, kInvPi));
    return __fmaf_rn(amp, sinpif(x), l0);
}

}  // namespace vis
