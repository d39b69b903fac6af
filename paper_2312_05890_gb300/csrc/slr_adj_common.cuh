// Pieces of the adjoint shared by its one-box-per-CTA kernel and its wide
// (per-layer tensor-core) form.
#pragma once

#include <cstdint>

#include "slr_kernels.h"

namespace slr {

__device__ __forceinline__ float sgnf(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

// Loss on the row bounds of one box, towards the nearer decision (Sec. 3
// check): SAFE needs every clause to have a row with hi < 0, so the safe loss
// is sum_c max(0, min_{r in c} hi_r); UNSAFE needs some clause with every
// lo_r >= 0, so the unsafe loss is min_c max(0, -min_{r in c} lo_r).  `dir`
// (1 safe, 2 unsafe) is taken when non-zero, else chosen (the smaller gap,
// SAFE on ties).  Writes the adjoints glo, ghi of the rows and returns the
// direction.
__device__ inline int8_t decision_grad(const NetParams<float> &net, const float *lo, const float *hi, float *glo,
                                       float *ghi, int8_t dir) {
    const int R = net.R;
    for (int r = 0; r < R; ++r) {
        glo[r] = 0.f;
        ghi[r] = 0.f;
    }
    float safe_gap = 0.f, unsafe_gap = INFINITY;
    int best_c = -1;
    int r0 = 0;
    for (int c = 0; c < net.n_clauses; ++c) {
        const int r1 = net.clause_end[c];
        float mh = INFINITY, ml = INFINITY;
        for (int r = r0; r < r1; ++r) {
            mh = fminf(mh, hi[r]);
            ml = fminf(ml, lo[r]);
        }
        safe_gap += fmaxf(mh, 0.f);
        const float ug = fmaxf(-ml, 0.f);
        if (ug < unsafe_gap) {
            unsafe_gap = ug;
            best_c = c;
        }
        r0 = r1;
    }
    if (dir == 0) dir = safe_gap <= unsafe_gap ? 1 : 2;
    r0 = 0;
    for (int c = 0; c < net.n_clauses; ++c) {
        const int r1 = net.clause_end[c];
        int rh = r0, rl = r0;
        for (int r = r0; r < r1; ++r) {
            if (hi[r] < hi[rh]) rh = r;
            if (lo[r] < lo[rl]) rl = r;
        }
        if (dir == 1 && hi[rh] > 0.f) ghi[rh] += 1.f;
        if (dir == 2 && c == best_c && lo[rl] < 0.f) glo[rl] = -1.f;
        r0 = r1;
    }
    return dir;
}

// One projected-Adam step on a slope with gradient g: descend, then clip to [0, 1].
__device__ __forceinline__ float adam_slope(const AdjArgs &a, int64_t ai, float al, float g) {
    const float m0 = a.adam_t == 1 ? 0.f : a.adam_m[ai];
    const float v0 = a.adam_t == 1 ? 0.f : a.adam_v[ai];
    const float mm = a.beta1 * m0 + (1.f - a.beta1) * g;
    const float vv = a.beta2 * v0 + (1.f - a.beta2) * g * g;
    a.adam_m[ai] = mm;
    a.adam_v[ai] = vv;
    const float mh = mm / (1.f - a.beta1_t);
    const float vh = vv / (1.f - a.beta2_t);
    const float nv = al - a.lr * mh / (sqrtf(vh) + a.eps);
    return fminf(fmaxf(nv, 0.f), 1.f);
}

}  // namespace slr
