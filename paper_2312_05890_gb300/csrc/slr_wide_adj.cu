// Adjoint of the SLR pass for wide networks: the state of a chunk of boxes
// lives in HBM and every affine layer, forward and backward, is one batched
// product on the tensor cores (wide_gemm_kernel).
//
// Forward, in plain float32 like the one-box adjoint kernel: the layer-1
// equations U = L = [W_1 diag(r) | W_1 m + b_1], then for every hidden layer k
// its pre-activation equations, kept in HBM as centre and radius
//   C_k = (U + L) / 2,  R_k = (U - L) / 2,
// the concrete bounds and slope of each neuron, and the relaxed equations
// (C', R') of Eq. 1, which the next product takes (Sec. 3):
//   C_{k+1} = W_k C' (+ b_k on the constant column),  R_{k+1} = |W_k| R'.
// Backward: the adjoints (gC, gR) = (gU + gL, gU - gL) of the equations of
// layer k + 1 go back through the product as
//   gC' = W_k^T gC,  gR' = |W_k|^T gR,
// (d/dU' = (gC' + gR') / 2, d/dL' = (gC' - gR') / 2), then through the
// relaxation of layer k row by row, with the slope gradient and the projected
// Adam step, to the adjoints of (C_k, R_k).  At layer 1 they give the box
// gradient.
//
// Layout as the sound wide path: [box][column][neuron], columns 0..d-1 the
// coefficients of the normalised inputs and column d the constant, neuron
// row stride NP.  Row kernels: a block is 32 neurons (threadIdx.x) of one box
// (blockIdx.y) with the columns split over 16 slices (threadIdx.y).
#include <algorithm>

#include "slr_adj_common.cuh"
#include "slr_eval.cuh"
#include "slr_kernels.h"

namespace slr {

namespace {

constexpr int kAX = 32, kAY = 16;

__device__ __forceinline__ size_t at(int64_t b, int Q, int c, int NP, int p) {
    return ((size_t)b * Q + c) * NP + p;
}

}  // namespace

// Centre and radius of each box of the chunk, rounded to nearest (the
// gradient only steers; no bound is taken from it).
__global__ void wadj_box_kernel(const BoxSource src, int64_t pos0, int nb, int d, float *m, float *r) {
    for (int64_t item = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; item < (int64_t)nb * d;
         item += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(item / d);
        const int i = (int)(item - (int64_t)b * d);
        const int64_t pos = pos0 + b;
        const int64_t idx = src.index != nullptr ? src.index[pos] : pos;
        double m64, r64;
        if (src.mode == 0) {
            unsigned long long kk;
            int c;
            code_dim(src, src.codes[idx], i, kk, c);
            const double w = src.root_w[i];
            r64 = ldexp(w, -(c + 1));
            m64 = src.root_lo[i] + w * ldexp((double)(2 * kk + 1), -(c + 1));
        } else {
            const double lo = (double)src.lo[idx * d + i];
            const double hi = (double)src.hi[idx * d + i];
            m64 = 0.5 * (lo + hi);
            r64 = 0.5 * (hi - lo);
        }
        m[item] = (float)m64;
        r[item] = (float)r64;
    }
}

// Layer 1: C = [W_1 diag(r) | W_1 m + b_1] (R = 0).  W0t: W_1 transposed (d x n_1).
__global__ void __launch_bounds__(kAX * kAY)
wadj_layer1_kernel(const NetParams<float> net, const float *W0t, int NP, const float *m, const float *r, float *C) {
    const int d = net.d, Q = d + 1, n1 = net.n[1];
    const int p = blockIdx.x * kAX + threadIdx.x;
    const int64_t b = blockIdx.y;
    if (p >= n1) return;
    const float *mb = m + b * d, *rb = r + b * d;
    for (int j = threadIdx.y; j < d; j += kAY) C[at(b, Q, j, NP, p)] = W0t[(size_t)j * n1 + p] * rb[j];
    if (threadIdx.y == 0) {
        float v = __ldg(net.b[0] + p);
        for (int i = 0; i < d; ++i) v = fmaf(W0t[(size_t)i * n1 + p], mb[i], v);
        C[at(b, Q, d, NP, p)] = v;
    }
}

// Hidden layer `layer`: bias on the constant column (bias non-null), concrete
// bounds of both equations, the slope, and the relaxed equations (Pc, Pr).
// sc: the five per-neuron scalars (ll, ul, lu, uu, slope), each nb_cap x NP.
__global__ void __launch_bounds__(kAX * kAY)
wadj_fwd_kernel(const AdjArgs a, int layer, int64_t pos0, int NP, float *C, const float *R, const float *bias,
                float *sc, int64_t sstride, float *Pc, float *Pr) {
    __shared__ float psu[kAY][kAX], psl[kAY][kAX];
    __shared__ float sp[5][kAX];
    const NetParams<float> &net = a.net;
    const int d = net.d, Q = d + 1, n = net.n[layer];
    const int lane = threadIdx.x, sl = threadIdx.y;
    const int p = blockIdx.x * kAX + lane;
    const int64_t b = blockIdx.y;
    const bool live = p < n;
    float su = 0.f, sv = 0.f;
    if (live) {
        if (sl == 0 && bias != nullptr) C[at(b, Q, d, NP, p)] += __ldg(bias + p);
        for (int c = sl; c < d; c += kAY) {
            const float cv = C[at(b, Q, c, NP, p)];
            const float rv = R != nullptr ? R[at(b, Q, c, NP, p)] : 0.f;
            su += fabsf(cv + rv);
            sv += fabsf(cv - rv);
        }
    }
    psu[sl][lane] = su;
    psl[sl][lane] = sv;
    __syncthreads();
    if (sl == 0 && live) {
        float tu = 0.f, tl = 0.f;
        for (int y = 0; y < kAY; ++y) {
            tu += psu[y][lane];
            tl += psl[y][lane];
        }
        const float cd = C[at(b, Q, d, NP, p)];
        const float rd = R != nullptr ? R[at(b, Q, d, NP, p)] : 0.f;
        const float ud = cd + rd, ldv = cd - rd;
        const float ll = ldv - tl, ul = ldv + tl, lu = ud - tu, uu = ud + tu;
        const bool lin = ll < 0.f && uu > 0.f && ul > 0.f;
        float al = lin ? ul / (ul - ll) : 0.f;
        int off = 0;
        for (int j = 1; j < layer; ++j) off += net.n[j];
        const int64_t ai = (pos0 + b) * a.H + off + p;
        if (a.alpha_mode == kAlphaFree) {
            al = fminf(fmaxf(a.alpha[ai], 0.f), 1.f);
        } else if (a.alpha_mode == kAlphaInit) {
            a.alpha[ai] = al;
        }
        const float v[5] = {ll, ul, lu, uu, al};
        for (int q = 0; q < 5; ++q) {
            sp[q][lane] = v[q];
            sc[q * sstride + b * NP + p] = v[q];
        }
    }
    __syncthreads();
    if (!live) return;
    const float ll = sp[0][lane], ul = sp[1][lane], lu = sp[2][lane], uu = sp[3][lane], al = sp[4][lane];
    for (int c = sl; c < Q; c += kAY) {
        const float cv = C[at(b, Q, c, NP, p)];
        const float rv = R != nullptr ? R[at(b, Q, c, NP, p)] : 0.f;
        const float u = cv + rv, l = cv - rv;
        float uh, lh;
        if (ll >= 0.f) {
            uh = u;
            lh = l;
        } else if (uu <= 0.f) {
            uh = 0.f;
            lh = 0.f;
        } else {
            if (lu >= 0.f) {
                uh = u;
            } else {
                const float sg = uu / (uu - lu);
                uh = sg * (c == d ? u - lu : u);
            }
            lh = ul > 0.f ? al * l : 0.f;
        }
        Pc[at(b, Q, c, NP, p)] = 0.5f * (uh + lh);
        Pr[at(b, Q, c, NP, p)] = 0.5f * (uh - lh);
    }
}

// Property rows of each box: lo = min L, hi = max U (bias on the constant
// column), the upstream adjoints (given, or the decision loss), and the
// adjoints (gC, gR) of the rows' equations.  One block per box.
__global__ void __launch_bounds__(256)
wadj_rows_kernel(const AdjArgs a, int64_t pos0, int NP, const float *C, const float *R, const float *bias, float *gC,
                 float *gR) {
    __shared__ float lo[kMaxRows], hi[kMaxRows], glo[kMaxRows], ghi[kMaxRows];
    const NetParams<float> &net = a.net;
    const int d = net.d, Q = d + 1, Rn = net.R;
    const int64_t b = blockIdx.x;
    const int64_t pos = pos0 + b;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < Rn; r += blockDim.x >> 5) {
        float su = 0.f, sv = 0.f;
        for (int c = lane; c < d; c += 32) {
            const float cv = C[at(b, Q, c, NP, r)], rv = R[at(b, Q, c, NP, r)];
            su += fabsf(cv + rv);
            sv += fabsf(cv - rv);
        }
        for (int o = 16; o > 0; o >>= 1) {
            su += __shfl_xor_sync(0xffffffffu, su, o);
            sv += __shfl_xor_sync(0xffffffffu, sv, o);
        }
        if (lane == 0) {
            const float cd = C[at(b, Q, d, NP, r)] + __ldg(bias + r), rd = R[at(b, Q, d, NP, r)];
            lo[r] = (cd - rd) - sv;
            hi[r] = (cd + rd) + su;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (a.g_lo != nullptr) {
            for (int r = 0; r < Rn; ++r) {
                glo[r] = a.g_lo[pos * Rn + r];
                ghi[r] = a.g_hi[pos * Rn + r];
            }
        } else {
            const int8_t dir = (a.alpha_mode == kAlphaInit || a.dir == nullptr) ? 0 : a.dir[pos];
            const int8_t got = decision_grad(net, lo, hi, glo, ghi, dir);
            if (dir == 0 && a.dir != nullptr) a.dir[pos] = got;
        }
        if (a.row_lo != nullptr) {
            for (int r = 0; r < Rn; ++r) {
                a.row_lo[pos * Rn + r] = lo[r];
                a.row_hi[pos * Rn + r] = hi[r];
            }
        }
    }
    __syncthreads();
    // d lo_r = d (L_r,d - sum |L_r,c|), d hi_r = d (U_r,d + sum |U_r,c|)
    for (int it = threadIdx.x; it < Q * Rn; it += blockDim.x) {
        const int c = it / Rn;
        const int r = it - c * Rn;
        const float cv = C[at(b, Q, c, NP, r)], rv = R[at(b, Q, c, NP, r)];
        const float gu = c == d ? ghi[r] : ghi[r] * sgnf(cv + rv);
        const float gl = c == d ? glo[r] : -glo[r] * sgnf(cv - rv);
        gC[at(b, Q, c, NP, r)] = gu + gl;
        gR[at(b, Q, c, NP, r)] = gu - gl;
    }
}

// Back through the relaxation of hidden layer `layer` (Eq. 1): from the
// adjoints (gPc, gPr) of the products' inputs to those of the pre-activation
// equations, written as (gC, gR) = (gU + gL, gU - gL) (gR null at layer 1,
// where U = L); the slope gradient and its projected-Adam step.
__global__ void __launch_bounds__(kAX * kAY)
wadj_bwd_kernel(const AdjArgs a, int layer, int64_t pos0, int NP, const float *C, const float *R, const float *sc,
                int64_t sstride, const float *gPc, const float *gPr, float *gC, float *gR) {
    __shared__ float ps[kAY][kAX], pa[kAY][kAX];
    __shared__ float sp[8][kAX];
    const NetParams<float> &net = a.net;
    const int d = net.d, Q = d + 1, n = net.n[layer];
    const int lane = threadIdx.x, sl = threadIdx.y;
    const int p = blockIdx.x * kAX + lane;
    const int64_t b = blockIdx.y;
    const bool live = p < n;
    float gs = 0.f, ga = 0.f;
    if (live) {
        for (int c = sl; c < Q; c += kAY) {
            const float gc = gPc[at(b, Q, c, NP, p)], gr = gPr[at(b, Q, c, NP, p)];
            const float cv = C[at(b, Q, c, NP, p)];
            const float rv = R != nullptr ? R[at(b, Q, c, NP, p)] : 0.f;
            gs = fmaf(0.5f * (gc + gr), cv + rv, gs);
            ga = fmaf(0.5f * (gc - gr), cv - rv, ga);
        }
    }
    ps[sl][lane] = gs;
    pa[sl][lane] = ga;
    __syncthreads();
    if (sl == 0 && live) {
        float g_s = 0.f, g_a = 0.f;
        for (int y = 0; y < kAY; ++y) {
            g_s += ps[y][lane];
            g_a += pa[y][lane];
        }
        const float ll = sc[0 * sstride + b * NP + p], ul = sc[1 * sstride + b * NP + p];
        const float lu = sc[2 * sstride + b * NP + p], uu = sc[3 * sstride + b * NP + p];
        const float al = sc[4 * sstride + b * NP + p];
        // kind: 0 active, 1 inactive, 2 unstable; then the chord and slope terms
        float kind = 0.f, sg = 1.f, du = 0.f, su = 0.f, dl = 0.f, sl2 = 0.f, lw = 0.f, chord = 0.f;
        float g_alpha = 0.f;
        if (ll >= 0.f) {
            kind = 0.f;
        } else if (uu <= 0.f) {
            kind = 1.f;
        } else {
            kind = 2.f;
            if (lu < 0.f) {
                chord = 1.f;
                const float gud = 0.5f * (gPc[at(b, Q, d, NP, p)] + gPr[at(b, Q, d, NP, p)]);
                const float den = uu - lu;
                sg = uu / den;
                const float gsum = g_s - lu * gud;
                const float g_uu = gsum * (-lu) / (den * den);
                const float g_lu = gsum * uu / (den * den) - sg * gud;
                du = g_uu - g_lu;
                su = g_uu + g_lu;
            }
            if (ul > 0.f) {
                lw = al;
                g_alpha = g_a;
                if (a.alpha_mode == kAlphaDefault) {
                    const float den = ul - ll;
                    const float g_ul = g_a * (-ll) / (den * den);
                    const float g_ll = g_a * ul / (den * den);
                    dl = g_ul - g_ll;
                    sl2 = g_ul + g_ll;
                }
            }
        }
        int off = 0;
        for (int j = 1; j < layer; ++j) off += net.n[j];
        const int64_t ai = (pos0 + b) * a.H + off + p;
        if (a.d_alpha != nullptr) a.d_alpha[ai] = g_alpha;
        if (a.adam_t > 0 && a.alpha_mode != kAlphaDefault) a.alpha[ai] = adam_slope(a, ai, al, g_alpha);
        const float v[8] = {kind, chord, sg, du, su, lw, dl, sl2};
        for (int q = 0; q < 8; ++q) sp[q][lane] = v[q];
    }
    __syncthreads();
    if (!live) return;
    const float kind = sp[0][lane], chord = sp[1][lane], sg = sp[2][lane], du = sp[3][lane], su = sp[4][lane];
    const float lw = sp[5][lane], dl = sp[6][lane], sl2 = sp[7][lane];
    for (int c = sl; c < Q; c += kAY) {
        const float gc = gPc[at(b, Q, c, NP, p)], gr = gPr[at(b, Q, c, NP, p)];
        const float gu = 0.5f * (gc + gr), gl = 0.5f * (gc - gr);
        float oU, oL;
        if (kind == 0.f) {
            oU = gu;
            oL = gl;
        } else if (kind == 1.f) {
            oU = 0.f;
            oL = 0.f;
        } else {
            const float cv = C[at(b, Q, c, NP, p)];
            const float rv = R != nullptr ? R[at(b, Q, c, NP, p)] : 0.f;
            if (chord != 0.f) {
                oU = c < d ? sg * gu + du * sgnf(cv + rv) : sg * gu + su;
            } else {
                oU = gu;
            }
            oL = lw * gl;
            if (dl != 0.f || sl2 != 0.f) oL += c < d ? dl * sgnf(cv - rv) : sl2;
        }
        gC[at(b, Q, c, NP, p)] = oU + oL;
        if (gR != nullptr) gR[at(b, Q, c, NP, p)] = oU - oL;
    }
}

// Box gradient from the adjoint gC1 of the layer-1 equations
// [W_1 diag(r) | W_1 m + b_1]: dM/dr_i = sum_p gC1[i][p] W_1[p][i],
// dM/dm_i = sum_p gC1[d][p] W_1[p][i].  One warp per (box, input).
__global__ void wadj_boxgrad_kernel(const AdjArgs a, int64_t pos0, int nb, int NP, const float *W0t, const float *gC1,
                                    float *gr_out) {
    const NetParams<float> &net = a.net;
    const int d = net.d, Q = d + 1, n1 = net.n[1];
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t item = wid; item < (int64_t)nb * d; item += nw) {
        const int64_t b = item / d;
        const int i = (int)(item - b * d);
        float gr = 0.f, gm = 0.f;
        for (int p = lane; p < n1; p += 32) {
            const float w = W0t[(size_t)i * n1 + p];
            gr = fmaf(gC1[at(b, Q, i, NP, p)], w, gr);
            gm = fmaf(gC1[at(b, Q, d, NP, p)], w, gm);
        }
        for (int o = 16; o > 0; o >>= 1) {
            gr += __shfl_xor_sync(0xffffffffu, gr, o);
            gm += __shfl_xor_sync(0xffffffffu, gm, o);
        }
        if (lane == 0) {
            const int64_t pos = pos0 + b;
            gr_out[b * d + i] = gr;
            if (a.d_r != nullptr) a.d_r[pos * d + i] = gr;
            if (a.d_lo != nullptr) {
                a.d_lo[pos * d + i] = 0.5f * (gm - gr);
                a.d_hi[pos * d + i] = 0.5f * (gm + gr);
            }
        }
    }
}

// Gradient split rule: the position in the split set of the dimension with
// the largest |dM/dr_i| r_i (the first on ties), into the box's code.
__global__ void wadj_split_kernel(const AdjArgs a, int64_t pos0, int nb, const float *gr, const float *r) {
    const int d = a.net.d;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const int64_t pos = pos0 + b;
        const int64_t idx = a.src.index != nullptr ? a.src.index[pos] : pos;
        if (a.split_cls[idx] != kUndecided) continue;
        int sel = 0;
        float best = -1.f;
        for (int j = 0; j < a.n_split; ++j) {
            const int i = a.split_dims[j];
            const float score = fabsf(gr[(size_t)b * d + i]) * r[(size_t)b * d + i];
            if (score > best) {
                best = score;
                sel = j;
            }
        }
        a.split_codes[idx] |= (unsigned long long)sel << (kSplitPathBits + 4 * a.src.t);
    }
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------
static int adj_grid_for(int64_t items, int sms) {
    const int64_t g = (items + 255) / 256;
    const int64_t cap = (int64_t)sms * 16;
    return (int)(g < 1 ? 1 : (g < cap ? g : cap));
}

cudaError_t launch_wadj_box(const BoxSource &src, int64_t pos0, int nb, int d, float *m, float *r, int sms,
                            cudaStream_t s) {
    wadj_box_kernel<<<adj_grid_for((int64_t)nb * d, sms), 256, 0, s>>>(src, pos0, nb, d, m, r);
    return cudaGetLastError();
}

cudaError_t launch_wadj_layer1(const NetParams<float> &net, const float *W0t, int nb, int NP, const float *m,
                               const float *r, float *C, cudaStream_t s) {
    wadj_layer1_kernel<<<dim3((net.n[1] + kAX - 1) / kAX, nb), dim3(kAX, kAY), 0, s>>>(net, W0t, NP, m, r, C);
    return cudaGetLastError();
}

cudaError_t launch_wadj_fwd(const AdjArgs &a, int layer, int64_t pos0, int nb, int NP, float *C, const float *R,
                            const float *bias, float *sc, int64_t sstride, float *Pc, float *Pr, cudaStream_t s) {
    wadj_fwd_kernel<<<dim3((a.net.n[layer] + kAX - 1) / kAX, nb), dim3(kAX, kAY), 0, s>>>(a, layer, pos0, NP, C, R,
                                                                                          bias, sc, sstride, Pc, Pr);
    return cudaGetLastError();
}

cudaError_t launch_wadj_rows(const AdjArgs &a, int64_t pos0, int nb, int NP, const float *C, const float *R,
                             const float *bias, float *gC, float *gR, cudaStream_t s) {
    wadj_rows_kernel<<<nb, 256, 0, s>>>(a, pos0, NP, C, R, bias, gC, gR);
    return cudaGetLastError();
}

cudaError_t launch_wadj_bwd(const AdjArgs &a, int layer, int64_t pos0, int nb, int NP, const float *C, const float *R,
                            const float *sc, int64_t sstride, const float *gPc, const float *gPr, float *gC, float *gR,
                            cudaStream_t s) {
    wadj_bwd_kernel<<<dim3((a.net.n[layer] + kAX - 1) / kAX, nb), dim3(kAX, kAY), 0, s>>>(
        a, layer, pos0, NP, C, R, sc, sstride, gPc, gPr, gC, gR);
    return cudaGetLastError();
}

cudaError_t launch_wadj_boxgrad(const AdjArgs &a, int64_t pos0, int nb, int NP, const float *W0t, const float *gC1,
                                float *gr, int sms, cudaStream_t s) {
    wadj_boxgrad_kernel<<<adj_grid_for((int64_t)nb * a.net.d * 32, sms), 256, 0, s>>>(a, pos0, nb, NP, W0t, gC1, gr);
    return cudaGetLastError();
}

cudaError_t launch_wadj_split(const AdjArgs &a, int64_t pos0, int nb, const float *gr, const float *r, int sms,
                              cudaStream_t s) {
    wadj_split_kernel<<<adj_grid_for(nb, sms), 256, 0, s>>>(a, pos0, nb, gr, r);
    return cudaGetLastError();
}

}  // namespace slr
