// Adjoint of the SLR pass and projected-Adam steps on the lower ReLU slopes.
//
// The lower line of an unstable ReLU (Eq. 1) may take any slope alpha in
// [0, 1] and stay sound, since relu(z) >= alpha z >= alpha Eq_l(x).  This file
// differentiates the row bounds of one box with respect to those slopes, the
// box endpoints, the weights and the biases (reverse mode through the
// concretisation, the relaxation and the affine contractions of Sec. 3), and
// applies projected Adam to the slopes.
//
// Arithmetic is plain float32 (round to nearest): the gradient only steers the
// slopes; every bound that decides a box comes from the sound evaluation
// kernel at the chosen slopes.
//
// One box per CTA.  Per hidden neuron the forward pass keeps five scalars
// (the concrete bounds of both equations and the slope used); the symbolic
// tensors of a hidden layer are kept in shared memory only for the first
// `nck` layers and are recomputed from the nearest kept layer during the
// backward sweep otherwise (layer-wise recomputation).
#include <cstdint>

#include "slr_kernels.h"
#include "slr_eval.cuh"

namespace slr {

namespace {

__device__ __forceinline__ float sgnf(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

struct AdjSmem {
    float *U, *L;        // pre-activation equations of the current layer, n x Q (Q = d + 1)
    float *C, *Rr;       // post-relaxation centre / radius of a hidden layer, n x Q
    float *gA, *gB;      // adjoints of the current layer's (U, L), reused as (gC', gR')
    float *gX, *gY;      // adjoints of the post-relaxation (U^, L^)
    float *scal;         // 5 x H: ll, ul, lu, uu, slope
    float *chk;          // nck x 2 x n_max x Q
    float *m, *r;        // box centre and radius (d)
    float *lo, *hi;      // row bounds (R)
    float *glo, *ghi;    // upstream adjoints of the row bounds (R)
    float *dm, *dr;      // box gradients (d)
    float *tmp;          // R x n_{K-1}: folded-layer weight gradient before unfolding
};

__device__ AdjSmem carve_adj(float *sp, const AdjArgs &a) {
    const int Q = a.net.d + 1;
    const size_t PQ = (size_t)a.n_max * Q;
    AdjSmem s;
    s.U = sp; sp += PQ;
    s.L = sp; sp += PQ;
    s.C = sp; sp += PQ;
    s.Rr = sp; sp += PQ;
    s.gA = sp; sp += PQ;
    s.gB = sp; sp += PQ;
    s.gX = sp; sp += PQ;
    s.gY = sp; sp += PQ;
    s.scal = sp; sp += 5 * (size_t)a.H;
    s.chk = sp; sp += 2 * (size_t)a.nck * PQ;
    s.m = sp; sp += a.net.d;
    s.r = sp; sp += a.net.d;
    s.lo = sp; sp += a.net.R;
    s.hi = sp; sp += a.net.R;
    s.glo = sp; sp += a.net.R;
    s.ghi = sp; sp += a.net.R;
    s.dm = sp; sp += a.net.d;
    s.dr = sp; sp += a.net.d;
    s.tmp = sp;
    return s;
}

// Weight w[p][i] of layer k (0-based, k = K-1 is the folded last layer).
__device__ __forceinline__ float weight(const NetParams<float> &net, int k, int p, int i) {
    if (k == 0) return __ldg(net.W0 + (size_t)p * net.d + i);
    return __ldg(net.Wt[k] + (size_t)i * net.n[k + 1] + p);
}

__device__ __forceinline__ int hidden_offset(const NetParams<float> &net, int layer) {
    int off = 0;
    for (int j = 1; j < layer; ++j) off += net.n[j];
    return off;
}

// Layer 1 in the normalised box coordinates x = m + r * xi:
// U = L = [W_1 diag(r) | W_1 m + b_1].
__device__ void build_layer1(const AdjArgs &a, const AdjSmem &s, float *U, float *L) {
    const NetParams<float> &net = a.net;
    const int d = net.d, Q = d + 1, n1 = net.n[1];
    for (int it = threadIdx.x; it < n1 * Q; it += blockDim.x) {
        const int p = it % n1;
        const int c = it / n1;
        float v;
        if (c < d) {
            v = weight(net, 0, p, c) * s.r[c];
        } else {
            v = __ldg(net.b[0] + p);
            for (int i = 0; i < d; ++i) v = fmaf(weight(net, 0, p, i), s.m[i], v);
        }
        U[p * Q + c] = v;
        L[p * Q + c] = v;
    }
}

// Relaxation of hidden layer `layer` (Eq. 1, per-equation bounds) from its
// pre-activation equations (U, L) and stored scalars, written as centre and
// radius of the post-activation pair.
__device__ void relax_layer(const AdjArgs &a, const AdjSmem &s, int layer, const float *U, const float *L) {
    const NetParams<float> &net = a.net;
    const int Q = net.d + 1, n = net.n[layer], H = a.H;
    const int off = hidden_offset(net, layer);
    for (int it = threadIdx.x; it < n * Q; it += blockDim.x) {
        const int j = it % n;
        const int c = it / n;
        const float ll = s.scal[off + j], ul = s.scal[H + off + j];
        const float lu = s.scal[2 * H + off + j], uu = s.scal[3 * H + off + j];
        const float al = s.scal[4 * H + off + j];
        const float u = U[j * Q + c], l = L[j * Q + c];
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
                uh = sg * (c == net.d ? u - lu : u);
            }
            lh = ul > 0.f ? al * l : 0.f;
        }
        s.C[j * Q + c] = 0.5f * (uh + lh);
        s.Rr[j * Q + c] = 0.5f * (uh - lh);
    }
}

// U' = W C + |W| Rr + b, L' = W C - |W| Rr + b for layer index k (0-based),
// mapping the post-activation of hidden layer k to layer k + 1.
__device__ void contract(const AdjArgs &a, const AdjSmem &s, int k, float *U, float *L) {
    const NetParams<float> &net = a.net;
    const int Q = net.d + 1, n_in = net.n[k], n_out = net.n[k + 1];
    for (int it = threadIdx.x; it < n_out * Q; it += blockDim.x) {
        const int p = it % n_out;
        const int c = it / n_out;
        float cc = c == net.d ? __ldg(net.b[k] + p) : 0.f, rr = 0.f;
        for (int i = 0; i < n_in; ++i) {
            const float w = weight(net, k, p, i);
            cc = fmaf(w, s.C[i * Q + c], cc);
            rr = fmaf(fabsf(w), s.Rr[i * Q + c], rr);
        }
        U[p * Q + c] = cc + rr;
        L[p * Q + c] = cc - rr;
    }
}

__device__ __forceinline__ float *chk_u(const AdjArgs &a, const AdjSmem &s, int layer) {
    return s.chk + (size_t)(layer - 1) * 2 * a.n_max * (a.net.d + 1);
}
__device__ __forceinline__ float *chk_l(const AdjArgs &a, const AdjSmem &s, int layer) {
    return chk_u(a, s, layer) + (size_t)a.n_max * (a.net.d + 1);
}

// Concrete bounds of hidden layer `layer` and the slope each neuron uses.
__device__ void concretize_layer(const AdjArgs &a, const AdjSmem &s, int layer, int64_t pos) {
    const NetParams<float> &net = a.net;
    const int d = net.d, Q = d + 1, n = net.n[layer], H = a.H;
    const int off = hidden_offset(net, layer);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        float su = 0.f, sl = 0.f;
        for (int c = 0; c < d; ++c) {
            su += fabsf(s.U[j * Q + c]);
            sl += fabsf(s.L[j * Q + c]);
        }
        const float ll = s.L[j * Q + d] - sl, ul = s.L[j * Q + d] + sl;
        const float lu = s.U[j * Q + d] - su, uu = s.U[j * Q + d] + su;
        const bool lin = ll < 0.f && uu > 0.f && ul > 0.f;
        float al = lin ? ul / (ul - ll) : 0.f;
        if (a.alpha_mode == kAlphaFree) {
            const float v = a.alpha[pos * H + off + j];
            al = fminf(fmaxf(v, 0.f), 1.f);
        } else if (a.alpha_mode == kAlphaInit) {
            a.alpha[pos * H + off + j] = al;
        }
        s.scal[off + j] = ll;
        s.scal[H + off + j] = ul;
        s.scal[2 * H + off + j] = lu;
        s.scal[3 * H + off + j] = uu;
        s.scal[4 * H + off + j] = al;
    }
}

// Recompute the pre-activation equations of hidden layer `layer` into (U, L)
// from the nearest kept layer, with the scalars stored by the forward pass.
__device__ void recompute(const AdjArgs &a, const AdjSmem &s, int layer) {
    int j = layer < a.nck ? layer : a.nck;
    if (j >= 1) {
        const int PQ = a.net.n[j] * (a.net.d + 1);
        for (int it = threadIdx.x; it < PQ; it += blockDim.x) {
            s.U[it] = chk_u(a, s, j)[it];
            s.L[it] = chk_l(a, s, j)[it];
        }
    } else {
        j = 1;
        build_layer1(a, s, s.U, s.L);
    }
    __syncthreads();
    for (; j < layer; ++j) {
        relax_layer(a, s, j, s.U, s.L);
        __syncthreads();
        contract(a, s, j, s.U, s.L);
        __syncthreads();
    }
}

// In-kernel loss on the row bounds of one box, towards the nearer decision
// (Sec. 3 check): SAFE needs every clause to have a row with hi < 0, so the
// safe loss is sum_c max(0, min_{r in c} hi_r); UNSAFE needs some clause with
// every lo_r >= 0, so the unsafe loss is min_c max(0, -min_{r in c} lo_r).
// The direction is fixed at the first step.  Sets glo, ghi (thread 0).
__device__ void decision_loss(const AdjArgs &a, const AdjSmem &s, int64_t pos) {
    const NetParams<float> &net = a.net;
    const int R = net.R;
    for (int r = 0; r < R; ++r) {
        s.glo[r] = 0.f;
        s.ghi[r] = 0.f;
    }
    float safe_gap = 0.f, unsafe_gap = INFINITY;
    int best_c = -1;
    int r0 = 0;
    for (int c = 0; c < net.n_clauses; ++c) {
        const int r1 = net.clause_end[c];
        float mh = INFINITY, ml = INFINITY;
        for (int r = r0; r < r1; ++r) {
            mh = fminf(mh, s.hi[r]);
            ml = fminf(ml, s.lo[r]);
        }
        safe_gap += fmaxf(mh, 0.f);
        const float ug = fmaxf(-ml, 0.f);
        if (ug < unsafe_gap) {
            unsafe_gap = ug;
            best_c = c;
        }
        r0 = r1;
    }
    int8_t dir = a.alpha_mode == kAlphaInit ? 0 : a.dir[pos];
    if (dir == 0) {
        dir = safe_gap <= unsafe_gap ? 1 : 2;
        a.dir[pos] = dir;
    }
    r0 = 0;
    for (int c = 0; c < net.n_clauses; ++c) {
        const int r1 = net.clause_end[c];
        int rh = r0, rl = r0;
        for (int r = r0; r < r1; ++r) {
            if (s.hi[r] < s.hi[rh]) rh = r;
            if (s.lo[r] < s.lo[rl]) rl = r;
        }
        if (dir == 1 && s.hi[rh] > 0.f) s.ghi[rh] += 1.f;
        if (dir == 2 && c == best_c && s.lo[rl] < 0.f) s.glo[rl] = -1.f;
        r0 = r1;
    }
}

}  // namespace

__global__ void __launch_bounds__(256) slr_adjoint_kernel(const AdjArgs a) {
    extern __shared__ __align__(16) float smem_adj[];
    const AdjSmem s = carve_adj(smem_adj, a);
    const NetParams<float> &net = a.net;
    const int K = net.K, d = net.d, Q = d + 1, R = net.R, H = a.H;

    int64_t n = a.n;
    if (a.count != nullptr) {
        const int64_t c = (int64_t)*a.count;
        n = c < n ? c : n;
    }
    for (int64_t pos = blockIdx.x; pos < n; pos += gridDim.x) {
        // ---- the box: centre and radius (Sec. 2.2 bisection for path codes) ----
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            const BoxSource &src = a.src;
            const int64_t idx = src.index != nullptr ? src.index[pos] : pos;
            double m64, r64;
            if (src.mode == 0) {
                const unsigned long long code = src.codes[idx];
                const unsigned long long mask = src.dim_mask[i] >> (src.D - src.t);
                const unsigned long long kk = pext64(code, mask);
                const int c = __popcll(mask);
                const double w = src.root_w[i];
                r64 = ldexp(w, -(c + 1));
                m64 = src.root_lo[i] + w * ldexp((double)(2 * kk + 1), -(c + 1));
            } else {
                const double lo = (double)src.lo[idx * d + i];
                const double hi = (double)src.hi[idx * d + i];
                m64 = 0.5 * (lo + hi);
                r64 = 0.5 * (hi - lo);
            }
            s.m[i] = (float)m64;
            s.r[i] = (float)r64;
            s.dm[i] = 0.f;
            s.dr[i] = 0.f;
        }
        __syncthreads();

        // ---- forward: equations, concrete bounds and slopes of every layer ----
        build_layer1(a, s, s.U, s.L);
        __syncthreads();
        for (int k = 1; k < K; ++k) {
            concretize_layer(a, s, k, pos);
            if (k <= a.nck) {
                const int PQ = net.n[k] * Q;
                for (int it = threadIdx.x; it < PQ; it += blockDim.x) {
                    chk_u(a, s, k)[it] = s.U[it];
                    chk_l(a, s, k)[it] = s.L[it];
                }
            }
            __syncthreads();
            relax_layer(a, s, k, s.U, s.L);
            __syncthreads();
            contract(a, s, k, s.U, s.L);
            __syncthreads();
        }
        // row bounds of the folded last layer
        for (int r = threadIdx.x; r < R; r += blockDim.x) {
            float su = 0.f, sl = 0.f;
            for (int c = 0; c < d; ++c) {
                su += fabsf(s.U[r * Q + c]);
                sl += fabsf(s.L[r * Q + c]);
            }
            s.lo[r] = s.L[r * Q + d] - sl;
            s.hi[r] = s.U[r * Q + d] + su;
            if (a.row_lo != nullptr) {
                a.row_lo[pos * R + r] = s.lo[r];
                a.row_hi[pos * R + r] = s.hi[r];
            }
            if (a.g_lo != nullptr) {
                s.glo[r] = a.g_lo[pos * R + r];
                s.ghi[r] = a.g_hi[pos * R + r];
            }
        }
        __syncthreads();
        if (a.g_lo == nullptr) {
            if (threadIdx.x == 0) decision_loss(a, s, pos);
            __syncthreads();
        }
        // d lo_r = d (L_r,d - sum |L_r,c|), d hi_r = d (U_r,d + sum |U_r,c|)
        for (int it = threadIdx.x; it < R * Q; it += blockDim.x) {
            const int r = it / Q;
            const int c = it - r * Q;
            s.gA[it] = c == d ? s.ghi[r] : s.ghi[r] * sgnf(s.U[it]);
            s.gB[it] = c == d ? s.glo[r] : -s.glo[r] * sgnf(s.L[it]);
        }
        __syncthreads();

        // ---- backward sweep: contraction k maps hidden layer k to layer k + 1 ----
        for (int k = K - 1; k >= 1; --k) {
            const int n_in = net.n[k], n_out = net.n[k + 1];
            const float *Uk, *Lk;
            if (k <= a.nck) {
                Uk = chk_u(a, s, k);
                Lk = chk_l(a, s, k);
            } else {
                recompute(a, s, k);
                Uk = s.U;
                Lk = s.L;
            }
            relax_layer(a, s, k, Uk, Lk);
            // (gU', gL') -> (gC', gR') = (gU' + gL', gU' - gL')
            for (int it = threadIdx.x; it < n_out * Q; it += blockDim.x) {
                const float u = s.gA[it], l = s.gB[it];
                s.gA[it] = u + l;
                s.gB[it] = u - l;
            }
            __syncthreads();
            // weight and bias gradients: dW[p][i] = sum_c gC'[p,c] C[i,c] + sgn(W) gR'[p,c] Rr[i,c]
            if (a.dW[k] != nullptr) {
                const bool last = k == K - 1;
                for (int it = threadIdx.x; it < n_out * n_in; it += blockDim.x) {
                    const int p = it / n_in;
                    const int i = it - p * n_in;
                    const float sw = sgnf(weight(net, k, p, i));
                    float v = 0.f;
                    for (int c = 0; c < Q; ++c)
                        v = fmaf(s.gA[p * Q + c], s.C[i * Q + c], fmaf(sw * s.gB[p * Q + c], s.Rr[i * Q + c], v));
                    if (last) s.tmp[it] = v;
                    else atomicAdd(a.dW[k] + it, v);
                }
                if (!last) {
                    for (int p = threadIdx.x; p < n_out; p += blockDim.x) atomicAdd(a.db[k] + p, s.gA[p * Q + d]);
                } else {
                    // the folded rows are C W_K: dW_K = C^T dW', db_K = C^T db'
                    __syncthreads();
                    const int no = a.n_out;
                    for (int it = threadIdx.x; it < no * n_in; it += blockDim.x) {
                        const int o = it / n_in;
                        const int i = it - o * n_in;
                        float v = 0.f;
                        for (int r = 0; r < R; ++r) v = fmaf(__ldg(a.Cprop + r * no + o), s.tmp[r * n_in + i], v);
                        atomicAdd(a.dW[k] + it, v);
                    }
                    for (int o = threadIdx.x; o < no; o += blockDim.x) {
                        float v = 0.f;
                        for (int r = 0; r < R; ++r) v = fmaf(__ldg(a.Cprop + r * no + o), s.gA[r * Q + d], v);
                        atomicAdd(a.db[k] + o, v);
                    }
                }
            }
            // adjoints of the post-relaxation pair: gU^ = (W^T gC' + |W|^T gR') / 2, gL^ = (W^T gC' - |W|^T gR') / 2
            for (int it = threadIdx.x; it < n_in * Q; it += blockDim.x) {
                const int i = it % n_in;
                const int c = it / n_in;
                float gc = 0.f, gr = 0.f;
                for (int p = 0; p < n_out; ++p) {
                    const float w = weight(net, k, p, i);
                    gc = fmaf(w, s.gA[p * Q + c], gc);
                    gr = fmaf(fabsf(w), s.gB[p * Q + c], gr);
                }
                s.gX[i * Q + c] = 0.5f * (gc + gr);
                s.gY[i * Q + c] = 0.5f * (gc - gr);
            }
            __syncthreads();
            // through the relaxation (Eq. 1) of hidden layer k, one neuron per thread
            const int off = hidden_offset(net, k);
            for (int j = threadIdx.x; j < n_in; j += blockDim.x) {
                const float ll = s.scal[off + j], ul = s.scal[H + off + j];
                const float lu = s.scal[2 * H + off + j], uu = s.scal[3 * H + off + j];
                const float al = s.scal[4 * H + off + j];
                const float *u = Uk + j * Q, *l = Lk + j * Q;
                const float *gu = s.gX + j * Q, *gl = s.gY + j * Q;
                float *oU = s.gA + j * Q, *oL = s.gB + j * Q;
                float g_alpha = 0.f;
                if (ll >= 0.f) {
                    for (int c = 0; c < Q; ++c) {
                        oU[c] = gu[c];
                        oL[c] = gl[c];
                    }
                } else if (uu <= 0.f) {
                    for (int c = 0; c < Q; ++c) {
                        oU[c] = 0.f;
                        oL[c] = 0.f;
                    }
                } else {
                    // upper: identity (lu >= 0) or chord sg (U - lu), sg = uu / (uu - lu)
                    if (lu >= 0.f) {
                        for (int c = 0; c < Q; ++c) oU[c] = gu[c];
                    } else {
                        const float den = uu - lu;
                        const float sg = uu / den;
                        float g_s = -lu * gu[d];
                        for (int c = 0; c < Q; ++c) g_s = fmaf(gu[c], u[c], g_s);
                        const float g_uu = g_s * (-lu) / (den * den);
                        const float g_lu = g_s * uu / (den * den) - sg * gu[d];
                        for (int c = 0; c < d; ++c) oU[c] = sg * gu[c] + (g_uu - g_lu) * sgnf(u[c]);
                        oU[d] = sg * gu[d] + g_uu + g_lu;
                    }
                    // lower: slope * L (ul > 0) or 0
                    if (ul > 0.f) {
                        for (int c = 0; c < Q; ++c) g_alpha = fmaf(gl[c], l[c], g_alpha);
                        for (int c = 0; c < Q; ++c) oL[c] = al * gl[c];
                        if (a.alpha_mode == kAlphaDefault) {
                            // slope ul / (ul - ll) depends on the box through (ll, ul)
                            const float den = ul - ll;
                            const float g_ul = g_alpha * (-ll) / (den * den);
                            const float g_ll = g_alpha * ul / (den * den);
                            for (int c = 0; c < d; ++c) oL[c] += (g_ul - g_ll) * sgnf(l[c]);
                            oL[d] += g_ul + g_ll;
                        }
                    } else {
                        for (int c = 0; c < Q; ++c) oL[c] = 0.f;
                    }
                }
                const int64_t ai = pos * H + off + j;
                if (a.d_alpha != nullptr) a.d_alpha[ai] = g_alpha;
                if (a.adam_t > 0 && a.alpha_mode != kAlphaDefault) {
                    // projected Adam on the loss: descend, then clip to [0, 1]
                    const float m0 = a.adam_t == 1 ? 0.f : a.adam_m[ai];
                    const float v0 = a.adam_t == 1 ? 0.f : a.adam_v[ai];
                    const float mm = a.beta1 * m0 + (1.f - a.beta1) * g_alpha;
                    const float vv = a.beta2 * v0 + (1.f - a.beta2) * g_alpha * g_alpha;
                    a.adam_m[ai] = mm;
                    a.adam_v[ai] = vv;
                    const float mh = mm / (1.f - a.beta1_t);
                    const float vh = vv / (1.f - a.beta2_t);
                    const float nv = al - a.lr * mh / (sqrtf(vh) + a.eps);
                    a.alpha[ai] = fminf(fmaxf(nv, 0.f), 1.f);
                }
            }
            __syncthreads();
        }

        // ---- layer 1: U = L = [W_1 diag(r) | W_1 m + b_1] ----
        for (int it = threadIdx.x; it < net.n[1] * Q; it += blockDim.x) s.gA[it] += s.gB[it];
        __syncthreads();
        const int n1 = net.n[1];
        if (a.dW[0] != nullptr) {
            if (K > 1) {
                for (int it = threadIdx.x; it < n1 * d; it += blockDim.x) {
                    const int p = it / d;
                    const int i = it - p * d;
                    atomicAdd(a.dW[0] + it, fmaf(s.gA[p * Q + i], s.r[i], s.gA[p * Q + d] * s.m[i]));
                }
                for (int p = threadIdx.x; p < n1; p += blockDim.x) atomicAdd(a.db[0] + p, s.gA[p * Q + d]);
            } else {
                // a single affine layer is the folded one: unfold with the property rows
                for (int it = threadIdx.x; it < R * d; it += blockDim.x) {
                    const int r = it / d;
                    const int i = it - r * d;
                    s.tmp[it] = fmaf(s.gA[r * Q + i], s.r[i], s.gA[r * Q + d] * s.m[i]);
                }
                __syncthreads();
                const int no = a.n_out;
                for (int it = threadIdx.x; it < no * d; it += blockDim.x) {
                    const int o = it / d;
                    const int i = it - o * d;
                    float v = 0.f;
                    for (int r = 0; r < R; ++r) v = fmaf(__ldg(a.Cprop + r * no + o), s.tmp[r * d + i], v);
                    atomicAdd(a.dW[0] + it, v);
                }
                for (int o = threadIdx.x; o < no; o += blockDim.x) {
                    float v = 0.f;
                    for (int r = 0; r < R; ++r) v = fmaf(__ldg(a.Cprop + r * no + o), s.gA[r * Q + d], v);
                    atomicAdd(a.db[0] + o, v);
                }
            }
        }
        if (a.d_lo != nullptr) {
            for (int i = threadIdx.x; i < d; i += blockDim.x) {
                float gr = 0.f, gm = 0.f;
                for (int p = 0; p < n1; ++p) {
                    const float w = weight(net, 0, p, i);
                    gr = fmaf(s.gA[p * Q + i], w, gr);
                    gm = fmaf(s.gA[p * Q + d], w, gm);
                }
                // m = (lo + hi) / 2, r = (hi - lo) / 2
                a.d_lo[pos * d + i] = 0.5f * (gm - gr);
                a.d_hi[pos * d + i] = 0.5f * (gm + gr);
            }
        }
        __syncthreads();
    }
}

// Best-so-far sound bounds over the slope steps: each step's bounds are sound,
// so their intersection is; the class follows from it (Sec. 3 check).
__global__ void slr_merge_bounds_kernel(const NetParams<float> net, int64_t n, const unsigned long long *count,
                                        const float *lo_new, const float *hi_new, float *lo_best, float *hi_best,
                                        uint8_t *cls_pos, uint8_t *cls_idx, const int64_t *index, int first,
                                        unsigned long long *decided) {
    const int R = net.R;
    if (count != nullptr) {
        const int64_t c = (int64_t)*count;
        n = c < n ? c : n;
    }
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        bool any_in = false, all_out = true;
        int r0 = 0;
        for (int c = 0; c < net.n_clauses; ++c) {
            const int r1 = net.clause_end[c];
            bool all_in = true, some_out = false;
            for (int r = r0; r < r1; ++r) {
                float lo = lo_new[b * R + r], hi = hi_new[b * R + r];
                if (!first) {
                    lo = fmaxf(lo, lo_best[b * R + r]);
                    hi = fminf(hi, hi_best[b * R + r]);
                }
                lo_best[b * R + r] = lo;
                hi_best[b * R + r] = hi;
                const bool st = net.strict[r] != 0;
                all_in = all_in && (st ? lo > 0.f : lo >= 0.f);
                some_out = some_out || (st ? hi <= 0.f : hi < 0.f);
            }
            any_in = any_in || all_in;
            all_out = all_out && some_out;
            r0 = r1;
        }
        const uint8_t cl = any_in ? kUnsafe : (all_out ? kSafe : kUndecided);
        if (cls_pos != nullptr) cls_pos[b] = cl;
        if (cls_idx != nullptr) cls_idx[index != nullptr ? index[b] : b] = cl;
        if (decided != nullptr && cl != kUndecided) atomicAdd(decided, 1ull);
    }
}

// Positions of the UNDECIDED boxes of a level (warp-aggregated append).
__global__ void slr_gather_undecided_kernel(const uint8_t *cls, const unsigned long long *n_ptr, int64_t cap,
                                            int64_t *list, unsigned long long *list_n, int64_t list_cap) {
    int64_t n = (int64_t)*n_ptr;
    n = n < cap ? n : cap;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        const bool und = i < n && cls[i] == kUndecided;
        const unsigned ballot = __ballot_sync(0xffffffffu, und);
        if (ballot == 0u) continue;
        unsigned long long start = 0;
        if (lane == 0) start = atomicAdd(list_n, (unsigned long long)__popc(ballot));
        start = __shfl_sync(0xffffffffu, start, 0);
        if (und) {
            const int64_t at = (int64_t)start + __popc(ballot & ((1u << lane) - 1u));
            if (at < list_cap) list[at] = i;
        }
    }
}

size_t adjoint_smem_bytes(const AdjArgs &a) {
    const size_t PQ = (size_t)a.n_max * (a.net.d + 1);
    const size_t tmp = (size_t)a.net.R * a.net.n[a.net.K - 1];
    return sizeof(float) * (8 * PQ + 5 * (size_t)a.H + 2 * (size_t)a.nck * PQ + 4 * (size_t)a.net.d +
                            4 * (size_t)a.net.R + tmp);
}

cudaError_t launch_adjoint(const AdjArgs &a, int grid, cudaStream_t s) {
    const size_t smem = adjoint_smem_bytes(a);
    cudaError_t e = cudaFuncSetAttribute(slr_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    slr_adjoint_kernel<<<grid, 256, smem, s>>>(a);
    return cudaGetLastError();
}

int adjoint_blocks_per_sm(size_t smem) {
    int nb = 0;
    cudaFuncSetAttribute(slr_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, slr_adjoint_kernel, 256, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_merge_bounds(const NetParams<float> &net, int64_t n, const unsigned long long *count,
                                const float *lo_new, const float *hi_new, float *lo_best, float *hi_best,
                                uint8_t *cls_pos, uint8_t *cls_idx, const int64_t *index, int first,
                                unsigned long long *decided, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    slr_merge_bounds_kernel<<<grid, 256, 0, s>>>(net, n, count, lo_new, hi_new, lo_best, hi_best, cls_pos, cls_idx,
                                                 index, first, decided);
    return cudaGetLastError();
}

cudaError_t launch_gather_undecided(const uint8_t *cls, const unsigned long long *n, int64_t cap, int64_t *list,
                                    unsigned long long *list_n, int64_t list_cap, int grid, cudaStream_t s) {
    slr_gather_undecided_kernel<<<grid, 256, 0, s>>>(cls, n, cap, list, list_n, list_cap);
    return cudaGetLastError();
}

}  // namespace slr
