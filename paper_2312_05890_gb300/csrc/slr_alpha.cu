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
// A CTA works on a group of boxes together (as many as fit its shared-memory
// share; one box with the state in global memory for networks whose state
// does not fit), every phase a flat loop over the group's elements.  Per
// hidden neuron the forward pass keeps five scalars
// (the concrete bounds of both equations and the slope used); the symbolic
// tensors of a hidden layer are kept in shared memory only for the first
// `nck` layers and are recomputed from the nearest kept layer during the
// backward sweep otherwise (layer-wise recomputation).
#include <cstdint>

#include "slr_kernels.h"
#include "slr_eval.cuh"
#include "slr_adj_common.cuh"

namespace slr {

namespace {

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
    float *tmp;          // R x n_{K-1}: folded-layer weight gradient before unfolding
};

// Floats of one box's shared-memory state.
__host__ __device__ inline size_t adj_box_floats(const AdjArgs &a) {
    const size_t PQ = (size_t)a.n_max * (a.net.d + 1);
    const size_t tmp = (size_t)a.net.R * (a.net.K > 1 ? a.net.n[a.net.K - 1] : a.net.d);
    const size_t f = 8 * PQ + 5 * (size_t)a.H + 2 * (size_t)a.nck * PQ + 2 * (size_t)a.net.d + 4 * (size_t)a.net.R + tmp;
    return (f + 3) & ~(size_t)3;
}

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
    s.tmp = sp;
    return s;
}

// Quotient by a loop-invariant divisor n >= 1 without a division per use:
// with m = floor((2^32 - 1) / n) + 1 (= ceil(2^32 / n) for n >= 2),
// floor(x m / 2^32) = floor(x / n) whenever x n <= 2^32, because the excess
// e = m n - 2^32 is below n and so x e / 2^32 < 1 cannot carry the fraction
// x / n past the next integer.  Larger operands and n = 1 divide plainly.
struct Div {
    uint32_t m;
    int n;
    bool fast;
    __device__ __forceinline__ Div(int n_, int x_end) : n(n_) {
        fast = n_ > 1 && (uint64_t)(uint32_t)x_end * (uint32_t)n_ <= (1ull << 32);
        m = fast ? 0xFFFFFFFFu / (uint32_t)n_ + 1u : 0u;
    }
    __device__ __forceinline__ int operator()(int x) const {
        return fast ? (int)__umulhi((uint32_t)x, m) : x / n;
    }
};

// The boxes a CTA works on together: box q (q < nb) at position pos0 + q,
// its state at base + q * stride floats.
struct Group {
    float *base;
    size_t stride;
    int nb;
    int64_t pos0;
    __device__ __forceinline__ AdjSmem box(const AdjArgs &a, int q) const { return carve_adj(base + q * stride, a); }
};

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

__device__ __forceinline__ float *chk_u(const AdjArgs &a, const AdjSmem &s, int layer) {
    return s.chk + (size_t)(layer - 1) * 2 * a.n_max * (a.net.d + 1);
}
__device__ __forceinline__ float *chk_l(const AdjArgs &a, const AdjSmem &s, int layer) {
    return chk_u(a, s, layer) + (size_t)a.n_max * (a.net.d + 1);
}

// Layer 1 in the normalised box coordinates x = m + r * xi:
// U = L = [W_1 diag(r) | W_1 m + b_1].
__device__ void build_layer1(const AdjArgs &a, const Group &g) {
    const NetParams<float> &net = a.net;
    const int d = net.d, Q = d + 1, n1 = net.n[1];
    const int work = n1 * Q;
    const Div by_work(work, g.nb * work), by_n(n1, work);
    for (int it = threadIdx.x; it < g.nb * work; it += blockDim.x) {
        const int q = by_work(it);
        const int li = it - q * work;
        const int c = by_n(li);
        const int p = li - c * n1;
        const AdjSmem s = g.box(a, q);
        float v;
        if (c < d) {
            v = weight(net, 0, p, c) * s.r[c];
        } else {
            v = __ldg(net.b[0] + p);
            for (int i = 0; i < d; ++i) v = fmaf(weight(net, 0, p, i), s.m[i], v);
        }
        s.U[p * Q + c] = v;
        s.L[p * Q + c] = v;
    }
}

// Relaxation of hidden layer `layer` (Eq. 1, per-equation bounds) from its
// pre-activation equations and stored scalars, written as centre and radius
// of the post-activation pair.  from_chk: read the kept copy of the layer.
__device__ void relax_layer(const AdjArgs &a, const Group &g, int layer, bool from_chk) {
    const NetParams<float> &net = a.net;
    const int Q = net.d + 1, n = net.n[layer], H = a.H;
    const int off = hidden_offset(net, layer);
    const int work = n * Q;
    const Div by_work(work, g.nb * work), by_n(n, work);
    for (int it = threadIdx.x; it < g.nb * work; it += blockDim.x) {
        const int q = by_work(it);
        const int li = it - q * work;
        const int c = by_n(li);
        const int j = li - c * n;
        const AdjSmem s = g.box(a, q);
        const float *U = from_chk ? chk_u(a, s, layer) : s.U;
        const float *L = from_chk ? chk_l(a, s, layer) : s.L;
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

constexpr int kAdjCols = 8;   // equation columns one thread carries through a product

// U' = W C + |W| Rr + b, L' = W C - |W| Rr + b for layer index k (0-based),
// mapping the post-activation of hidden layer k to layer k + 1.  One item is
// an output row of one box and up to kAdjCols columns (independent sums).
__device__ void contract(const AdjArgs &a, const Group &g, int k) {
    const NetParams<float> &net = a.net;
    const int Q = net.d + 1, n_in = net.n[k], n_out = net.n[k + 1];
    const int nch = (Q + kAdjCols - 1) / kAdjCols;
    const int work = n_out * nch;
    const Div by_work(work, g.nb * work), by_n(n_out, work);
    for (int it = threadIdx.x; it < g.nb * work; it += blockDim.x) {
        const int q = by_work(it);
        const int li = it - q * work;
        const int ch = by_n(li);
        const int p = li - ch * n_out;
        const int c0 = ch * kAdjCols;
        const int nc = Q - c0 < kAdjCols ? Q - c0 : kAdjCols;
        const AdjSmem s = g.box(a, q);
        float cc[kAdjCols], rr[kAdjCols];
#pragma unroll
        for (int c = 0; c < kAdjCols; ++c) {
            cc[c] = 0.f;
            rr[c] = 0.f;
        }
        for (int i = 0; i < n_in; ++i) {
            const float w = weight(net, k, p, i);
            const float aw = fabsf(w);
            const float *ci = s.C + i * Q + c0, *ri = s.Rr + i * Q + c0;
#pragma unroll
            for (int c = 0; c < kAdjCols; ++c) {
                if (c < nc) {
                    cc[c] = fmaf(w, ci[c], cc[c]);
                    rr[c] = fmaf(aw, ri[c], rr[c]);
                }
            }
        }
        const float bp = __ldg(net.b[k] + p);
#pragma unroll
        for (int c = 0; c < kAdjCols; ++c) {
            if (c < nc) {
                const float cv = c0 + c == net.d ? cc[c] + bp : cc[c];
                s.U[p * Q + c0 + c] = cv + rr[c];
                s.L[p * Q + c0 + c] = cv - rr[c];
            }
        }
    }
}

// Concrete bounds of hidden layer `layer` and the slope each neuron uses; the
// layer's equations are kept when it is among the first nck.
__device__ void concretize_layer(const AdjArgs &a, const Group &g, int layer) {
    const NetParams<float> &net = a.net;
    const int d = net.d, Q = d + 1, n = net.n[layer], H = a.H;
    const int off = hidden_offset(net, layer);
    const Div by_n(n, g.nb * n);
    for (int it = threadIdx.x; it < g.nb * n; it += blockDim.x) {
        const int q = by_n(it);
        const int j = it - q * n;
        const AdjSmem s = g.box(a, q);
        const int64_t pos = g.pos0 + q;
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
    if (layer <= a.nck) {
        const int work = n * Q;
        const Div by_work(work, g.nb * work);
        for (int it = threadIdx.x; it < g.nb * work; it += blockDim.x) {
            const int q = by_work(it);
            const int li = it - q * work;
            const AdjSmem s = g.box(a, q);
            chk_u(a, s, layer)[li] = s.U[li];
            chk_l(a, s, layer)[li] = s.L[li];
        }
    }
}

// Recompute the pre-activation equations of hidden layer `layer` into (U, L)
// from the nearest kept layer, with the scalars stored by the forward pass.
__device__ void recompute(const AdjArgs &a, const Group &g, int layer) {
    int j = layer < a.nck ? layer : a.nck;
    if (j >= 1) {
        const int work = a.net.n[j] * (a.net.d + 1);
        const Div by_work(work, g.nb * work);
        for (int it = threadIdx.x; it < g.nb * work; it += blockDim.x) {
            const int q = by_work(it);
            const int li = it - q * work;
            const AdjSmem s = g.box(a, q);
            s.U[li] = chk_u(a, s, j)[li];
            s.L[li] = chk_l(a, s, j)[li];
        }
    } else {
        j = 1;
        build_layer1(a, g);
    }
    __syncthreads();
    for (; j < layer; ++j) {
        relax_layer(a, g, j, false);
        __syncthreads();
        contract(a, g, j);
        __syncthreads();
    }
}

// The decision loss of one box (decision_grad).  The direction is kept from
// the first step of an optimisation; without a direction array it is chosen
// afresh and not kept.
__device__ void decision_loss(const AdjArgs &a, const AdjSmem &s, int64_t pos) {
    const int8_t dir = (a.alpha_mode == kAlphaInit || a.dir == nullptr) ? 0 : a.dir[pos];
    const int8_t got = decision_grad(a.net, s.lo, s.hi, s.glo, s.ghi, dir);
    if (dir == 0 && a.dir != nullptr) a.dir[pos] = got;
}

// Folded-layer weight gradients (R rows) of one box, unfolded with the
// property rows: dW_K = C^T dW', db_K = C^T db'.
__device__ void unfold_add(const AdjArgs &a, const AdjSmem &s, int n_in, float *dW, float *db, int lane, int nl) {
    const int R = a.net.R, no = a.n_out, Q = a.net.d + 1;
    for (int it = lane; it < no * n_in; it += nl) {
        const int o = it / n_in;
        const int i = it - o * n_in;
        float v = 0.f;
        for (int r = 0; r < R; ++r) v = fmaf(__ldg(a.Cprop + r * no + o), s.tmp[r * n_in + i], v);
        atomicAdd(dW + it, v);
    }
    for (int o = lane; o < no; o += nl) {
        float v = 0.f;
        for (int r = 0; r < R; ++r) v = fmaf(__ldg(a.Cprop + r * no + o), s.gA[r * Q + a.net.d], v);
        atomicAdd(db + o, v);
    }
}

}  // namespace

// kGlobal: the boxes' state in global memory (a.gscratch) instead of shared
// memory; two instantiations so that the shared one keeps shared-memory
// instructions.
template <bool kGlobal>
__global__ void __launch_bounds__(256, 2) slr_adjoint_kernel(const AdjArgs a) {
    extern __shared__ __align__(16) float smem_adj[];
    const NetParams<float> &net = a.net;
    const int K = net.K, d = net.d, Q = d + 1, R = net.R, H = a.H;
    const int B = a.boxes_per_cta;
    const size_t stride = adj_box_floats(a);
    float *const state = kGlobal ? a.gscratch + (size_t)blockIdx.x * B * stride : smem_adj;

    int64_t n = a.n;
    if (a.count != nullptr) {
        const int64_t c = (int64_t)*a.count;
        n = c < n ? c : n;
    }
    for (int64_t pos0 = (int64_t)blockIdx.x * B; pos0 < n; pos0 += (int64_t)gridDim.x * B) {
        Group g;
        g.base = state;
        g.stride = stride;
        g.pos0 = pos0;
        g.nb = (int)((n - pos0) < B ? (n - pos0) : B);

        // ---- the boxes: centre and radius (Sec. 2.2 bisection for path codes) ----
        const Div by_d(d, B * d);
        for (int it = threadIdx.x; it < g.nb * d; it += blockDim.x) {
            const int q = by_d(it);
            const int i = it - q * d;
            const AdjSmem s = g.box(a, q);
            const BoxSource &src = a.src;
            const int64_t pos = pos0 + q;
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
            s.m[i] = (float)m64;
            s.r[i] = (float)r64;
        }
        __syncthreads();

        // ---- forward: equations, concrete bounds and slopes of every layer ----
        build_layer1(a, g);
        __syncthreads();
        for (int k = 1; k < K; ++k) {
            concretize_layer(a, g, k);
            __syncthreads();
            relax_layer(a, g, k, false);
            __syncthreads();
            contract(a, g, k);
            __syncthreads();
        }
        // row bounds of the folded last layer and their upstream adjoints
        const Div by_R(R, B * R);
        for (int it = threadIdx.x; it < g.nb * R; it += blockDim.x) {
            const int q = by_R(it);
            const int r = it - q * R;
            const AdjSmem s = g.box(a, q);
            const int64_t pos = pos0 + q;
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
            for (int q = threadIdx.x; q < g.nb; q += blockDim.x) decision_loss(a, g.box(a, q), pos0 + q);
            __syncthreads();
        }
        // d lo_r = d (L_r,d - sum |L_r,c|), d hi_r = d (U_r,d + sum |U_r,c|)
        const Div by_RQ(R * Q, B * R * Q), by_Q(Q, R * Q);
        for (int it = threadIdx.x; it < g.nb * R * Q; it += blockDim.x) {
            const int q = by_RQ(it);
            const int li = it - q * R * Q;
            const int r = by_Q(li);
            const int c = li - r * Q;
            const AdjSmem s = g.box(a, q);
            s.gA[li] = c == d ? s.ghi[r] : s.ghi[r] * sgnf(s.U[li]);
            s.gB[li] = c == d ? s.glo[r] : -s.glo[r] * sgnf(s.L[li]);
        }
        __syncthreads();

        // ---- backward sweep: contraction k maps hidden layer k to layer k + 1 ----
        for (int k = K - 1; k >= 1; --k) {
            const int n_in = net.n[k], n_out = net.n[k + 1];
            const bool kept = k <= a.nck;
            if (!kept) recompute(a, g, k);
            relax_layer(a, g, k, kept);
            // (gU', gL') -> (gC', gR') = (gU' + gL', gU' - gL')
            const Div by_oQ(n_out * Q, B * n_out * Q);
            for (int it = threadIdx.x; it < g.nb * n_out * Q; it += blockDim.x) {
                const int q = by_oQ(it);
                const int li = it - q * n_out * Q;
                const AdjSmem s = g.box(a, q);
                const float u = s.gA[li], l = s.gB[li];
                s.gA[li] = u + l;
                s.gB[li] = u - l;
            }
            __syncthreads();
            // weight and bias gradients: dW[p][i] = sum_c gC'[p,c] C[i,c] + sgn(W) gR'[p,c] Rr[i,c]
            if (a.dW[k] != nullptr) {
                const bool last = k == K - 1;
                const Div by_in(n_in, n_out * n_in);
                for (int it = threadIdx.x; it < n_out * n_in; it += blockDim.x) {
                    const int p = by_in(it);
                    const int i = it - p * n_in;
                    const float sw = sgnf(weight(net, k, p, i));
                    float acc = 0.f;
                    for (int q = 0; q < g.nb; ++q) {
                        const AdjSmem s = g.box(a, q);
                        float v = 0.f;
                        for (int c = 0; c < Q; ++c)
                            v = fmaf(s.gA[p * Q + c], s.C[i * Q + c], fmaf(sw * s.gB[p * Q + c], s.Rr[i * Q + c], v));
                        if (last) s.tmp[it] = v;
                        acc += v;
                    }
                    if (!last) atomicAdd(a.dW[k] + it, acc);
                }
                if (!last) {
                    for (int p = threadIdx.x; p < n_out; p += blockDim.x) {
                        float acc = 0.f;
                        for (int q = 0; q < g.nb; ++q) acc += g.box(a, q).gA[p * Q + d];
                        atomicAdd(a.db[k] + p, acc);
                    }
                } else {
                    __syncthreads();
                    for (int q = 0; q < g.nb; ++q) unfold_add(a, g.box(a, q), n_in, a.dW[k], a.db[k], threadIdx.x,
                                                              blockDim.x);
                }
            }
            // adjoints of the post-relaxation pair: gU^ = (W^T gC' + |W|^T gR') / 2, gL^ = (W^T gC' - |W|^T gR') / 2
            const int nch = (Q + kAdjCols - 1) / kAdjCols;
            const Div by_ich(n_in * nch, B * n_in * nch), by_i(n_in, n_in * nch);
            for (int it = threadIdx.x; it < g.nb * n_in * nch; it += blockDim.x) {
                const int q = by_ich(it);
                const int li = it - q * n_in * nch;
                const int ch = by_i(li);
                const int i = li - ch * n_in;
                const int c0 = ch * kAdjCols;
                const int nc = Q - c0 < kAdjCols ? Q - c0 : kAdjCols;
                const AdjSmem s = g.box(a, q);
                float gc[kAdjCols], gr[kAdjCols];
#pragma unroll
                for (int c = 0; c < kAdjCols; ++c) {
                    gc[c] = 0.f;
                    gr[c] = 0.f;
                }
                for (int p = 0; p < n_out; ++p) {
                    const float w = weight(net, k, p, i);
                    const float aw = fabsf(w);
                    const float *ap = s.gA + p * Q + c0, *bp = s.gB + p * Q + c0;
#pragma unroll
                    for (int c = 0; c < kAdjCols; ++c) {
                        if (c < nc) {
                            gc[c] = fmaf(w, ap[c], gc[c]);
                            gr[c] = fmaf(aw, bp[c], gr[c]);
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < kAdjCols; ++c) {
                    if (c < nc) {
                        s.gX[i * Q + c0 + c] = 0.5f * (gc[c] + gr[c]);
                        s.gY[i * Q + c0 + c] = 0.5f * (gc[c] - gr[c]);
                    }
                }
            }
            __syncthreads();
            // through the relaxation (Eq. 1) of hidden layer k, one neuron per thread
            const int off = hidden_offset(net, k);
            const Div by_j(n_in, B * n_in);
            for (int it = threadIdx.x; it < g.nb * n_in; it += blockDim.x) {
                const int q = by_j(it);
                const int j = it - q * n_in;
                const AdjSmem s = g.box(a, q);
                const int64_t pos = pos0 + q;
                const float *Uk = kept ? chk_u(a, s, k) : s.U;
                const float *Lk = kept ? chk_l(a, s, k) : s.L;
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
                if (a.adam_t > 0 && a.alpha_mode != kAlphaDefault) a.alpha[ai] = adam_slope(a, ai, al, g_alpha);
            }
            __syncthreads();
        }

        // ---- layer 1: U = L = [W_1 diag(r) | W_1 m + b_1] ----
        const int n1 = net.n[1];
        const Div by_1Q(n1 * Q, B * n1 * Q);
        for (int it = threadIdx.x; it < g.nb * n1 * Q; it += blockDim.x) {
            const int q = by_1Q(it);
            const int li = it - q * n1 * Q;
            const AdjSmem s = g.box(a, q);
            s.gA[li] += s.gB[li];
        }
        __syncthreads();
        if (a.dW[0] != nullptr) {
            if (K > 1) {
                for (int it = threadIdx.x; it < n1 * d; it += blockDim.x) {
                    const int p = it / d;
                    const int i = it - p * d;
                    float acc = 0.f;
                    for (int q = 0; q < g.nb; ++q) {
                        const AdjSmem s = g.box(a, q);
                        acc += fmaf(s.gA[p * Q + i], s.r[i], s.gA[p * Q + d] * s.m[i]);
                    }
                    atomicAdd(a.dW[0] + it, acc);
                }
                for (int p = threadIdx.x; p < n1; p += blockDim.x) {
                    float acc = 0.f;
                    for (int q = 0; q < g.nb; ++q) acc += g.box(a, q).gA[p * Q + d];
                    atomicAdd(a.db[0] + p, acc);
                }
            } else {
                // a single affine layer is the folded one: unfold with the property rows
                for (int q = 0; q < g.nb; ++q) {
                    const AdjSmem s = g.box(a, q);
                    for (int it = threadIdx.x; it < R * d; it += blockDim.x) {
                        const int r = it / d;
                        const int i = it - r * d;
                        s.tmp[it] = fmaf(s.gA[r * Q + i], s.r[i], s.gA[r * Q + d] * s.m[i]);
                    }
                }
                __syncthreads();
                for (int q = 0; q < g.nb; ++q) unfold_add(a, g.box(a, q), d, a.dW[0], a.db[0], threadIdx.x,
                                                          blockDim.x);
            }
        }
        if (a.d_lo != nullptr) {
            for (int it = threadIdx.x; it < g.nb * d; it += blockDim.x) {
                const int q = by_d(it);
                const int i = it - q * d;
                const AdjSmem s = g.box(a, q);
                const int64_t pos = pos0 + q;
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
        if (a.d_r != nullptr) {
            for (int it = threadIdx.x; it < g.nb * d; it += blockDim.x) {
                const int q = by_d(it);
                const int i = it - q * d;
                const AdjSmem s = g.box(a, q);
                float gr = 0.f;
                for (int p = 0; p < n1; ++p) gr = fmaf(s.gA[p * Q + i], weight(net, 0, p, i), gr);
                a.d_r[(pos0 + q) * d + i] = gr;
            }
        }
        if (a.split_codes != nullptr) {
            // split the dimension whose halving is predicted to lower the loss
            // most: the largest |dM/dr_i| r_i over the split set
            for (int q = threadIdx.x; q < g.nb; q += blockDim.x) {
                const int64_t pos = pos0 + q;
                const int64_t idx = a.src.index != nullptr ? a.src.index[pos] : pos;
                if (a.split_cls[idx] != kUndecided) continue;
                const AdjSmem s = g.box(a, q);
                int sel = 0;
                float best = -1.f;
                for (int j = 0; j < a.n_split; ++j) {
                    const int i = a.split_dims[j];
                    float gr = 0.f;
                    for (int p = 0; p < n1; ++p) gr = fmaf(s.gA[p * Q + i], weight(net, 0, p, i), gr);
                    const float score = fabsf(gr) * s.r[i];
                    if (score > best) {
                        best = score;
                        sel = j;
                    }
                }
                a.split_codes[idx] |= (unsigned long long)sel << (kSplitPathBits + 4 * a.src.t);
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

// Keeps the listed boxes (positions p < *n_in of lo, hi) whose decision gap
// (the smaller of the SAFE gap sum_c max(0, min_{r in c} hi_r) and the UNSAFE
// gap min_c max(0, -min_{r in c} lo_r)) is at most tau times the widest
// hi_r - lo_r of the box; appends their frontier indices list_in[p] to
// list_out (order across warps unspecified).
__global__ void slr_margin_filter_kernel(const NetParams<float> net, const float *lo, const float *hi,
                                         const unsigned long long *n_in, int64_t cap, const int64_t *list_in,
                                         int64_t *list_out, unsigned long long *n_out, float tau) {
    int64_t n = (int64_t)*n_in;
    n = n < cap ? n : cap;
    const int R = net.R;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t p = base + threadIdx.x;
        bool keep = false;
        if (p < n) {
            const float *l = lo + p * R, *h = hi + p * R;
            float safe_gap = 0.f, unsafe_gap = INFINITY, width = 0.f;
            int r0 = 0;
            for (int c = 0; c < net.n_clauses; ++c) {
                const int r1 = net.clause_end[c];
                float mh = INFINITY, ml = INFINITY;
                for (int r = r0; r < r1; ++r) {
                    mh = fminf(mh, h[r]);
                    ml = fminf(ml, l[r]);
                    width = fmaxf(width, h[r] - l[r]);
                }
                safe_gap += fmaxf(mh, 0.f);
                unsafe_gap = fminf(unsafe_gap, fmaxf(-ml, 0.f));
                r0 = r1;
            }
            keep = fminf(safe_gap, unsafe_gap) <= tau * width;
        }
        const unsigned ballot = __ballot_sync(0xffffffffu, keep);
        if (ballot == 0u) continue;
        unsigned long long start = 0;
        if (lane == 0) start = atomicAdd(n_out, (unsigned long long)__popc(ballot));
        start = __shfl_sync(0xffffffffu, start, 0);
        if (keep) list_out[start + __popc(ballot & ((1u << lane) - 1u))] = list_in[p];
    }
}

size_t adjoint_box_bytes(const AdjArgs &a) { return sizeof(float) * adj_box_floats(a); }

size_t adjoint_smem_bytes(const AdjArgs &a) {
    return a.gscratch != nullptr ? 0 : sizeof(float) * adj_box_floats(a) * (size_t)a.boxes_per_cta;
}


cudaError_t launch_adjoint(const AdjArgs &a, int grid, cudaStream_t s) {
    if (a.gscratch != nullptr) {
        slr_adjoint_kernel<true><<<grid, 256, 0, s>>>(a);
        return cudaGetLastError();
    }
    const size_t smem = adjoint_smem_bytes(a);
    cudaError_t e = cudaFuncSetAttribute(slr_adjoint_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    slr_adjoint_kernel<false><<<grid, 256, smem, s>>>(a);
    return cudaGetLastError();
}

int adjoint_blocks_per_sm(size_t smem) {
    int nb = 0;
    cudaFuncSetAttribute(slr_adjoint_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, slr_adjoint_kernel<false>, 256, smem) != cudaSuccess)
        return 0;
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

cudaError_t launch_margin_filter(const NetParams<float> &net, const float *lo, const float *hi,
                                 const unsigned long long *n_in, int64_t cap, const int64_t *list_in,
                                 int64_t *list_out, unsigned long long *n_out, float tau, int grid, cudaStream_t s) {
    slr_margin_filter_kernel<<<grid, 256, 0, s>>>(net, lo, hi, n_in, cap, list_in, list_out, n_out, tau);
    return cudaGetLastError();
}

}  // namespace slr
