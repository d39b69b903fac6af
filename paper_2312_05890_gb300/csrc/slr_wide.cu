// Wide networks: the SLR state of a chunk of boxes lives in HBM and every
// affine layer is one batched GEMM on the tensor cores.
//
// For networks whose per-box state does not fit a shared-memory tile (many
// inputs, wide layers: Sec. 3 notes that SLR's memory grows with the number of
// input nodes), each box keeps, per neuron p of the current layer,
//   C[b][j][p]  j < d        centre-equation coefficients (normalised input),
//   Rr[b][j][p] j < d + 3    radius coefficients, radius constant, N (row
//                            magnitude) and E (rounding-error bound),
//   Ch[b][p], Cl[b][p]       centre constant as a float-float pair,
// with neurons the fastest index (row stride NP, a multiple of 32).  Each
// column (b, j) is then a K-major operand of the next layer's product
//   C' = W C   (M = n_out, K = n_in, N = boxes x d columns),
//   R' = |W| R (N = boxes x (d + 3) columns, R, N and E together),
// computed by `wide_gemm_kernel` with tcgen05 (kind::tf32) in three-term split
// precision: x = hi + lo in TF32 pieces, products lo*hi + hi*lo + hi*hi
// accumulated in FP32 in tensor memory, covered in E by gamma_tc(K) of
// sum |W| N like the tile kernel's tensor-core path.  The constants (one
// column) take the float-float route on the CUDA cores (`wide_const_kernel`),
// and `wide_hidden_kernel` applies the error update, the concrete bounds and
// the ReLU relaxation (Eq. 1) row by row in place, with the same code as the
// tile kernel (EvalTile::relax_row).
#include <algorithm>

#include "slr_eval.cuh"
#include "slr_kernels.h"
#include "slr_tc_util.cuh"

namespace slr {

using namespace tc;

namespace {

using WTile = EvalTile<float, 1, 1>;   // only its static row helpers are used

constexpr int kWN = 256;                          // GEMM tile: columns
constexpr int kWM = 128;                          // rows (tensor-memory lanes)
constexpr int kWK = 16;                           // K per pipeline stage (two stages: 108 KB, 2 CTAs per SM)
constexpr int kWQ = kWK / 4;                      // float4 of one operand row per stage
constexpr int kWSbo = (kWK / 4) * kTcLbo;         // bytes between 8-row core-matrix groups
constexpr int kWABytes = (kWM / 8) * kWSbo;       // one A piece of a stage
constexpr int kWBBytes = (kWN / 8) * kWSbo;       // one B piece of a stage
constexpr int kWStage = 2 * kWABytes + 2 * kWBBytes;
constexpr int kWThreads = 256;

// One row (box b, neuron p) of the HBM state, with the tile kernel's column numbering.
struct WideRow {
    float *C, *Rr, *Ch, *Cl;
    int64_t b;
    int p, d, NP;
    __device__ __forceinline__ float &operator()(int c) const {
        if (c < d) return C[((size_t)b * d + c) * NP + p];
        if (c == d) return Ch[(size_t)b * NP + p];
        if (c == 2 * d + 4) return Cl[(size_t)b * NP + p];
        return Rr[((size_t)b * (d + 3) + (c - d - 1)) * NP + p];
    }
};

__device__ __forceinline__ int wboff(int r, int k) { return (r >> 3) * kWSbo + (k >> 2) * kTcLbo + (r & 7) * 16; }

}  // namespace

// ---------------------------------------------------------------------------
// Boxes of the chunk: centre (float-float) and radius, outward (Sec. 2.2).
// ---------------------------------------------------------------------------
__global__ void wide_box_kernel(const BoxSource src, int64_t base, int nb, int d, float *mh, float *ml, float *rr,
                                int64_t *bidx) {
    for (int64_t item = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; item < (int64_t)nb * d;
         item += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(item / d);
        const int i = (int)(item - (int64_t)b * d);
        const int64_t k = base + b;
        const int64_t idx = src.index != nullptr ? src.index[k] : k;
        double m64, r64, pad;
        if (src.mode == 0) {
            unsigned long long kk;
            int c;
            code_dim(src, src.codes[idx], i, kk, c);
            const double w = src.root_w[i];
            const double a = src.root_lo[i];
            r64 = ldexp(w, -(c + 1));
            m64 = a + w * ldexp((double)(2 * kk + 1), -(c + 1));
            pad = ldexp(fabs(m64) + fabs(a) + w, -50);
        } else {
            const double lo = (double)src.lo[idx * d + i];
            const double hi = (double)src.hi[idx * d + i];
            m64 = 0.5 * (lo + hi);
            r64 = 0.5 * (hi - lo);
            pad = ldexp(fabs(m64) + fabs(r64), -52);
        }
        float h, l, r;
        split_centre<float>(m64, r64, pad, h, l, r);
        mh[item] = h;
        ml[item] = l;
        rr[item] = r;
        if (i == 0) bidx[b] = idx;
    }
}

// ---------------------------------------------------------------------------
// Row kernels: a block is 32 rows (threadIdx.x) of one box (blockIdx.y) with
// the d coefficients of each row split over 16 slices (threadIdx.y), so that a
// warp reads 32 consecutive neurons of one coefficient column.  The slices'
// partial sums are merged in shared memory, one thread per row plans the
// relaxation, and all slices apply it.
// ---------------------------------------------------------------------------
constexpr int kRowsX = 32, kSlicesY = 16;

// Layer 1: C = [W_1 diag(r) | W_1 m + b_1], R = 0 (Sec. 3), then its ReLU
// relaxation when it is a hidden layer.  W0t: W_1 transposed (d x n_1).
// The coefficients c_j = W_1[p][j] r_j are formed twice, bit for bit the same:
// for the concrete bounds, then, once the plan is known, to be stored as
// relaxed (one write per value).  The constant's terms W_1[p][j] m_j are
// summed in the slices' share (error-free products, compensated sums), and
// the 16 partial pairs added by TwoSum with their error terms in float: a
// summation tree whose partial sums add up to no more than the sequential
// chain's, so the chain's bound 2 gamma_{d+2}^2 (1 + gamma_d) sum |p_j| holds.
__global__ void __launch_bounds__(kRowsX * kSlicesY)
wide_init_kernel(const NetParams<float> net, const float *W0t, int NP, const float *mh, const float *ml,
                 const float *rr, float *C, float *Rr, float *Ch, float *Cl, const float *alpha, int64_t alpha_ld,
                 int64_t base) {
    using A = Arith<float>;
    __shared__ RowBounds<float> part[kSlicesY][kRowsX];
    __shared__ float cpart[3][kSlicesY][kRowsX];
    __shared__ RelaxPlan<float> plan[kRowsX];
    const int d = net.d;
    const int n1 = net.n[1];
    const int lane = threadIdx.x, sl = threadIdx.y;
    const int p = blockIdx.x * kRowsX + lane;
    const int64_t b = blockIdx.y;
    const bool live = p < n1;
    const WideRow R{C, Rr, Ch, Cl, b, live ? p : 0, d, NP};
    const float *rb = rr + b * d;
    const float *mb = mh + b * d, *lb = ml + b * d;
    RowBounds<float> bd;
    bd.reset();
    float s = 0.f, e = 0.f, sabs = 0.f;
    if (live) {
        if (sl == 0) {
            s = net.b[0][p];
            sabs = fabsf(s);
        }
#pragma unroll 4
        for (int j = sl; j < d; j += kSlicesY) {
            const float wj = W0t[(size_t)j * n1 + p];
            bd.add(A::mul_rn(wj, rb[j]), 0.f);
            float p1, pe, tt, se;
            two_prod<float>(wj, mb[j], p1, pe);
            two_sum<float>(s, p1, tt, se);
            s = tt;
            e = A::fma_rn(wj, lb[j], e + (pe + se));
            sabs = sabs + fabsf(p1);
        }
    }
    part[sl][lane] = bd;
    cpart[0][sl][lane] = s;
    cpart[1][sl][lane] = e;
    cpart[2][sl][lane] = sabs;
    __syncthreads();
    if (sl == 0 && live) {
        RowBounds<float> t = part[0][lane];
        for (int y = 1; y < kSlicesY; ++y) t.merge(part[y][lane]);
        // the constant W_1 m + b_1: the slices' partial pairs, in slice order
        for (int y = 1; y < kSlicesY; ++y) {
            float tt, se;
            two_sum<float>(s, cpart[0][y][lane], tt, se);
            s = tt;
            e = e + (cpart[1][y][lane] + se);
            sabs = sabs + cpart[2][y][lane];
        }
        float chi, clo;
        two_sum<float>(s, e, chi, clo);
        const float S1 = t.NC;
        const float g = gam<float>(d + 2);
        float E = A::add_up(uerr<float>(S1), A::mul_up(A::mul_up(2.f * g, g), A::mul_up(sabs, 1.f + gam<float>(d))));
        E = A::add_up(E, (float)(d + 4) * A::tiny);
        if (net.K == 1) {
            // folded property layer applied to x itself: |x_j| <= |m_j| + r_j
            float fe = net.fold_berr[p];
            for (int j = 0; j < d; ++j) {
                const float xm = A::add_up(A::add_up(fabsf(mh[b * d + j]), fabsf(ml[b * d + j])), rb[j]);
                fe = A::add_up(fe, A::mul_up(net.fold_err[p * d + j], xm));
            }
            E = A::add_up(E, fe);
        }
        RelaxPlan<float> pl;
        pl.kind = 0;
        pl.pp = 1.f;
        pl.qq = 0.f;
        pl.nh = chi;
        pl.nl = clo;
        pl.rd = 0.f;
        pl.N = S1;
        pl.E = E;
        if (net.K > 1) {
            t.finish(chi, clo, 0.f);
            const float *a_ptr = alpha != nullptr ? alpha + (base + b) * alpha_ld + p : nullptr;
            pl = WTile::plan_row(t, d, net.relax_mode, chi, clo, 0.f, E, a_ptr, net.act[0]);
        }
        plan[lane] = pl;
    }
    __syncthreads();
    if (live) {
        const RelaxPlan<float> pl = plan[lane];
#pragma unroll 4
        for (int j = sl; j < d; j += kSlicesY) {
            float c = pl.kind == 1 ? 0.f : A::mul_rn(W0t[(size_t)j * n1 + p], rb[j]), r = 0.f;
            WTile::apply_plan(pl, c, r);
            R(j) = c;
            R(WTile::cR(d) + j) = r;
        }
        if (sl == 0) {
            R(WTile::cCh(d)) = pl.nh;
            R(WTile::cCl(d)) = pl.nl;
            R(WTile::cRd(d)) = pl.rd;
            R(WTile::cN(d)) = pl.N;
            R(WTile::cE(d)) = pl.E;
        }
    }
}

// ---------------------------------------------------------------------------
// Constants of layer k + 1: sum_i W[p][i] (Ch_i + Cl_i) + b_p, error-free
// products and compensated sums, with the error bound (and, for the folded
// property layer, the rounding of the folded weights).
// ---------------------------------------------------------------------------
__global__ void wide_const_kernel(const NetParams<float> net, int k, int nb, int NP, const float *Ch, const float *Cl,
                                  const float *Rr, float *Kh, float *Kl, float *Ke) {
    using A = Arith<float>;
    const int d = net.d;
    const int n_in = net.n[k];
    const int n_out = net.n[k + 1];
    const bool last = k + 1 == net.K;
    const float *Wt = net.Wt[k];
    for (int64_t item = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; item < (int64_t)nb * n_out;
         item += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = item / n_out;
        const int p = (int)(item - b * n_out);
        float s = net.b[k][p], e = 0.f, a = fabsf(s), f = 0.f;
        for (int i = 0; i < n_in; ++i) {
            const float w = Wt[(size_t)i * n_out + p];
            const float h = Ch[b * NP + i];
            const float l = Cl[b * NP + i];
            float p1, pe, t, se;
            two_prod<float>(w, h, p1, pe);
            two_sum<float>(s, p1, t, se);
            s = t;
            e = A::fma_rn(w, l, e + (pe + se));
            a = a + fabsf(p1);
            if (last) {
                const float nN = Rr[((size_t)b * (d + 3) + d + 1) * NP + i];
                const float nE = Rr[((size_t)b * (d + 3) + d + 2) * NP + i];
                const float z = A::add_up(A::add_up(fabsf(nN), fabsf(h)), A::add_up(fabsf(l), fabsf(nE)));
                f = A::add_up(f, A::mul_up(net.fold_err[p * n_in + i], z));
            }
        }
        const float g = gam<float>(n_in + 2);
        const float g2 = A::mul_up(2.f * g, g);
        float hi, lo;
        two_sum<float>(s, e, hi, lo);
        float err = A::mul_up(g2, A::mul_up(a, 1.f + gam<float>(n_in)));
        if (last) err = A::add_up(err, A::add_up(f, net.fold_berr[p]));
        Kh[b * NP + p] = hi;
        Kl[b * NP + p] = lo;
        Ke[b * NP + p] = err;
    }
}

namespace {

// The contraction's constant and error (E' = |W| E (1 + 2 g) + g |W| N (1 + g) + constant error).
__device__ __forceinline__ void wide_finish(const WideRow &R, const float *Kh, const float *Kl, const float *Ke,
                                            int NP, int n_in, float gcoef, float &chi, float &clo, float &E) {
    using A = Arith<float>;
    const int d = R.d;
    chi = Kh[R.b * NP + R.p];
    clo = Kl[R.b * NP + R.p];
    const float wN = R(WTile::cN(d));
    float eps = A::mul_up(gcoef, A::mul_up(wN, 1.f + gcoef));
    eps = A::add_up(A::add_up(eps, Ke[R.b * NP + R.p]), (float)(n_in + 4) * A::tiny);
    E = A::add_up(A::mul_up(R(WTile::cE(d)), 1.f + 2.f * gcoef), eps);
}

}  // namespace

// Hidden layer `layer` after its product: error, bounds, ReLU relaxation in place.
// A block is 128 rows of one box: each thread holds four neighbouring rows
// (one float4 of every coefficient column: 512-byte accesses per warp) for
// its eighth of the d columns; the slices' partial bounds are merged in
// shared memory, one thread per row plans the relaxation, and every thread
// applies its rows' plans, reading and writing a float4 only where a row
// changes.  Rows from n to the next multiple of 4 lie inside the row stride
// and are planned as zero rows (nothing reads them).
constexpr int kH4X = 32, kH4Y = 8, kH4Rows = 4 * kH4X;

__global__ void __launch_bounds__(kH4X * kH4Y, 2)
wide_hidden_kernel(const NetParams<float> net, int layer, int NP, float gcoef, float *C, float *Rr, float *Ch,
                   float *Cl, const float *Kh, const float *Kl, const float *Ke, const float *alpha, int64_t alpha_ld,
                   int64_t base) {
    __shared__ RowBounds<float> part[kH4Y][kH4Rows];
    __shared__ RelaxPlan<float> plan[kH4Rows];
    const int d = net.d;
    const int n = net.n[layer];
    const int n_in = net.n[layer - 1];
    const int lane = threadIdx.x, sl = threadIdx.y;
    const int pb = blockIdx.x * kH4Rows;
    const int p0 = pb + 4 * lane;
    const int64_t b = blockIdx.y;
    const bool any = p0 < n;
    float *Cb = C + (size_t)b * d * NP + p0;
    float *Rb = Rr + (size_t)b * (d + 3) * NP + p0;
    RowBounds<float> bd[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) bd[u].reset();
    if (any) {
#pragma unroll 4
        for (int j = sl; j < d; j += kH4Y) {
            const float4 c = *reinterpret_cast<const float4 *>(Cb + (size_t)j * NP);
            const float4 r = *reinterpret_cast<const float4 *>(Rb + (size_t)j * NP);
            bd[0].add(c.x, r.x);
            bd[1].add(c.y, r.y);
            bd[2].add(c.z, r.z);
            bd[3].add(c.w, r.w);
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) part[sl][4 * lane + u] = bd[u];
    __syncthreads();
    if (sl < kH4Rows / kH4X) {
        const int rr = sl * kH4X + lane;
        const int p = pb + rr;
        RelaxPlan<float> pl;
        pl.kind = 1;
        pl.pp = pl.qq = 0.f;
        pl.nh = pl.nl = pl.rd = pl.N = pl.E = 0.f;
        if (p < n) {
            const WideRow R{C, Rr, Ch, Cl, b, p, d, NP};
            RowBounds<float> t = part[0][rr];
            for (int y = 1; y < kH4Y; ++y) t.merge(part[y][rr]);
            float chi, clo, E;
            wide_finish(R, Kh, Kl, Ke, NP, n_in, gcoef, chi, clo, E);
            const float rd = R(WTile::cRd(d));
            t.finish(chi, clo, rd);
            const float *a_ptr = nullptr;
            if (alpha != nullptr) {
                int off = 0;
                for (int j = 1; j < layer; ++j) off += net.n[j];
                a_ptr = alpha + (base + b) * alpha_ld + off + p;
            }
            pl = WTile::plan_row(t, d, net.relax_mode, chi, clo, rd, E, a_ptr, net.act[layer - 1]);
            R(WTile::cCh(d)) = pl.nh;
            R(WTile::cCl(d)) = pl.nl;
            R(WTile::cRd(d)) = pl.rd;
            R(WTile::cN(d)) = pl.N;
            R(WTile::cE(d)) = pl.E;
        }
        plan[rr] = pl;
    }
    __syncthreads();
    if (any) {
        RelaxPlan<float> pl[4];
        bool keep = false, zero = false, mix = false;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            pl[u] = plan[4 * lane + u];
            keep = keep || pl[u].kind == 0;
            zero = zero || pl[u].kind == 1;
            mix = mix || pl[u].kind == 2;
        }
        // a float4 is read when a row's values are needed (kept beside changed
        // rows, or mixed by the plan) and written when some row changes
        const bool load = mix || (keep && zero);
        if (zero || mix) {
#pragma unroll 4
            for (int j = sl; j < d; j += kH4Y) {
                float4 c = make_float4(0.f, 0.f, 0.f, 0.f), r = c;
                if (load) {
                    c = *reinterpret_cast<const float4 *>(Cb + (size_t)j * NP);
                    r = *reinterpret_cast<const float4 *>(Rb + (size_t)j * NP);
                }
                WTile::apply_plan(pl[0], c.x, r.x);
                WTile::apply_plan(pl[1], c.y, r.y);
                WTile::apply_plan(pl[2], c.z, r.z);
                WTile::apply_plan(pl[3], c.w, r.w);
                *reinterpret_cast<float4 *>(Cb + (size_t)j * NP) = c;
                *reinterpret_cast<float4 *>(Rb + (size_t)j * NP) = r;
            }
        }
    }
}

// Property rows: sound bounds lo = min L' - E, hi = max U' + E (Sec. 3 check).
__global__ void __launch_bounds__(kRowsX * kSlicesY)
wide_final_kernel(const NetParams<float> net, int NP, float gcoef, float *C, float *Rr, float *Ch, float *Cl,
                  const float *Kh, const float *Kl, const float *Ke, float *lo, float *hi, float *err) {
    using A = Arith<float>;
    __shared__ RowBounds<float> part[kSlicesY][kRowsX];
    const int d = net.d;
    const int R = net.R;
    const int n_in = net.n[net.K - 1];
    const int lane = threadIdx.x, sl = threadIdx.y;
    const int r = blockIdx.x * kRowsX + lane;
    const int64_t b = blockIdx.y;
    const bool live = r < R;
    const WideRow Rw{C, Rr, Ch, Cl, b, live ? r : 0, d, NP};
    RowBounds<float> bd;
    bd.reset();
    if (live)
#pragma unroll 8
        for (int j = sl; j < d; j += kSlicesY) bd.add(Rw(j), Rw(WTile::cR(d) + j));
    part[sl][lane] = bd;
    __syncthreads();
    if (sl == 0 && live) {
        RowBounds<float> t = part[0][lane];
        for (int y = 1; y < kSlicesY; ++y) t.merge(part[y][lane]);
        float chi, clo, E;
        if (net.K > 1) {
            wide_finish(Rw, Kh, Kl, Ke, NP, n_in, gcoef, chi, clo, E);
        } else {
            chi = Rw(WTile::cCh(d));
            clo = Rw(WTile::cCl(d));
            E = Rw(WTile::cE(d));
        }
        t.finish(chi, clo, Rw(WTile::cRd(d)));
        lo[b * R + r] = A::add_dn(t.ll, -E);
        hi[b * R + r] = A::add_up(t.uu, E);
        err[b * R + r] = A::add_up(E, t.delta);
    }
}

namespace {

__device__ __forceinline__ uint8_t wide_class(const NetParams<float> &net, const float *lo, const float *hi,
                                              const float *err, float shift) {
    bool any_in = false, all_out = true;
    int r0 = 0;
    for (int cl = 0; cl < net.n_clauses; ++cl) {
        const int r1 = net.clause_end[cl];
        bool all_in = true, some_out = false;
        for (int r = r0; r < r1; ++r) {
            const float e2 = shift * err[r];
            const float l = lo[r] + e2;
            const float h = hi[r] - e2;
            const bool st = net.strict[r] != 0;
            all_in = all_in && (st ? (l > 0.f) : (l >= 0.f));
            some_out = some_out || (st ? (h <= 0.f) : (h < 0.f));
        }
        any_in = any_in || all_in;
        all_out = all_out && some_out;
        r0 = r1;
    }
    return any_in ? kUnsafe : (all_out ? kSafe : kUndecided);
}

}  // namespace

// Class of each box of the chunk (Sec. 3 check) and the outputs.  Boxes whose
// class depends on E (their optimistic class differs) stay UNDECIDED and are
// counted in tie_count: the wide path has no FP64 re-check.
__global__ void wide_classify_kernel(const NetParams<float> net, int nb, int64_t base, const float *lo,
                                     const float *hi, const float *err, const int64_t *bidx, const EvalOutputs out) {
    const int R = net.R;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const float *l = lo + (size_t)b * R, *h = hi + (size_t)b * R, *e = err + (size_t)b * R;
        const uint8_t cls = wide_class(net, l, h, e, 0.f);
        const uint8_t opt = wide_class(net, l, h, e, 2.f);
        const int64_t oidx = out.by_position ? base + b : bidx[b];
        if (out.cls != nullptr) out.cls[oidx] = cls;
        if (out.row_lo != nullptr) {
            for (int r = 0; r < R; ++r) {
                out.row_lo[oidx * R + r] = l[r];
                out.row_hi[oidx * R + r] = h[r];
            }
        }
        if (out.row_err != nullptr)
            for (int r = 0; r < R; ++r) out.row_err[oidx * R + r] = e[r];
        if (cls == kUndecided && opt != kUndecided) {
            // the class depends on the widening: to the FP64 re-check if there
            // is one, else counted as a tie
            if (out.near_list != nullptr) {
                const unsigned long long pos = atomicAdd(out.near_count, 1ull);
                if ((int64_t)pos < out.near_cap) out.near_list[pos] = bidx[b];
                else atomicOr(out.status, kStatusNearOverflow);
            } else if (out.tie_count != nullptr) {
                atomicAdd(out.tie_count, 1ull);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// D[col][m] = sum_k A[m][k] B[col][k] for m < M, col < ncols: one 128 x 256
// tile per CTA, K in stages of 32 (two stages in shared memory, loads of the
// next stage overlapping the tensor core), accumulator in tensor memory.
// ---------------------------------------------------------------------------
// Operands of one K stage, held in registers between their global loads and
// their shared-memory stores (the loads of stage c + 1 are in flight while
// stage c is stored and multiplied).
struct WideStageRegs {
    float4 ah[kWM * kWK / 4 / kWThreads], al[kWM * kWK / 4 / kWThreads];
    float4 b[kWN * kWK / 4 / kWThreads];
};

__device__ __forceinline__ void wide_load_stage(const WideGemm &G, int m0, int n0, int k0, int tid, WideStageRegs &r) {
#pragma unroll
    for (int u = 0; u < kWM * kWK / 4 / kWThreads; ++u) {
        const int q = tid + u * kWThreads;
        const size_t g = (size_t)(m0 + q / kWQ) * G.Kpad + k0 + (q % kWQ) * 4;
        r.ah[u] = __ldg(reinterpret_cast<const float4 *>(G.Ahi + g));
        r.al[u] = __ldg(reinterpret_cast<const float4 *>(G.Alo + g));
    }
#pragma unroll
    for (int u = 0; u < kWN * kWK / 4 / kWThreads; ++u) {
        const int q = tid + u * kWThreads;
        const int col = n0 + q / kWQ;
        const int k = k0 + (q % kWQ) * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (col < G.ncols) {
            const float *src = G.B + (size_t)col * G.ldb + k;
            if (k + 3 < G.K) {
                v = *reinterpret_cast<const float4 *>(src);
            } else {
                if (k < G.K) v.x = src[0];
                if (k + 1 < G.K) v.y = src[1];
                if (k + 2 < G.K) v.z = src[2];
            }
        }
        r.b[u] = v;
    }
}

__device__ __forceinline__ void wide_store_stage(unsigned char *st, int tid, const WideStageRegs &r) {
    unsigned char *sAh = st, *sAl = st + kWABytes, *sBh = st + 2 * kWABytes, *sBl = st + 2 * kWABytes + kWBBytes;
#pragma unroll
    for (int u = 0; u < kWM * kWK / 4 / kWThreads; ++u) {
        const int q = tid + u * kWThreads;
        const int o = wboff(q / kWQ, (q % kWQ) * 4);
        *reinterpret_cast<float4 *>(sAh + o) = r.ah[u];
        *reinterpret_cast<float4 *>(sAl + o) = r.al[u];
    }
#pragma unroll
    for (int u = 0; u < kWN * kWK / 4 / kWThreads; ++u) {
        const int q = tid + u * kWThreads;
        const int o = wboff(q / kWQ, (q % kWQ) * 4);
        const float4 v = r.b[u];
        float4 h, l;
        h.x = tf32_rna(v.x);
        h.y = tf32_rna(v.y);
        h.z = tf32_rna(v.z);
        h.w = tf32_rna(v.w);
        l.x = tf32_rna(v.x - h.x);
        l.y = tf32_rna(v.y - h.y);
        l.z = tf32_rna(v.z - h.z);
        l.w = tf32_rna(v.w - h.w);
        *reinterpret_cast<float4 *>(sBh + o) = h;
        *reinterpret_cast<float4 *>(sBl + o) = l;
    }
}

__global__ void __launch_bounds__(kWThreads, 2) wide_gemm_kernel(const WideGemmArgs args, int gy) {
    extern __shared__ __align__(1024) unsigned char smem_w[];
    const WideGemm &G = args.g[blockIdx.z];
    // the M tiles of one column block are neighbours in the launch order, so
    // the second reads the B columns from L2
    const int n0 = (blockIdx.x / gy) * kWN;
    const int m0 = (blockIdx.x % gy) * kWM;
    if (n0 >= G.ncols || m0 >= G.M) return;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_w + 2 * kWStage);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem_w + 2 * kWStage + 2 * sizeof(uint64_t));
    int *sAbort = reinterpret_cast<int *>(smem_w + 2 * kWStage + 2 * sizeof(uint64_t) + 4);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
        *sAbort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kWN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const int wait_limit = 1 << 24;
    // kind::tf32, FP32 accumulate, both operands K-major, N = 256, M = 128
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kWN >> 3) << 17) |
                           ((uint32_t)(kWM >> 4) << 24);
    const int nch = G.Kpad / kWK;
    bool ok = true;
    WideStageRegs regs;
    if (nch > 0) wide_load_stage(G, m0, n0, 0, tid, regs);
    for (int c = 0; c < nch; ++c) {
        const int s = c & 1;
        unsigned char *st = smem_w + s * kWStage;
        unsigned char *sAh = st, *sAl = st + kWABytes, *sBh = st + 2 * kWABytes, *sBl = st + 2 * kWABytes + kWBBytes;
        if (c >= 2 && ok) {
            // the products of stage s issued two chunks ago have finished reading it
            if (!mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((c - 2) >> 1) & 1), wait_limit)) ok = false;
        }
        if (!ok) atomicExch(sAbort, 1);
        if (ok) wide_store_stage(st, tid, regs);
        if (c + 1 < nch) wide_load_stage(G, m0, n0, (c + 1) * kWK, tid, regs);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (*sAbort) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t pa[3] = {smem_u32(sAh), smem_u32(sAl), smem_u32(sAh)};
            const uint32_t pb[3] = {smem_u32(sBl), smem_u32(sBh), smem_u32(sBh)};
            for (int step = 0; step < kWK / 8; ++step) {
                for (int ps = 0; ps < 3; ++ps) {
                    const uint64_t da = umma_desc(pa[ps] + step * 2 * kTcLbo, kTcLbo, kWSbo);
                    const uint64_t db = umma_desc(pb[ps] + step * 2 * kTcLbo, kTcLbo, kWSbo);
                    const uint32_t acc = (c > 0 || step > 0 || ps > 0) ? 1u : 0u;
                    asm volatile(
                        "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(tmem),
                        "l"(da), "l"(db), "r"(idesc), "r"(acc));
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&mbar[s]))
                : "memory");
        }
    }
    // the last commit covers every product issued before it
    if (!*sAbort && nch > 0) {
        const int cl = nch - 1;
        if (!mbar_wait(smem_u32(&mbar[cl & 1]), (uint32_t)((cl >> 1) & 1), wait_limit)) atomicExch(sAbort, 1);
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (!*sAbort) {
        const int quad = warp & 3;
        const int half = warp >> 2;
        const int m = m0 + quad * 32 + lane;
        // 32 accumulator columns per read, one wait per read
        for (int cc = 0; cc < kWN / 2; cc += 32) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * (kWN / 2) + cc);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (m < G.M) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = n0 + half * (kWN / 2) + cc + j;
                    if (col < G.ncols) G.D[(size_t)col * G.ldd + m] = __uint_as_float(r[j]);
                }
            }
        }
    } else if (tid == 0) {
        atomicOr(args.status, kStatusTimeout);
        // a timed-out product may still be running: give it a bounded chance to finish
        for (int s = 0; s < 2; ++s) mbar_wait(smem_u32(&mbar[s]), 0u, wait_limit);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWN));
}

size_t wide_gemm_smem_bytes() { return 2 * (size_t)kWStage + 64; }

// The property layer's products on the CUDA cores: with at most 16 rows a
// tensor-core tile (M = 128) would be mostly padding.  Column `col` of B (the
// n_in values at B + col * ldb) times the weights (Wt: n_in x R, input-major;
// |W| when abs_w) into D[col * ldd + r], r < R, each a plain FP32 FMA chain
// over the inputs in order (rounding within gamma_{n_in} of sum |W| |x|).
template <int RM>
__global__ void __launch_bounds__(256)
wide_rows_product_kernel(const float *__restrict__ Wt, int n_in, int R, const float *__restrict__ B, int ldb,
                         float *__restrict__ D, int ldd, int64_t ncols, int abs_w) {
    extern __shared__ float sWt[];   // n_in x RM, zero beyond R
    for (int q = threadIdx.x; q < n_in * RM; q += blockDim.x) {
        const int i = q / RM, r = q - i * RM;
        const float w = r < R ? Wt[(size_t)i * R + r] : 0.f;
        sWt[q] = abs_w ? fabsf(w) : w;
    }
    __syncthreads();
    for (int64_t col = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; col < ncols;
         col += (int64_t)gridDim.x * blockDim.x) {
        float acc[RM];
#pragma unroll
        for (int r = 0; r < RM; ++r) acc[r] = 0.f;
        const float *x = B + (size_t)col * ldb;
        int i = 0;
        for (; i + 4 <= n_in; i += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(x + i);
            const float xv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int r = 0; r < RM; ++r) acc[r] = fmaf(sWt[(i + u) * RM + r], xv[u], acc[r]);
        }
        for (; i < n_in; ++i)
#pragma unroll
            for (int r = 0; r < RM; ++r) acc[r] = fmaf(sWt[i * RM + r], x[i], acc[r]);
#pragma unroll
        for (int r = 0; r < RM; ++r)
            if (r < R) D[(size_t)col * ldd + r] = acc[r];
    }
}

// The bounded wait of the tensor-core kernels on a barrier whose phase nothing
// completes: it must give up after `limit` polls and report kStatusTimeout.
__global__ void wait_selfcheck_kernel(unsigned int *status, int limit) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(smem_u32(&bar), 0u, limit)) atomicOr(status, kStatusTimeout);
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------
static int grid_for(int64_t items, int sms) {
    const int64_t g = (items + 255) / 256;
    const int64_t cap = (int64_t)sms * 16;
    return (int)(g < 1 ? 1 : (g < cap ? g : cap));
}

cudaError_t launch_wide_box(const BoxSource &src, int64_t base, int nb, int d, float *mh, float *ml, float *rr,
                            int64_t *bidx, int sms, cudaStream_t s) {
    wide_box_kernel<<<grid_for((int64_t)nb * d, sms), 256, 0, s>>>(src, base, nb, d, mh, ml, rr, bidx);
    return cudaGetLastError();
}

cudaError_t launch_wide_init(const NetParams<float> &net, const float *W0t, int nb, int NP, const float *mh,
                             const float *ml, const float *rr, float *C, float *Rr, float *Ch, float *Cl,
                             const float *alpha, int64_t alpha_ld, int64_t base, cudaStream_t s) {
    const dim3 grid((net.n[1] + kRowsX - 1) / kRowsX, nb), block(kRowsX, kSlicesY);
    wide_init_kernel<<<grid, block, 0, s>>>(net, W0t, NP, mh, ml, rr, C, Rr, Ch, Cl, alpha, alpha_ld, base);
    return cudaGetLastError();
}

cudaError_t launch_wide_const(const NetParams<float> &net, int k, int nb, int NP, const float *Ch, const float *Cl,
                              const float *Rr, float *Kh, float *Kl, float *Ke, int sms, cudaStream_t s) {
    wide_const_kernel<<<grid_for((int64_t)nb * net.n[k + 1], sms), 256, 0, s>>>(net, k, nb, NP, Ch, Cl, Rr, Kh, Kl,
                                                                                  Ke);
    return cudaGetLastError();
}

cudaError_t launch_wide_hidden(const NetParams<float> &net, int layer, int nb, int NP, float gcoef, float *C, float *Rr,
                               float *Ch, float *Cl, const float *Kh, const float *Kl, const float *Ke,
                               const float *alpha, int64_t alpha_ld, int64_t base, cudaStream_t s) {
    const dim3 grid((net.n[layer] + kH4Rows - 1) / kH4Rows, nb), block(kH4X, kH4Y);
    wide_hidden_kernel<<<grid, block, 0, s>>>(net, layer, NP, gcoef, C, Rr, Ch, Cl, Kh, Kl, Ke, alpha, alpha_ld, base);
    return cudaGetLastError();
}

cudaError_t launch_wide_final(const NetParams<float> &net, int nb, int NP, float gcoef, float *C, float *Rr, float *Ch,
                              float *Cl, const float *Kh, const float *Kl, const float *Ke, float *lo, float *hi,
                              float *err, cudaStream_t s) {
    const dim3 grid((net.R + kRowsX - 1) / kRowsX, nb), block(kRowsX, kSlicesY);
    wide_final_kernel<<<grid, block, 0, s>>>(net, NP, gcoef, C, Rr, Ch, Cl, Kh, Kl, Ke, lo, hi, err);
    return cudaGetLastError();
}

cudaError_t launch_wide_classify(const NetParams<float> &net, int nb, int64_t base, const float *lo, const float *hi,
                                 const float *err, const int64_t *bidx, const EvalOutputs &out, int sms,
                                 cudaStream_t s) {
    wide_classify_kernel<<<grid_for(nb, sms), 256, 0, s>>>(net, nb, base, lo, hi, err, bidx, out);
    return cudaGetLastError();
}

cudaError_t launch_wide_rows_product(const float *Wt, int n_in, int R, const float *B, int ldb, float *D, int ldd,
                                     int64_t ncols, bool abs_w, int sms, cudaStream_t s) {
    const int grid = grid_for(ncols, sms);
    if (R <= 4) {
        wide_rows_product_kernel<4><<<grid, 256, (size_t)n_in * 4 * sizeof(float), s>>>(Wt, n_in, R, B, ldb, D, ldd,
                                                                                       ncols, abs_w ? 1 : 0);
    } else if (R <= 8) {
        wide_rows_product_kernel<8><<<grid, 256, (size_t)n_in * 8 * sizeof(float), s>>>(Wt, n_in, R, B, ldb, D, ldd,
                                                                                       ncols, abs_w ? 1 : 0);
    } else if (R <= 16) {
        wide_rows_product_kernel<16><<<grid, 256, (size_t)n_in * 16 * sizeof(float), s>>>(Wt, n_in, R, B, ldb, D,
                                                                                         ldd, ncols, abs_w ? 1 : 0);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_wait_selfcheck(unsigned int *status, int limit, cudaStream_t s) {
    wait_selfcheck_kernel<<<1, 32, 0, s>>>(status, limit);
    return cudaGetLastError();
}

cudaError_t launch_wide_gemm(const WideGemmArgs &args, int nprob, cudaStream_t s) {
    int gx = 1, gy = 1;
    for (int i = 0; i < nprob; ++i) {
        gx = std::max(gx, (args.g[i].ncols + kWN - 1) / kWN);
        gy = std::max(gy, (args.g[i].M + kWM - 1) / kWM);
    }
    const size_t smem = wide_gemm_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(wide_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    wide_gemm_kernel<<<dim3(gx * gy, 1, nprob), kWThreads, smem, s>>>(args, gy);
    return cudaGetLastError();
}

}  // namespace slr
