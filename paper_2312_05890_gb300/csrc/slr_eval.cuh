// Fused SLR evaluation of a tile of boxes held in shared memory.
//
// One CTA takes a tile of T boxes and carries their symbolic state through all
// layers without leaving the SM:
//   decode     path code -> box centre m (float-float) and radius r, outward
//   layer 1    C = [W_1 diag(r) | W_1 m + b_1], R = 0, error E of the rounding
//   per hidden layer k:
//     finish   constant and error of the contraction that produced the layer
//     bounds   concrete bounds of both equations over the box (Sec. 2.2):
//              max/min of (C +- R) = const +- sum_j |coeff_j|, outward
//     relax    ReLU relaxation, Eq. 1 (per-equation or one-pair reading)
//     offsets  (float) the constant of every box as box 0's plus an offset
//     contract C' = W C + b, R' = |W| R (the per-layer symbolic matrix product)
//   last layer the property rows are folded into W_K; row bounds lo_r, hi_r
//   classify  Sec. 3 containment check: UNSAFE / SAFE / UNDECIDED, and flag
//              undecided boxes whose margins lie within the rounding budget.
//
// State layout in shared memory: element (row p, column c, box b) at
// S[p * NS + c * T + b], NS = state_stride(T, d) >= T (2d + 5).  Columns:
// C coefficients (0..d-1), C constant (high part, d), R coefficients
// (d+1..2d), R constant (2d+1), N = magnitude of the row's product columns
// (2d+2), E = error bound (2d+3), C constant low part (2d+4).  Boxes are the
// fastest index so that a warp reads one column of 32 boxes; NS is T modulo
// 32, so a warp's items of consecutive rows fall in distinct banks.
#pragma once

#include "slr_device.cuh"

namespace slr {

// ---- thread-block cluster (PTX): rank, barrier, stores to a peer's shared memory ----
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_index_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// Every thread of every CTA of the cluster arrives (its earlier shared-memory
// writes released) and waits for all (acquiring theirs).
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_map(const void *p, uint32_t rank) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void st_cluster4(uint32_t addr, const double (&v)[4]) {
    asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(addr), "d"(v[0]), "d"(v[1]) : "memory");
    asm volatile("st.shared::cluster.v2.f64 [%0+16], {%1, %2};" ::"r"(addr), "d"(v[2]), "d"(v[3]) : "memory");
}

// Four consecutive values from shared memory at a 32-bit shared address.
// volatile: the asm names no memory operand, so without it the compiler could
// move these loads across the block barriers and cp.async waits that order
// them after the stores they read.
template <typename Real> __device__ __forceinline__ void lds4(uint32_t addr, Real (&v)[4]);
template <> __device__ __forceinline__ void lds4<float>(uint32_t addr, float (&v)[4]) {
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "r"(addr));
}
template <> __device__ __forceinline__ void lds4<double>(uint32_t addr, double (&v)[4]) {
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "r"(addr));
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2+16];" : "=d"(v[2]), "=d"(v[3]) : "r"(addr));
}

template <typename Real> struct V4;
template <> struct V4<float> {
    static __device__ __forceinline__ void ld(const float *p, float (&v)[4]) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    static __device__ __forceinline__ void st(float *p, const float (&v)[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct V4<double> {
    static __device__ __forceinline__ void ld(const double *p, double (&v)[4]) {
        const double2 a = *reinterpret_cast<const double2 *>(p);
        const double2 b = *reinterpret_cast<const double2 *>(p + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    static __device__ __forceinline__ void st(double *p, const double (&v)[4]) {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
    }
};

__device__ __forceinline__ unsigned long long pext64(unsigned long long x, unsigned long long mask) {
    unsigned long long res = 0;
    int pos = 0;
    while (mask) {
        const unsigned long long low = mask & (~mask + 1ull);
        if (x & low) res |= 1ull << pos;
        ++pos;
        mask &= mask - 1ull;
    }
    return res;
}

// Half index k and split count c of input dimension i in the depth-t box with
// path code `code` (Sec. 2.2 bisection): dimension i spans
// [a_i + w_i k 2^-c, a_i + w_i (k + 1) 2^-c].  Widest-side schedule: the splits
// on i are the code bits dim_mask[i].  Per-box split dimensions: split j took
// the upper half when bit t-1-j is set and dimension split_set[nibble j].
__device__ __forceinline__ void code_dim(const BoxSource &src, unsigned long long code, int i,
                                         unsigned long long &k, int &c) {
    if (src.split_of == nullptr) {
        const unsigned long long mask = src.dim_mask[i] >> (src.D - src.t);
        k = pext64(code, mask);
        c = __popcll(mask);
        return;
    }
    k = 0ull;
    c = 0;
    const int s = src.split_of[i];
    if (s < 0) return;
    for (int j = 0; j < src.t; ++j) {
        if ((int)((code >> (kSplitPathBits + 4 * j)) & 15ull) == s) {
            k = 2ull * k + ((code >> (src.t - 1 - j)) & 1ull);
            ++c;
        }
    }
}

// Centre m64 as a pair hi + lo in Real and radius r rounded up so that
// [hi + lo - r, hi + lo + r] covers [m64 - r64, m64 + r64] plus `pad` (the
// float64 error of computing m64 and r64).
template <typename Real>
__device__ __forceinline__ void split_centre(double m64, double r64, double pad, Real &mh, Real &ml, Real &r);
template <>
__device__ __forceinline__ void split_centre<float>(double m64, double r64, double pad, float &mh, float &ml, float &r) {
    mh = (float)m64;
    const double rem = m64 - (double)mh;
    ml = (float)rem;
    const double off = fabs(rem - (double)ml);
    r = __double2float_ru(__dadd_ru(__dadd_ru(r64, off), pad));
}
template <>
__device__ __forceinline__ void split_centre<double>(double m64, double r64, double pad, double &mh, double &ml,
                                                     double &r) {
    mh = m64;
    ml = 0.0;
    r = __dadd_ru(r64, pad);
}

template <typename Real> __device__ __forceinline__ float to_lo(Real v);
template <typename Real> __device__ __forceinline__ float to_hi(Real v);
template <> __device__ __forceinline__ float to_lo<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_hi<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_lo<double>(double v) { return __double2float_rd(v); }
template <> __device__ __forceinline__ float to_hi<double>(double v) { return __double2float_ru(v); }

// Error-free transformations (Knuth's TwoSum, FMA-based TwoProduct) used to
// carry the constant of C as an unevaluated pair hi + lo.
template <typename Real>
__device__ __forceinline__ void two_sum(Real a, Real b, Real &s, Real &e);
template <>
__device__ __forceinline__ void two_sum<float>(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
template <>
__device__ __forceinline__ void two_sum<double>(double a, double b, double &s, double &e) {
    s = __dadd_rn(a, b);
    const double z = __dsub_rn(s, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, z)), __dsub_rn(b, z));
}
template <typename Real>
__device__ __forceinline__ void two_prod(Real a, Real b, Real &p, Real &e) {
    p = Arith<Real>::mul_rn(a, b);
    e = Arith<Real>::fma_rn(a, b, -p);
}

// gamma_n-style constant (n + 2) u, u the unit roundoff; (n+2)u >= n u / (1 - n u) for n <= 1024.
template <typename Real>
__device__ __forceinline__ Real gam(int n) {
    return (Real)(n + 2) * ((Real)0.5 * Arith<Real>::ulp2);
}

// Rigorous bound u |x| (1 + tiny) of one round-to-nearest of a value of magnitude x.
template <typename Real>
__device__ __forceinline__ Real uerr(Real x) {
    return Arith<Real>::mul_up(x, (Real)0.50001 * Arith<Real>::ulp2);
}

// Relative rounding bound of an n-term float-float dot product sum_i w_i x_i
// (w_i float, x_i float64 split into float hi + lo, products exact by
// TwoProduct, hi parts added by TwoSum, the error terms and w_i lo_i summed
// in float; Ogita, Rump and Oishi, "Accurate sum and dot product", 2005:
// gamma_n^2 sum |w_i x_i|, taken here with a factor 4 and n + 2 terms for the
// lo products and the combination of partial sums), plus the split of the
// inputs (2^-48 relative) and the rounding of hi + lo to float64 (2^-53),
// rounded upward.  The underflow of these float operations is bounded apart
// (ff_abs).
__device__ __forceinline__ double gam_ff(int n) {
    const double g = (double)(n + 4) * 0x1p-24;     // >= gamma_{n+2} in float
    const double gn = (double)(n + 2) * 0x1p-24;    // >= gamma_n
    return __dadd_ru(__dmul_ru(__dmul_ru(4.0 * g, g), 1.0 + gn), 0x1p-47);
}

// Absolute bound of what the float-float products lose to underflow in one
// bound of a row: every split input and float operation loses at most 2^-150,
// times the row's weight magnitude (wabs >= sum_i |w_i|) or once per term,
// over the 2d + 3 product columns a bound reads (taken as 2d + 8, doubled).
__device__ __forceinline__ double ff_abs(double wabs, int n, int d) {
    return __dmul_ru((double)(2 * d + 8) * 0x1p-149, __dadd_ru(wabs, (double)(2 * n + 8)));
}

// Multiply-add of a float weight and a float-float input into a float-float
// accumulator (s, e): the product exactly as p + pe, p added to s by TwoSum,
// the error terms and w lo added to e in float.
__device__ __forceinline__ void ff_mac(float w, float h, float l, float &s, float &e) {
    float p, pe, t, se;
    two_prod<float>(w, h, p, pe);
    two_sum<float>(s, p, t, se);
    s = t;
    e = __fmaf_rn(w, l, __fadd_rn(e, __fadd_rn(pe, se)));
}

// Row accessors.  A row view R maps a column of one row (SIMT numbering: C
// coefficients 0..d-1, C constant hi d, R coefficients d+1..2d, R constant
// 2d+1, N 2d+2, E 2d+3, C constant lo 2d+4) to a Real& in shared memory.
template <typename Real, int T>
struct SimtLayout {
    Real *S;
    int NS;
    struct Row {
        Real *p;
        __device__ __forceinline__ Real &operator()(int c) const { return p[c * T]; }
    };
    __device__ __forceinline__ Row row(int p, int b) const { return Row{S + p * NS + b}; }
    // upper bound of |value| of a column (exact here)
    __device__ __forceinline__ Real mag(int p, int b, int c) const { return Arith<Real>::abs(S[p * NS + c * T + b]); }
    __device__ __forceinline__ void finish_row(int, int) const {}
};

// Concrete bounds of the raw equations U = C + R, L = C - R of one row over
// the box (Sec. 2.2: const +- sum_j |coeff_j| in the normalised input), with
// outward rounding so that they bound the stored equations exactly; the same
// sums in round-to-nearest give `delta`, how far the outward bounds lie from
// the nearest-rounded ones (reported with the property rows' error, so that
// bound -+ error is the plain FP32 SLR bound).
template <typename Real>
struct RowBounds {
    Real uu, lu, ul, ll;   // max U, min U, max L, min L (outward)
    Real NC, NR;           // sum |C_j| over coefficients, sum |R_j| incl. its constant
    Real delta;            // outward minus nearest-rounded, for max U and min L
    Real SU, SL;           // sum |C_j + R_j|, sum |C_j - R_j| (upward)
    Real SUn, SLn;         // the same sums rounded to nearest
    __device__ __forceinline__ void reset() {
        SU = SL = SUn = SLn = NC = NR = 0;
    }
    __device__ __forceinline__ void add(Real c, Real r) {
        using A = Arith<Real>;
        const Real u = A::abs(c + r), l = A::abs(c - r);
        SU = A::add_up(SU, u);
        SL = A::add_up(SL, l);
        SUn = SUn + u;
        SLn = SLn + l;
        NC = A::add_up(NC, A::abs(c));
        NR = A::add_up(NR, A::abs(r));
    }
    // partial sums over disjoint coefficient sets
    __device__ __forceinline__ void merge(const RowBounds &o) {
        using A = Arith<Real>;
        SU = A::add_up(SU, o.SU);
        SL = A::add_up(SL, o.SL);
        SUn = SUn + o.SUn;
        SLn = SLn + o.SLn;
        NC = A::add_up(NC, o.NC);
        NR = A::add_up(NR, o.NR);
    }
    __device__ __forceinline__ void finish(Real chi, Real clo, Real rd) {
        using A = Arith<Real>;
        NR = A::add_up(NR, A::abs(rd));
        // |c +- r| <= |fl(c +- r)| (1 + u): cover the round-to-nearest of each term
        const Real su = A::mul_up(SU, (Real)1 + A::ulp2);
        const Real sl = A::mul_up(SL, (Real)1 + A::ulp2);
        uu = A::add_up(A::add_up(A::add_up(chi, rd), clo), su);
        lu = A::add_dn(A::add_dn(A::add_dn(chi, rd), clo), -su);
        ul = A::add_up(A::add_up(A::add_up(chi, -rd), clo), sl);
        ll = A::add_dn(A::add_dn(A::add_dn(chi, -rd), clo), -sl);
        const Real uun = ((chi + rd) + clo) + SUn;
        const Real lln = ((chi - rd) + clo) - SLn;
        const Real du = A::add_up(uu, -uun), dl = A::add_up(lln, -ll);
        delta = du > dl ? du : dl;
        delta = delta > (Real)0 ? delta : (Real)0;
    }
    template <class Row>
    __device__ __forceinline__ void compute(const Row &R, int d, Real chi, Real clo) {
        reset();
        for (int j = 0; j < d; ++j) add(R(j), R(d + 1 + j));
        finish(chi, clo, R(2 * d + 1));
    }
};

// What the ReLU relaxation (Eq. 1) does to one row: keep it (active), zero it
// (inactive) or map every coefficient pair (c, r) to (pp c + qq r, qq c + pp r)
// (unstable), and the row's new constant, radius constant, N and E.
template <typename Real>
struct RelaxPlan {
    int kind;              // 0 active, 1 inactive, 2 unstable
    Real pp, qq;
    Real nh, nl, rd, E, N;
};

// S-shaped activations (tanh, logistic sigmoid): the value and derivative at
// z with bounds of their errors.  CUDA documents tanhf and expf as accurate
// to 2 ulp and tanh and exp to 1 ulp; with the roundings added here the
// value's error stays below 16 units of 2^-24 (float) or 2^-53 (double)
// relative, and the derivative's (1 - t^2, s (1 - s), both in [0, 1]) below
// 16 such units absolutely: those are the margins returned.
template <typename Real> __device__ __forceinline__ Real act_tanh(Real z);
template <> __device__ __forceinline__ float act_tanh<float>(float z) { return tanhf(z); }
template <> __device__ __forceinline__ double act_tanh<double>(double z) { return tanh(z); }
template <typename Real> __device__ __forceinline__ Real act_exp(Real z);
template <> __device__ __forceinline__ float act_exp<float>(float z) { return expf(z); }
template <> __device__ __forceinline__ double act_exp<double>(double z) { return exp(z); }

template <typename Real>
__device__ __forceinline__ void act_eval(int act, Real z, Real &v, Real &ev, Real &dv, Real &ed) {
    using A = Arith<Real>;
    if (act == kActTanh) {
        v = act_tanh<Real>(z);
        dv = A::fma_rn(-v, v, (Real)1);
    } else {
        const Real e = act_exp<Real>(-z);
        v = A::div_rn((Real)1, (Real)1 + e);
        dv = A::mul_rn(v, (Real)1 - v);
    }
    dv = dv > (Real)0 ? dv : (Real)0;
    ev = A::add_up(A::mul_up(A::abs(v), (Real)8 * A::ulp2), A::tiny);
    ed = (Real)8 * A::ulp2;
}

// DC > 0: the network has DC inputs, known at compile time (loops over the
// input coefficients unrolled, column offsets constant); DC = 0: read from net.d.
template <typename Real, int T, int NT, int KI = 2, int DC = 0>
struct EvalTile {
    using A = Arith<Real>;
    static __device__ __forceinline__ int dim_of(const NetParams<Real> &net) { return DC > 0 ? DC : net.d; }
    // FP32 carries the constants as compensated pairs; FP64 is precise enough
    // with a plain FMA chain (its gamma_n error bound is ~1e-14 relative).
    static constexpr bool kCompensated = sizeof(Real) == 4;

    // Column offsets of one row (times T in memory): C coefficients [0, d),
    // C constant hi (d), R coefficients [d+1, 2d+1), R constant (2d+1),
    // N (2d+2), E (2d+3), C constant lo (2d+4).
    static __device__ __forceinline__ int cCh(int d) { return d; }
    static __device__ __forceinline__ int cR(int d) { return d + 1; }
    static __device__ __forceinline__ int cRd(int d) { return 2 * d + 1; }
    static __device__ __forceinline__ int cN(int d) { return 2 * d + 2; }
    static __device__ __forceinline__ int cE(int d) { return 2 * d + 3; }
    static __device__ __forceinline__ int cCl(int d) { return 2 * d + 4; }

    // ---- layer 1: C = [W_1 diag(r) | W_1 m + b_1], R = 0 ------------------------
    template <class L>
    static __device__ void init_layer(const L &lay, const NetParams<Real> &net, const Real *sMh, const Real *sMl,
                                      const Real *sR) {
        const int d = dim_of(net);
        const int n1 = net.n[1];
        for (int item = threadIdx.x; item < n1 * T; item += NT) {
            const int p = item / T;
            const int b = item - p * T;
            const auto R = lay.row(p, b);
            const Real *w = net.W0 + (size_t)p * d;
            const Real bp = net.b[0][p];
            Real S1 = 0, s = bp, e = 0, sabs = A::abs(bp);
            for (int j = 0; j < d; ++j) {
                const Real wj = w[j];
                const Real c = A::mul_rn(wj, sR[b * d + j]);
                R(j) = c;
                S1 = A::add_up(S1, A::abs(c));
                Real p1, pe, t, se;
                two_prod<Real>(wj, sMh[b * d + j], p1, pe);
                two_sum<Real>(s, p1, t, se);
                s = t;
                e = A::fma_rn(wj, sMl[b * d + j], e + (pe + se));
                sabs = sabs + A::abs(p1);
            }
            Real chi, clo;
            two_sum<Real>(s, e, chi, clo);
            R(cCh(d)) = chi;
            R(cCl(d)) = clo;
            const Real g = gam<Real>(d + 2);
            Real E = A::add_up(uerr<Real>(S1),
                               A::mul_up(A::mul_up((Real)2 * g, g), A::mul_up(sabs, (Real)1 + gam<Real>(d))));
            E = A::add_up(E, (Real)(d + 4) * A::tiny);
            if (net.K == 1) {
                // folded property layer applied to x itself: |x_j| <= |m_j| + r_j
                Real fe = net.fold_berr[p];
                for (int j = 0; j < d; ++j) {
                    const Real xm = A::add_up(A::add_up(A::abs(sMh[b * d + j]), A::abs(sMl[b * d + j])), sR[b * d + j]);
                    fe = A::add_up(fe, A::mul_up(net.fold_err[p * d + j], xm));
                }
                E = A::add_up(E, fe);
            }
            for (int j = 0; j <= d; ++j) R(cR(d) + j) = 0;
            R(cN(d)) = S1;
            R(cE(d)) = E;
        }
    }

    // ---- constants of the next layer, before the contraction overwrites the state --
    // For output rows p0 = 2q and p0 + 1 and box b: the error-free constant dot
    // product over the input rows, its error bound, and (last layer only) the
    // rounding of the folded property weights, sum_i delta_pi |z_i| with
    // |z_i| <= N_i + |C_i const| + E_i.  Written to sConst = [hi | lo | err].
    // sW holds the layer's float weights transposed (row i, column p, stride Mpad).
    template <class L>
    static __device__ void const_phase(const L &lay, Real *sConst, const Real *sW, int Mpad,
                                       const NetParams<Real> &net, int layer) {
        const int pairs = (net.n[layer + 1] + 1) / 2;
        for (int item = threadIdx.x; item < pairs * T; item += NT) const_item(lay, sConst, sW, Mpad, net, layer, item);
    }

    // kList: sum only over the input rows ridx[0 .. n_rows) (the others are
    // zero in every box of the tile); else over all n_in rows.  WT: the type
    // of the staged weights (float for the float64 tile's float-float
    // products; exact either way).
    template <bool kList = false, class L, class WT>
    static __device__ __forceinline__ void const_item(const L &lay, Real *sConst, const WT *sW, int Mpad,
                                                      const NetParams<Real> &net, int layer, int item,
                                                      const int *ridx = nullptr, int n_rows = 0) {
        const int d = dim_of(net);
        const int n_in = net.n[layer];
        const int n_out = net.n[layer + 1];
        const bool last = layer + 1 == net.K;
        const Real *bias = net.b[layer];
        const int nmp = net.n_max_pad;
        {
            const int q = item / T;
            const int b = item - q * T;
            const int p0 = 2 * q;
            const bool two = p0 + 1 < n_out;
            Real s0 = bias[p0], e0 = 0, a0 = A::abs(s0);
            Real s1 = two ? bias[p0 + 1] : (Real)0, e1 = 0, a1 = A::abs(s1);
            Real f0 = 0, f1 = 0;
            const int nr = kList ? n_rows : n_in;
            for (int ii = 0; ii < nr; ++ii) {
                const int i = kList ? ridx[ii] : ii;
                const auto Ri = lay.row(i, b);
                const Real h = Ri(cCh(d));
                const Real l = Ri(cCl(d));
                const Real w0 = (Real)sW[i * Mpad + p0];
                const Real w1 = (Real)sW[i * Mpad + p0 + 1];
                if (kCompensated) {
                    Real p1, pe, t, se;
                    two_prod<Real>(w0, h, p1, pe);
                    two_sum<Real>(s0, p1, t, se);
                    s0 = t;
                    e0 = A::fma_rn(w0, l, e0 + (pe + se));
                    a0 = a0 + A::abs(p1);
                    two_prod<Real>(w1, h, p1, pe);
                    two_sum<Real>(s1, p1, t, se);
                    s1 = t;
                    e1 = A::fma_rn(w1, l, e1 + (pe + se));
                    a1 = a1 + A::abs(p1);
                } else {
                    // float64: a plain FMA chain, |error| <= gamma_2n sum |w| (|h| + |l|)
                    s0 = A::fma_rn(w0, h, A::fma_rn(w0, l, s0));
                    s1 = A::fma_rn(w1, h, A::fma_rn(w1, l, s1));
                    a0 = A::fma_rn(A::abs(w0), A::abs(h) + A::abs(l), a0);
                    a1 = A::fma_rn(A::abs(w1), A::abs(h) + A::abs(l), a1);
                }
                if (last) {
                    const Real z = A::add_up(A::add_up(lay.mag(i, b, cN(d)), A::abs(h)),
                                             A::add_up(A::abs(l), lay.mag(i, b, cE(d))));
                    f0 = A::add_up(f0, A::mul_up(net.fold_err[p0 * n_in + i], z));
                    if (two) f1 = A::add_up(f1, A::mul_up(net.fold_err[(p0 + 1) * n_in + i], z));
                }
            }
            const Real g = gam<Real>(kCompensated ? n_in + 2 : 2 * n_in + 2);
            const Real g2 = kCompensated ? A::mul_up((Real)2 * g, g) : (Real)2 * g;
            const Real ga = (Real)1 + gam<Real>(n_in);
            Real hi, lo;
            two_sum<Real>(s0, e0, hi, lo);
            sConst[p0 * T + b] = hi;
            sConst[(nmp + p0) * T + b] = lo;
            Real err = A::mul_up(g2, A::mul_up(a0, ga));
            if (last) err = A::add_up(err, A::add_up(f0, net.fold_berr[p0]));
            sConst[(2 * nmp + p0) * T + b] = err;
            if (two) {
                two_sum<Real>(s1, e1, hi, lo);
                sConst[(p0 + 1) * T + b] = hi;
                sConst[(nmp + p0 + 1) * T + b] = lo;
                err = A::mul_up(g2, A::mul_up(a1, ga));
                if (last) err = A::add_up(err, A::add_up(f1, net.fold_berr[p0 + 1]));
                sConst[(2 * nmp + p0 + 1) * T + b] = err;
            }
        }
    }

    // ---- add the contraction's constant and error; returns (chi, clo, E) -------
    // gcoef bounds the relative rounding of the contraction's coefficient
    // columns (gamma_n * sum_i |W_pi| N_i, from the |W| N column).
    // With `delta`, the constant is the reference box's (slot b = 0 of sConst)
    // plus the product W delta the contraction left in the constant column.
    // gabs: an absolute bound the products lose beyond gcoef (float-float
    // products: underflow, ff_abs), else 0.
    template <class Row>
    static __device__ __forceinline__ void finish_contraction(const Row &R, const Real *sConst, int nmp, int p, int b,
                                                              int d, int n_in, Real gcoef, Real &chi, Real &clo,
                                                              Real &E, bool delta = false, Real gabs = 0) {
        Real cerr;
        if (delta) {
            const Real ch = sConst[p * T], cl = sConst[(nmp + p) * T];
            cerr = sConst[(2 * nmp + p) * T];
            if (b == 0) {
                chi = ch;
                clo = cl;
            } else {
                Real e;
                two_sum<Real>(ch, R(cCh(d)), chi, e);
                clo = e + cl;
                cerr = A::add_up(cerr, uerr<Real>(A::abs(clo)));
            }
        } else {
            chi = sConst[p * T + b];
            clo = sConst[(nmp + p) * T + b];
            cerr = sConst[(2 * nmp + p) * T + b];
        }
        const Real wN = R(cN(d));
        Real eps = A::mul_up(gcoef, A::mul_up(wN, (Real)1 + gcoef));
        eps = A::add_up(A::add_up(eps, cerr), A::add_up((Real)(n_in + 4) * A::tiny, gabs));
        // |W| E was summed from non-negative terms with the same relative rounding
        E = A::add_up(A::mul_up(R(cE(d)), (Real)1 + (Real)2 * gcoef), eps);
    }

    // ---- ReLU relaxation (Eq. 1) of one hidden row from its concrete bounds ---------
    // chi, clo: the row's constant (float-float); rd: its radius constant; E: its
    // error bound.  a_ptr: the supplied lower slope of the
    // row, or null for u_l / (u_l - l_l).
    // ---- relaxation of an S-shaped activation (tanh, sigmoid) of one hidden row ----
    // Lines a z + b bounding s on [zl, zu] = [ll, uu], the concrete bounds of
    // the stored equations (a >= 0): on the concave side (zl >= 0) the tangent
    // at the midpoint above and the chord below, on the convex side (zu <= 0)
    // the other way round, and across 0 the slope lam = min(s'(zl), s'(zu))
    // through (zu, s(zu)) above and (zl, s(zl)) below (s' is largest at 0, so
    // s' >= lam on [zl, zu]).  The stored equations take the nominal lines (the
    // intercepts rounded to nearest, as plain SLR computes them); the same
    // slopes with intercepts rounded outward by the margins of act_eval are
    // sound (a chord kept on the right side of both end values suffices for a
    // convex or concave s; a tangent loses at most ed |z - m| to its inexact
    // slope), and the gap between the two intercepts, mu, joins E.  The true
    // pre-activation z lies in [L - E, U + E] and may leave [zl, zu] by E; there
    // s moves by at most its Lipschitz constant q (1 for tanh, 1/4 for the
    // sigmoid) times E, so U' = a_u U + b_u and L' = a_l L + b_l bound s(z) up
    // to max(q, a) E + mu (plus the rounding of the new row).
    static __device__ __forceinline__ RelaxPlan<Real> plan_sshape(const RowBounds<Real> &bd, int d, int act,
                                                                  int relax_mode, Real chi, Real clo, Real rd,
                                                                  Real E) {
        RelaxPlan<Real> pl;
        const Real lip = act == kActTanh ? (Real)1 : (Real)0.25;
        const Real zl = bd.ll, zu = bd.uu;
        Real vl, evl, dl, edl, vu, evu, du, edu;
        act_eval<Real>(act, zl, vl, evl, dl, edl);
        act_eval<Real>(act, zu, vu, evu, du, edu);
        if (relax_mode == kRelaxInterval || !(zu > zl)) {
            // the constant interval [s(zl), s(zu)] (s is increasing)
            const Real a = vl < vu ? vl : vu, b = vl < vu ? vu : vl;
            pl.kind = 1;
            pl.pp = 0;
            pl.qq = 0;
            two_sum<Real>(a, b, pl.nh, pl.nl);
            pl.nh *= (Real)0.5;
            pl.nl *= (Real)0.5;
            pl.rd = A::mul_up(A::add_up(b, -a), (Real)0.5);
            pl.N = pl.rd;
            const Real ev = evl > evu ? evl : evu;
            pl.E = A::add_up(A::add_up(A::mul_up(lip, E), ev), (Real)4 * A::tiny);
            return pl;
        }
        const Real width = A::add_up(zu, -zl);
        Real a_u, b_u, a_l, b_l, bu_out, bl_out;
        if (zl >= (Real)0 || zu <= (Real)0) {
            Real sc = A::div_rn(vu - vl, zu - zl);
            sc = sc < (Real)0 ? (Real)0 : (sc > lip ? lip : sc);
            const Real m = (zl + zu) * (Real)0.5;
            Real vm, evm, dm, edm;
            act_eval<Real>(act, m, vm, evm, dm, edm);
            const Real slack = A::mul_up(edm, width);   // |z - m| <= width
            const Real b_tan = A::fma_rn(-dm, m, vm);
            const Real b_chord = A::fma_rn(-sc, zl, vl);
            if (zl >= (Real)0) {
                // concave: tangent above, chord below
                a_u = dm;
                b_u = b_tan;
                bu_out = A::add_up(A::add_up(A::add_up(vm, evm), -A::mul_dn(dm, m)), slack);
                a_l = sc;
                b_l = b_chord;
                const Real b1 = A::add_dn(A::add_dn(vl, -evl), -A::mul_up(sc, zl));
                const Real b2 = A::add_dn(A::add_dn(vu, -evu), -A::mul_up(sc, zu));
                bl_out = b1 < b2 ? b1 : b2;
            } else {
                // convex: chord above, tangent below
                a_u = sc;
                b_u = b_chord;
                const Real b1 = A::add_up(A::add_up(vl, evl), -A::mul_dn(sc, zl));
                const Real b2 = A::add_up(A::add_up(vu, evu), -A::mul_dn(sc, zu));
                bu_out = b1 > b2 ? b1 : b2;
                a_l = dm;
                b_l = b_tan;
                bl_out = A::add_dn(A::add_dn(A::add_dn(vm, -evm), -A::mul_up(dm, m)), -slack);
            }
        } else {
            // nominal slope min(s'(zl), s'(zu)); a slope lam_r below the true
            // minimum of s' gives the sound lines through (zu, s(zu) + ev) and
            // (zl, s(zl) - ev), which lie within (lam - lam_r) width + ev of the
            // nominal ones on [zl, zu]
            Real lam = dl < du ? dl : du;
            lam = lam > (Real)0 ? lam : (Real)0;
            const Real m1 = A::add_dn(dl, -edl), m2 = A::add_dn(du, -edu);
            Real lam_r = m1 < m2 ? m1 : m2;
            lam_r = lam_r > (Real)0 ? lam_r : (Real)0;
            a_u = lam;
            a_l = lam;
            b_u = A::fma_rn(-lam, zu, vu);
            b_l = A::fma_rn(-lam, zl, vl);
            const Real tilt = A::mul_up(A::add_up(lam, -lam_r), width);
            const Real ru = uerr<Real>(A::add_up(A::abs(vu), A::mul_up(lam, A::abs(zu))));
            const Real rl = uerr<Real>(A::add_up(A::abs(vl), A::mul_up(lam, A::abs(zl))));
            bu_out = A::add_up(b_u, A::add_up(A::add_up(tilt, evu), ru));
            bl_out = A::add_dn(b_l, -A::add_up(A::add_up(tilt, evl), rl));
        }
        Real mu = A::add_up(bu_out, -b_u);
        const Real mu_l = A::add_up(b_l, -bl_out);
        mu = mu > mu_l ? mu : mu_l;
        mu = mu > (Real)0 ? mu : (Real)0;
        // E also bounds how far the nominal lines lie from the exact ones: a
        // chord built from inexact end values moves by up to both margins
        if (zl >= (Real)0 || zu <= (Real)0) {
            const Real chord_dev = A::add_up(A::add_up(evl, evu), uerr<Real>(A::add_up(A::abs(vl), A::abs(vu))));
            mu = mu > chord_dev ? mu : chord_dev;
        }
        // (C, R) <- ((U' + L') / 2, (U' - L') / 2)
        pl.kind = 2;
        pl.pp = (a_u + a_l) * (Real)0.5;
        pl.qq = (a_u - a_l) * (Real)0.5;
        const Real hc = (b_u + b_l) * (Real)0.5, hr = (b_u - b_l) * (Real)0.5;
        Real ph, pe;
        two_prod<Real>(pl.pp, chi, ph, pe);
        const Real rest = pe + A::fma_rn(pl.pp, clo, A::fma_rn(pl.qq, rd, hc));
        two_sum<Real>(ph, rest, pl.nh, pl.nl);
        pl.rd = A::fma_rn(pl.qq, chi, A::fma_rn(pl.qq, clo, A::fma_rn(pl.pp, rd, hr)));
        const Real a_max = a_u > a_l ? a_u : a_l;
        const Real tot = A::add_up(A::add_up(bd.NC, bd.NR), A::add_up(A::abs(chi), A::abs(clo)));
        const Real mag = A::add_up(A::mul_up(a_max, tot), A::add_up(A::abs(b_u), A::abs(b_l)));
        const Real err = A::add_up(A::mul_up((Real)8 * A::ulp2, mag), (Real)(2 * d + 8) * A::tiny);
        pl.E = A::add_up(A::add_up(A::mul_up(a_max > lip ? a_max : lip, E), err), mu);
        pl.N = A::mul_up(A::add_up(mag, A::add_up(err, err)), (Real)1 + (Real)4 * A::ulp2);
        return pl;
    }

    static __device__ __forceinline__ RelaxPlan<Real> plan_row(const RowBounds<Real> &bd, int d, int relax_mode,
                                                               Real chi, Real clo, Real rd, Real E,
                                                               const float *a_ptr, int act = kActRelu) {
        RelaxPlan<Real> pl;
        if (act != kActRelu) return plan_sshape(bd, d, act, relax_mode, chi, clo, rd, E);
        if (relax_mode == kRelaxInterval) {
            // Moore intervals: relu is monotone and 1-Lipschitz, so the row becomes
            // the constant interval [relu(ll), relu(uu)] (centre exact as a
            // float-float pair, radius rounded up) and E carries over
            const Real a = bd.ll > (Real)0 ? bd.ll : (Real)0;
            const Real b = bd.uu > (Real)0 ? bd.uu : (Real)0;
            pl.kind = 1;
            pl.pp = 0;
            pl.qq = 0;
            two_sum<Real>(a, b, pl.nh, pl.nl);
            pl.nh *= (Real)0.5;
            pl.nl *= (Real)0.5;
            pl.rd = A::mul_up(A::add_up(b, -a), (Real)0.5);
            pl.N = pl.rd;
            pl.E = A::add_up(E, (Real)4 * A::tiny);
            return pl;
        }
        if (bd.ll >= (Real)0) {
            // stable active: relu is the identity on [L - E, U + E] up to
            // U + E >= lu + E >= 0, so the equations and E carry over
            pl.kind = 0;
            pl.pp = 1;
            pl.qq = 0;
            pl.nh = chi;
            pl.nl = clo;
            pl.rd = rd;
            pl.N = A::add_up(bd.NC, bd.NR);
            pl.E = E;
            return pl;
        }
        if (bd.uu <= (Real)0) {
            // stable inactive: relu(z) lies in [0, max(0, uu + E)]
            pl.kind = 1;
            pl.pp = 0;
            pl.qq = 0;
            pl.nh = 0;
            pl.nl = 0;
            pl.rd = 0;
            pl.N = 0;
            const Real top = A::add_up(bd.uu, E);
            pl.E = top > (Real)0 ? top : (Real)0;
            return pl;
        }
        // unstable: U' = sig_u (U - l) and L' = sig_l L (Eq. 1).  Applied to
        // U + E over [lu + E, uu + E] the chord misses relu by (1 - sig_u) E
        // and shifts by sig_u E, and sig_l (L - E) <= relu(L - E): E carries over.
        Real sig_u, sig_l, h;
        if (relax_mode == kRelaxPaperLiteral) {
            sig_u = A::div_up(bd.uu, A::add_dn(bd.uu, -bd.ll));
            sig_u = sig_u < (Real)1 ? sig_u : (Real)1;
            h = A::mul_rn(sig_u, -bd.ll);
            sig_l = A::div_rn(bd.uu, bd.uu - bd.ll);
        } else {
            if (bd.lu >= (Real)0) {
                sig_u = 1;
                h = 0;
            } else {
                sig_u = A::div_up(bd.uu, A::add_dn(bd.uu, -bd.lu));
                sig_u = sig_u < (Real)1 ? sig_u : (Real)1;
                h = A::mul_rn(sig_u, -bd.lu);
            }
            if (bd.ul <= (Real)0) {
                sig_l = 0;
            } else if (a_ptr != nullptr) {
                // a supplied slope, clamped to [0, 1] (NaN -> 0)
                sig_l = (Real)fminf(fmaxf(*a_ptr, 0.f), 1.f);
            } else {
                sig_l = A::div_rn(bd.ul, bd.ul - bd.ll);
            }
        }
        sig_l = sig_l < (Real)0 ? (Real)0 : (sig_l > (Real)1 ? (Real)1 : sig_l);
        // (C, R) <- ((U' + L') / 2, (U' - L') / 2)
        pl.kind = 2;
        pl.pp = (sig_u + sig_l) * (Real)0.5;
        pl.qq = (sig_u - sig_l) * (Real)0.5;
        const Real hh = h * (Real)0.5;
        Real ph, pe;
        two_prod<Real>(pl.pp, chi, ph, pe);
        const Real rest = pe + A::fma_rn(pl.pp, clo, A::fma_rn(pl.qq, rd, hh));
        two_sum<Real>(ph, rest, pl.nh, pl.nl);
        pl.rd = A::fma_rn(pl.qq, chi, A::fma_rn(pl.qq, clo, A::fma_rn(pl.pp, rd, hh)));
        const Real sig_max = sig_u > sig_l ? sig_u : sig_l;
        const Real tot = A::add_up(A::add_up(bd.NC, bd.NR), A::add_up(A::abs(chi), A::abs(clo)));
        const Real mag = A::add_up(A::mul_up(sig_max, tot), h);
        const Real err = A::add_up(A::mul_up((Real)8 * A::ulp2, mag), (Real)(2 * d + 8) * A::tiny);
        pl.E = A::add_up(E, err);
        pl.N = A::mul_up(A::add_up(mag, A::add_up(err, err)), (Real)1 + (Real)4 * A::ulp2);
        return pl;
    }

    // one coefficient pair of a row under the plan
    static __device__ __forceinline__ void apply_plan(const RelaxPlan<Real> &pl, Real &c, Real &r) {
        if (pl.kind == 1) {
            c = 0;
            r = 0;
        } else if (pl.kind == 2) {
            const Real c0 = c, r0 = r;
            c = A::fma_rn(pl.pp, c0, pl.qq * r0);
            r = A::fma_rn(pl.qq, c0, pl.pp * r0);
        }
    }

    // ---- bounds and ReLU relaxation of one hidden row, in place ----------------------
    // Returns true when the relaxed row is identically zero (a stable inactive
    // neuron whose error bound is 0): its columns add nothing to the next product.
    template <class Row>
    static __device__ __forceinline__ bool relax_row(const Row &R, int d, int relax_mode, Real chi, Real clo, Real E,
                                                     const float *a_ptr, int act = kActRelu) {
        const int cr = cR(d);
        RowBounds<Real> bd;
        bd.compute(R, d, chi, clo);
        const RelaxPlan<Real> pl = plan_row(bd, d, relax_mode, chi, clo, R(cr + d), E, a_ptr, act);
        if (pl.kind == 1) {
            // a constant row: the coefficients are zeros, nothing to read
            for (int j = 0; j < d; ++j) {
                R(j) = 0;
                R(cr + j) = 0;
            }
        } else if (pl.kind == 2) {
            for (int j = 0; j < d; ++j) {
                Real c = R(j), r = R(cr + j);
                apply_plan(pl, c, r);
                R(j) = c;
                R(cr + j) = r;
            }
        }
        R(cCh(d)) = pl.nh;
        R(cCl(d)) = pl.nl;
        R(cr + d) = pl.rd;
        R(cN(d)) = pl.N;
        R(cE(d)) = pl.E;
        return pl.kind == 1 && pl.nh == (Real)0 && pl.nl == (Real)0 && pl.rd == (Real)0 && pl.N == (Real)0 &&
               pl.E == (Real)0;
    }

    // ---- one hidden layer: constant, error, concrete bounds, ReLU relaxation ----
    // `live` (nullable): live[p] is set to 1 for every row p that is not
    // identically zero in some box of the tile (the flags start at 0).
    template <class L>
    static __device__ void hidden_epilogue(const L &lay, const Real *sConst, const NetParams<Real> &net, int layer,
                                           Real gcoef, const float *alpha = nullptr, int64_t alpha_ld = 0,
                                           int64_t base = 0, int64_t n = 0, int alpha_off = 0, bool delta = false,
                                           int *live = nullptr, Real gabs = 0) {
        const int d = dim_of(net);
        const int nrows = net.n[layer];
        const int n_in = net.n[layer - 1];
        for (int item = threadIdx.x; item < nrows * T; item += NT) {
            const int p = item / T;
            const int b = item - p * T;
            const auto R = lay.row(p, b);
            Real chi, clo, E;
            if (layer > 1) {
                finish_contraction(R, sConst, net.n_max_pad, p, b, d, n_in, gcoef, chi, clo, E, delta, gabs);
            } else {
                chi = R(cCh(d));
                clo = R(cCl(d));
                E = R(cE(d));
            }
            const float *a_ptr = nullptr;
            if (alpha != nullptr) {
                // padding slots of the last tile repeat the tile's first box
                const int64_t pos = base + b < n ? base + b : base;
                a_ptr = alpha + pos * alpha_ld + alpha_off + p;
            }
            const bool zero = relax_row(R, d, net.relax_mode, chi, clo, E, a_ptr, net.act[layer - 1]);
            if (live != nullptr && !zero) live[p] = 1;
            lay.finish_row(p, b);
        }
    }

    // ---- constants as reference + offset (float path, hidden -> hidden layers) -----
    // The boxes of a tile are neighbours in the bisection tree, so their
    // constants are close.  Box 0's float-float constants go to sRef; every
    // other box keeps delta = (h + l) - (h_0 + l_0) in its constant column,
    // which the contraction then multiplies by W with the coefficients.  The
    // rounding of delta joins the row's E, and |delta| its magnitude N (the
    // product's rounding is bounded by gamma |W| N).  Box 0's own constant
    // column is left unchanged and ignored after the product.
    // `live` (nullable): rows with live[i] == 0 are zero in every box and are
    // left out of every sum of the next product, so they are skipped here.
    template <class L>
    static __device__ void delta_prep(const L &lay, Real *sRef, const NetParams<Real> &net, int layer,
                                      const int *live = nullptr) {
        const int d = dim_of(net);
        const int n_in = net.n[layer];
        const int nmp = net.n_max_pad;
        for (int item = threadIdx.x; item < n_in * T; item += NT) {
            const int i = item / T;
            const int b = item - i * T;
            if (live != nullptr && live[i] == 0) continue;
            const auto Rb = lay.row(i, b);
            const auto R0 = lay.row(i, 0);
            const Real hr = R0(cCh(d)), lr = R0(cCl(d));
            if (b == 0) {
                sRef[i] = hr;
                sRef[nmp + i] = lr;
                continue;
            }
            const Real h = Rb(cCh(d)), l = Rb(cCl(d));
            Real s, e;
            two_sum<Real>(h, -hr, s, e);
            const Real dl = l - lr;
            const Real t = e + dl;
            const Real dv = s + t;
            const Real err = A::add_up(A::add_up(uerr<Real>(A::add_up(A::abs(l), A::abs(lr))), uerr<Real>(A::abs(t))),
                                       uerr<Real>(A::abs(dv)));
            Rb(cCh(d)) = dv;
            Rb(cE(d)) = A::add_up(Rb(cE(d)), err);
            Rb(cN(d)) = A::add_up(Rb(cN(d)), A::abs(dv));
        }
    }

    // One output row's constant at the reference box: sum_i W[p][i] (h_i + l_i) + b_p,
    // error-free products and compensated sums, written to slot b = 0 of sConst.
    // over the input rows ridx[0 .. n_rows) (the others are zero in every box)
    // On the property layer the error slot also takes the fold's share at the
    // reference constant, sum_i delta_pi (|h_i| + |l_i|) + the bias fold bound,
    // delta_pi staged in column n_out + p of sW (see final_rows).
    static __device__ __forceinline__ void ref_item(Real *sConst, const Real *sRef, const Real *sW, int Mpad,
                                                    const NetParams<Real> &net, int layer, int p, const int *ridx,
                                                    int n_rows) {
        const int n_in = net.n[layer];
        const int nmp = net.n_max_pad;
        const bool last = layer + 1 == net.K;
        const int pf = net.n[layer + 1] + p;
        Real s = net.b[layer][p], e = 0, a = A::abs(s), f = 0;
        for (int ii = 0; ii < n_rows; ++ii) {
            const int i = ridx[ii];
            const Real w = sW[i * Mpad + p];
            const Real h = sRef[i], l = sRef[nmp + i];
            Real p1, pe, t, se;
            two_prod<Real>(w, h, p1, pe);
            two_sum<Real>(s, p1, t, se);
            s = t;
            e = A::fma_rn(w, l, e + (pe + se));
            a = a + A::abs(p1);
            if (last) f = A::add_up(f, A::mul_up(sW[i * Mpad + pf], A::add_up(A::abs(h), A::abs(l))));
        }
        const Real g = gam<Real>(n_in + 2);
        Real hi, lo;
        two_sum<Real>(s, e, hi, lo);
        sConst[p * T] = hi;
        sConst[(nmp + p) * T] = lo;
        Real err = A::mul_up(A::mul_up((Real)2 * g, g), A::mul_up(a, (Real)1 + gam<Real>(n_in)));
        if (last) err = A::add_up(err, A::add_up(f, net.fold_berr[p]));
        sConst[(2 * nmp + p) * T] = err;
    }

    // ---- C' = W C, R' = |W| R over the coefficient, N and E columns ---------------
    // The constant of C is not part of this product: const_item computes it
    // with error-free transformations.  The state is updated in place: every
    // thread first accumulates its (at most kItems) 8 x 4 tiles in registers,
    // then, after a barrier, overwrites the rows.
    static constexpr int kItems = KI;

    // Row group g and column quad q (q < QW: W products, else |W|) of product
    // tile `item`.  The divisions by QW and QA are multiplications by their
    // reciprocals rW = ceil(2^32 / QW), rA = ceil(2^32 / QA) keeping the high
    // word: exact for item < 2^32 / QW, far beyond the tiles of one CTA.
    static __device__ __forceinline__ uint32_t recip32(int q) { return 0xFFFFFFFFu / (uint32_t)q + 1u; }
    static __device__ __forceinline__ void item_tile(int item, int G, int QW, int QA, uint32_t rW, uint32_t rA,
                                                     int &g, int &q) {
        const int nW = G * QW;
        if (item < nW) {
            g = (int)__umulhi((uint32_t)item, rW);
            q = item - g * QW;
        } else {
            const int k = item - nW;
            g = (int)__umulhi((uint32_t)k, rA);
            q = QW + (k - g * QA);
        }
    }

    // The same product over the rows of a list: rows[ii] = byte offsets (i Mpad,
    // i NS) of the rows i to sum over; a row that is zero in every box of the
    // tile adds exact zeros, so leaving it out changes no sum.
    static __device__ __forceinline__ void tile_mac_rows(const Real *wp, const Real *xp, const int2 *rows, int n_rows,
                                                         bool is_abs, Real (&acc)[8][4]) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = 0;
        const uint32_t w0 = (uint32_t)__cvta_generic_to_shared(wp), x0 = (uint32_t)__cvta_generic_to_shared(xp);
        if (is_abs) {
#pragma unroll 2
            for (int ii = 0; ii < n_rows; ++ii) {
                const int2 o = rows[ii];
                Real a0[4], a1[4], x[4];
                lds4<Real>(w0 + (uint32_t)o.x, a0);
                lds4<Real>(w0 + (uint32_t)o.x + 4 * (uint32_t)sizeof(Real), a1);
                lds4<Real>(x0 + (uint32_t)o.y, x);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        acc[r][c] = A::fma_rn(A::abs(a0[r]), x[c], acc[r][c]);
                        acc[r + 4][c] = A::fma_rn(A::abs(a1[r]), x[c], acc[r + 4][c]);
                    }
                }
            }
        } else {
#pragma unroll 2
            for (int ii = 0; ii < n_rows; ++ii) {
                const int2 o = rows[ii];
                Real a0[4], a1[4], x[4];
                lds4<Real>(w0 + (uint32_t)o.x, a0);
                lds4<Real>(w0 + (uint32_t)o.x + 4 * (uint32_t)sizeof(Real), a1);
                lds4<Real>(x0 + (uint32_t)o.y, x);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        acc[r][c] = A::fma_rn(a0[r], x[c], acc[r][c]);
                        acc[r + 4][c] = A::fma_rn(a1[r], x[c], acc[r + 4][c]);
                    }
                }
            }
        }
    }

    static __device__ __forceinline__ void tile_mac(const Real *wp, const Real *xp, int n_in, int Mpad, int NS,
                                                    bool is_abs, Real (&acc)[8][4]) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = 0;
        if (is_abs) {
#pragma unroll 2
            for (int i = 0; i < n_in; ++i) {
                Real a0[4], a1[4], x[4];
                V4<Real>::ld(wp + i * Mpad, a0);
                V4<Real>::ld(wp + i * Mpad + 4, a1);
                V4<Real>::ld(xp + i * NS, x);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        acc[r][c] = A::fma_rn(A::abs(a0[r]), x[c], acc[r][c]);
                        acc[r + 4][c] = A::fma_rn(A::abs(a1[r]), x[c], acc[r + 4][c]);
                    }
                }
            }
        } else {
#pragma unroll 2
            for (int i = 0; i < n_in; ++i) {
                Real a0[4], a1[4], x[4];
                V4<Real>::ld(wp + i * Mpad, a0);
                V4<Real>::ld(wp + i * Mpad + 4, a1);
                V4<Real>::ld(xp + i * NS, x);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        acc[r][c] = A::fma_rn(a0[r], x[c], acc[r][c]);
                        acc[r + 4][c] = A::fma_rn(a1[r], x[c], acc[r + 4][c]);
                    }
                }
            }
        }
    }

    // The next layer's constants (n_const items of const_item) share the phase:
    // they fill the threads that hold fewer product tiles, and they read the
    // state before the barrier like the tiles do.
    // `rows`: the input rows to sum over (see tile_mac_rows), n_rows of them,
    // and ridx their indices.
    template <class L>
    static __device__ void contract(const L &lay, Real *sConst, const Real *sRef, const NetParams<Real> &net,
                                    int layer, Real *S, const Real *sW, int n_in, int Mpad, int d, int NS,
                                    bool delta, uint32_t rW, uint32_t rA, const int2 *rows, const int *ridx,
                                    int n_rows) {
        const int QW = (d + 1) * T / 4;       // quads of C coefficient columns and the constant column
        const int QA = (d + 3) * T / 4;       // quads of R, N, E columns
        const int Q = QW + QA;
        const int G = Mpad / 8;               // groups of 8 output rows
        const int total = G * Q;
        // items: first every W product tile, then every |W| one, each row-group
        // major, so that the branch below diverges in one warp only and a warp's
        // lanes share their weights and write neighbouring columns
        const int n_const = delta ? net.n[layer + 1] : ((net.n[layer + 1] + 1) / 2) * T;
        Real acc[kItems][8][4];
        // few tiles (the property rows; the re-check's small tiles): each
        // tile's inputs in 2 or 4 parts on neighbouring lanes, added in a fixed
        // order ((p0 + p1) + (p2 + p3)) after the products
        const int parts = (4 * total <= NT && n_in >= 16) ? 4 : ((2 * total <= NT && n_in >= 8) ? 2 : 1);
        const bool split = parts > 1;
        const int busy = parts * total;   // threads busy with products
        if (split) {
            const int item = (int)threadIdx.x / parts, part = (int)threadIdx.x % parts;
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[0][r][c] = 0;
            if (item < total) {
                int g, q;
                item_tile(item, G, QW, QA, rW, rA, g, q);
                const bool is_abs = q >= QW;
                const int j0 = is_abs ? (d + 1) * T + (q - QW) * 4 : q * 4;
                const int i0 = part * n_rows / parts, i1 = (part + 1) * n_rows / parts;
                tile_mac_rows(sW + g * 8, S + j0, rows + i0, i1 - i0, is_abs, acc[0]);
            }
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    acc[0][r][c] += __shfl_xor_sync(0xffffffffu, acc[0][r][c], 1);
                    if (parts == 4) acc[0][r][c] += __shfl_xor_sync(0xffffffffu, acc[0][r][c], 2);
                }
        } else {
#pragma unroll
            for (int it = 0; it < kItems; ++it) {
                const int item = threadIdx.x + it * NT;
                if (item < total) {
                    int g, q;
                    item_tile(item, G, QW, QA, rW, rA, g, q);
                    const bool is_abs = q >= QW;
                    const int j0 = is_abs ? (d + 1) * T + (q - QW) * 4 : q * 4;
                    tile_mac_rows(sW + g * 8, S + j0, rows, n_rows, is_abs, acc[it]);
                }
            }
        }
        // combined index space [0, busy + n_const): indices past `busy` are constants
        {
            int idx = threadIdx.x + ((busy - (int)threadIdx.x + NT - 1) / NT) * NT;
            if (idx < busy) idx += NT;
            for (; idx < busy + n_const; idx += NT) {
                if (delta) ref_item(sConst, sRef, sW, Mpad, net, layer, idx - busy, ridx, n_rows);
                else const_item<true>(lay, sConst, sW, Mpad, net, layer, idx - busy, ridx, n_rows);
            }
        }
        __syncthreads();
        if (split) {
            const int item = (int)threadIdx.x / parts;
            if ((int)threadIdx.x % parts == 0 && item < total) {
                int g, q;
                item_tile(item, G, QW, QA, rW, rA, g, q);
                const int j0 = q >= QW ? (d + 1) * T + (q - QW) * 4 : q * 4;
#pragma unroll
                for (int r = 0; r < 8; ++r) V4<Real>::st(S + (g * 8 + r) * NS + j0, acc[0][r]);
            }
            return;
        }
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const int item = threadIdx.x + it * NT;
            if (item < total) {
                int g, q;
                item_tile(item, G, QW, QA, rW, rA, g, q);
                const int j0 = q >= QW ? (d + 1) * T + (q - QW) * 4 : q * 4;
#pragma unroll
                for (int r = 0; r < 8; ++r) V4<Real>::st(S + (g * 8 + r) * NS + j0, acc[it][r]);
            }
        }
    }

    // ---- float64 tile: hidden -> hidden products as float-float pairs -----------
    // The float64 pipes are a small fraction of the float32 ones; the
    // products, most of a layer's float64 work, run on the float32 pipes
    // instead: every input x of the state is split into float hi + lo
    // (x - hi is exact, lo = fl(x - hi): |x - hi - lo| <= 2^-48 |x| + 2^-150),
    // each term w hi is formed exactly, and the sums carry a float error term
    // (ff_mac).  The result hi + lo, rounded to float64, is within
    // gam_ff(n) sum_i |w_i| |x_i| + ff_abs of the exact product: the
    // contraction's rounding bound that the next epilogue takes in place of
    // gamma_n.

    // The state's product columns (0 .. 2d + 3) of rows 0 .. n_in - 1 as planes
    // of row stride NP (eval_plane_stride: rows on 16 bytes).
    static __device__ void split_state(const Real *S, float *Xh, float *Xl, int n_in, int NS, int NP, int d) {
        const int per = (2 * d + 4) * T;
        for (int item = threadIdx.x; item < n_in * per; item += NT) {
            const int i = item / per;
            const int j = item - i * per;
            const double x = (double)S[i * NS + j];
            const float h = __double2float_rn(x);
            Xh[i * NP + j] = h;
            Xl[i * NP + j] = __double2float_rn(__dsub_rn(x, (double)h));
        }
    }

    // An 8 x 4 product tile over the input rows ridx[0 .. n_rows) (see
    // tile_mac_rows): float weights of row stride Mpad, planes of stride NP.
    static __device__ __forceinline__ void tile_mac_rows_ff(const float *wp, const float *xh, const float *xl,
                                                            const int *ridx, int n_rows, int Mpad, int NP,
                                                            bool is_abs, float (&sh)[8][4], float (&sl)[8][4]) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) sh[r][c] = sl[r][c] = 0.f;
        const uint32_t w0 = (uint32_t)__cvta_generic_to_shared(wp);
        const uint32_t h0 = (uint32_t)__cvta_generic_to_shared(xh), l0 = (uint32_t)__cvta_generic_to_shared(xl);
        for (int ii = 0; ii < n_rows; ++ii) {
            const uint32_t i = (uint32_t)ridx[ii];
            const uint32_t ow = i * (uint32_t)(Mpad * 4), ox = i * (uint32_t)(NP * 4);
            float a0[4], a1[4], h[4], l[4];
            lds4<float>(w0 + ow, a0);
            lds4<float>(w0 + ow + 16u, a1);
            lds4<float>(h0 + ox, h);
            lds4<float>(l0 + ox, l);
            if (is_abs) {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    a0[r] = fabsf(a0[r]);
                    a1[r] = fabsf(a1[r]);
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    ff_mac(a0[r], h[c], l[c], sh[r][c], sl[r][c]);
                    ff_mac(a1[r], h[c], l[c], sh[r + 4][c], sl[r + 4][c]);
                }
        }
    }

    // hi + lo of a finished tile into the state, all but the constant column
    // (its product is not used; the constants' items read that column of the
    // input rows during this phase, so it is left alone).
    static __device__ __forceinline__ void store_ff(Real *S, int g, int j0, int d, int NS, const float (&sh)[8][4],
                                                    const float (&sl)[8][4]) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = j0 + c;
            if (j / T == d) continue;
#pragma unroll
            for (int r = 0; r < 8; ++r) S[(g * 8 + r) * NS + j] = (Real)__dadd_rn((double)sh[r][c], (double)sl[r][c]);
        }
    }

    // The phase of contract() with float-float products.  No product reads
    // the state (they read the planes), so each tile is stored as soon as it
    // is done; the constants (float64, as in contract) read the constant
    // columns, which no tile writes.
    template <class L>
    static __device__ void contract_ff(const L &lay, Real *sConst, const NetParams<Real> &net, int layer, Real *S,
                                       const float *sWf, const float *Xh, const float *Xl, int n_in, int Mpad,
                                       int d, int NS, int NP, uint32_t rW, uint32_t rA, const int *ridx,
                                       int n_rows) {
        const int QW = (d + 1) * T / 4;
        const int QA = (d + 3) * T / 4;
        const int Q = QW + QA;
        const int G = Mpad / 8;
        const int total = G * Q;
        const int n_const = ((net.n[layer + 1] + 1) / 2) * T;
        const int parts = (4 * total <= NT && n_in >= 16) ? 4 : ((2 * total <= NT && n_in >= 8) ? 2 : 1);
        const int busy = parts * total;
        float sh[8][4], sl[8][4];
        if (parts > 1) {
            const int item = (int)threadIdx.x / parts, part = (int)threadIdx.x % parts;
            int g = 0, q = 0, j0 = 0;
            if (item < total) {
                item_tile(item, G, QW, QA, rW, rA, g, q);
                const bool is_abs = q >= QW;
                j0 = is_abs ? (d + 1) * T + (q - QW) * 4 : q * 4;
                const int i0 = part * n_rows / parts, i1 = (part + 1) * n_rows / parts;
                tile_mac_rows_ff(sWf + g * 8, Xh + j0, Xl + j0, ridx + i0, i1 - i0, Mpad, NP, is_abs, sh, sl);
            } else {
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) sh[r][c] = sl[r][c] = 0.f;
            }
            // the parts' pairs added by TwoSum, in a fixed order
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    for (int m = 1; m < parts; m <<= 1) {
                        const float oh = __shfl_xor_sync(0xffffffffu, sh[r][c], m);
                        const float ol = __shfl_xor_sync(0xffffffffu, sl[r][c], m);
                        float t, se;
                        two_sum<float>(sh[r][c], oh, t, se);
                        sh[r][c] = t;
                        sl[r][c] = __fadd_rn(sl[r][c], __fadd_rn(ol, se));
                    }
                }
            if (item < total && part == 0) store_ff(S, g, j0, d, NS, sh, sl);
        } else {
#pragma unroll 1
            for (int it = 0; it < kItems; ++it) {
                const int item = threadIdx.x + it * NT;
                if (item < total) {
                    int g, q;
                    item_tile(item, G, QW, QA, rW, rA, g, q);
                    const bool is_abs = q >= QW;
                    const int j0 = is_abs ? (d + 1) * T + (q - QW) * 4 : q * 4;
                    tile_mac_rows_ff(sWf + g * 8, Xh + j0, Xl + j0, ridx, n_rows, Mpad, NP, is_abs, sh, sl);
                    store_ff(S, g, j0, d, NS, sh, sl);
                }
            }
        }
        {
            int idx = threadIdx.x + ((busy - (int)threadIdx.x + NT - 1) / NT) * NT;
            if (idx < busy) idx += NT;
            for (; idx < busy + n_const; idx += NT) const_item<true>(lay, sConst, sWf, Mpad, net, layer, idx - busy, ridx, n_rows);
        }
    }

    // ---- the same phase split over the CL CTAs of a thread-block cluster (float64) ----
    // Every CTA of the cluster holds the tile's whole state and does the
    // per-row work itself; the product tiles and the constant items are dealt
    // round-robin (item i to rank i mod CL), and each CTA writes its results
    // into the shared memory of every CTA of the cluster.  A product tile's
    // inputs are split over up to 8 lanes (at least 4 inputs each), added in
    // a fixed order.  Two cluster barriers: every CTA has read the state
    // before any overwrites it, and every CTA sees all results before the
    // next phase.
    template <int CL, class L>
    static __device__ void contract_cluster(const L &lay, Real *sConst, const NetParams<Real> &net, int layer,
                                            Real *S, const Real *sW, int n_in, int Mpad, int d, int NS,
                                            uint32_t rW, uint32_t rA) {
        static_assert(sizeof(Real) == 8, "cluster contraction is the float64 re-check's");
        const int QW = (d + 1) * T / 4;
        const int QA = (d + 3) * T / 4;
        const int G = Mpad / 8;
        const int total = G * (QW + QA);
        const int rank = (int)cluster_ctarank();
        const int most = (total + CL - 1) / CL;   // product tiles of rank 0, the most of any rank
        int parts = 1;
        while (parts < 8 && 2 * parts * most <= NT && n_in >= 8 * parts) parts *= 2;
        const int busy = parts * most;
        const int n_out = net.n[layer + 1];
        const int n_const = ((n_out + 1) / 2) * T;
        const int my_const = (n_const - rank + CL - 1) / CL;
        const int li = (int)threadIdx.x / parts, part = (int)threadIdx.x % parts;
        const int item = rank + CL * li;
        const bool has = (int)threadIdx.x < busy && item < total;
        Real acc[8][4];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = 0;
        int g = 0, q = 0;
        if (has) {
            item_tile(item, G, QW, QA, rW, rA, g, q);
            const bool is_abs = q >= QW;
            const int j0 = is_abs ? (d + 1) * T + (q - QW) * 4 : q * 4;
            const int i0 = part * n_in / parts, i1 = (part + 1) * n_in / parts;
            tile_mac(sW + g * 8 + i0 * Mpad, S + j0 + i0 * NS, i1 - i0, Mpad, NS, is_abs, acc);
        }
        for (int m = 1; m < parts; m *= 2) {
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] += __shfl_xor_sync(0xffffffffu, acc[r][c], m);
        }
        // this rank's constant items on the threads past the products
        for (int t = (int)threadIdx.x - busy; t < my_const; t += NT)
            if (t >= 0) const_item(lay, sConst, sW, Mpad, net, layer, rank + CL * t);
        __syncthreads();
        cluster_barrier();
        if (has && part == 0) {
            const int j0 = q >= QW ? (d + 1) * T + (q - QW) * 4 : q * 4;
#pragma unroll 1
            for (int c = 0; c < CL; ++c) {
#pragma unroll
                for (int r = 0; r < 8; ++r) st_cluster4(cluster_map(S + (g * 8 + r) * NS + j0, c), acc[r]);
            }
        }
        const int nmp = net.n_max_pad;
        for (int t = (int)threadIdx.x - busy; t < my_const; t += NT) {
            if (t < 0) continue;
            const int ci = rank + CL * t;
            const int qq = ci / T, b = ci - qq * T;
            for (int p = 2 * qq; p < 2 * qq + 2 && p < n_out; ++p) {
                for (int k = 0; k < 3; ++k) {
                    const Real *v = sConst + (k * nmp + p) * T + b;
                    for (int c = 0; c < CL; ++c)
                        if (c != rank) st_cluster(cluster_map(v, c), *v);
                }
            }
        }
        cluster_barrier();
    }

    // Starts the copy of a layer's weight image (n_in x Mpad, already padded
    // in global memory) into sW: 16-byte cp.async pieces spread over the
    // threads, L2 only.  The epilogue runs while they land; stage_wait, then
    // a block barrier, make sW readable.  n_in Mpad sizeof(Real) is a multiple
    // of 32 bytes (Mpad of 8), and both ends are 16-byte aligned.
    template <typename W>
    static __device__ __forceinline__ void stage_weights_async(void *sW, const W *Ws, int n_in, int Mpad) {
        const int pieces = n_in * Mpad * (int)sizeof(W) / 16;
        const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(sW);
        const char *g0 = reinterpret_cast<const char *>(Ws);
        for (int c = threadIdx.x; c < pieces; c += NT) {
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s0 + 16u * (uint32_t)c),
                         "l"(g0 + 16 * (size_t)c)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    static __device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

    // ---- property rows: constant, error (incl. the fold), sound bounds ----------
    // `delta`: the property layer ran in reference + offset form with the
    // fold's error bounds fe in the weight image's padding columns, so that
    // rows R + r of the product hold sum_i fe_ri N_i and sum_i fe_ri E_i over
    // the offset rows.  With |h_i + l_i| <= |h_i^0| + |l_i^0| + |delta_i| + err_i
    // (box 0's constant, the offset, its rounding: the last two joined N_i and
    // E_i in delta_prep), the fold's share sum_i fe_ri (N_i + |h_i + l_i| + E_i)
    // is at most the reference term of ref_item plus those two sums, which
    // add non-negative terms rounded to nearest: each at most its computed
    // value (1 + 2 gcoef), plus n_in underflows.
    template <class L>
    static __device__ void final_rows(const L &lay, const Real *sConst, const NetParams<Real> &net, Real gcoef,
                                      Real *sLo, Real *sHi, Real *sErr, bool delta = false) {
        const int d = dim_of(net);
        const int R = net.R;
        const int K = net.K;
        const int n_in = net.n[K - 1];
        for (int item = threadIdx.x; item < R * T; item += NT) {
            const int r = item / T;
            const int b = item - r * T;
            const auto Rw = lay.row(r, b);
            Real chi, clo, E;
            if (K > 1) {
                finish_contraction(Rw, sConst, net.n_max_pad, r, b, d, n_in, gcoef, chi, clo, E, delta);
                if (delta) {
                    const auto Rf = lay.row(R + r, b);
                    const Real fz = A::mul_up(A::add_up(Rf(cN(d)), Rf(cE(d))), (Real)1 + (Real)2 * gcoef);
                    E = A::add_up(E, A::add_up(fz, (Real)(2 * n_in) * A::tiny));
                }
            } else {
                chi = Rw(cCh(d));
                clo = Rw(cCl(d));
                E = Rw(cE(d));
            }
            RowBounds<Real> bd;
            bd.compute(Rw, d, chi, clo);
            sLo[r * T + b] = A::add_dn(bd.ll, -E);
            sHi[r * T + b] = A::add_up(bd.uu, E);
            sErr[r * T + b] = A::add_up(E, bd.delta);
        }
    }
};

// Class of a box from its row bounds (Sec. 3 containment check): UNSAFE if
// some clause has all rows satisfied on the whole box, SAFE if every clause
// has a row violated on the whole box, UNDECIDED otherwise.
template <typename Real, int T>
__device__ __forceinline__ uint8_t classify_rows(const NetParams<Real> &net, const Real *sLo, const Real *sHi,
                                                 const Real *sErr, int b, Real shift) {
    bool any_in = false, all_out = true;
    int r0 = 0;
    for (int cl = 0; cl < net.n_clauses; ++cl) {
        const int r1 = net.clause_end[cl];
        bool all_in = true, some_out = false;
        for (int r = r0; r < r1; ++r) {
            const Real e2 = shift * sErr[r * T + b];
            const Real lo = sLo[r * T + b] + e2;
            const Real hi = sHi[r * T + b] - e2;
            const bool st = net.strict[r] != 0;
            all_in = all_in && (st ? (lo > (Real)0) : (lo >= (Real)0));
            some_out = some_out || (st ? (hi <= (Real)0) : (hi < (Real)0));
        }
        any_in = any_in || all_in;
        all_out = all_out && some_out;
        r0 = r1;
    }
    return any_in ? kUnsafe : (all_out ? kSafe : kUndecided);
}

// ---------------------------------------------------------------------------
// Shared-memory views of one tile, carved from the dynamic allocation for the
// largest shapes the launch serves.
// ---------------------------------------------------------------------------
template <typename Real>
struct TileSmem {
    Real *sS, *sConst, *sRef, *sW, *sMh, *sMl, *sR, *sLo, *sHi, *sErr;
    int64_t *sIdx;
    int2 *sRows;    // input rows of the next product: byte offsets (i Mpad, i NS)
    int *sRowIdx;   // the same rows' indices i
    int *sLive;     // per row: not identically zero in some box of the tile
    int *sNRows;    // length of sRows
    float *sXh, *sXl;   // float64 tile: the state as float hi + lo planes (allocated where
                        // pass 2 runs: the single-problem kernel with that footprint)
};

template <typename Real, int T>
__device__ __forceinline__ TileSmem<Real> carve_smem(unsigned char *sp, int nmp, int d, int n_in_max, int R) {
    TileSmem<Real> m;
    const int NS = state_stride(T, d);
    m.sXh = m.sXl = nullptr;
    if (sizeof(Real) == 8) {
        m.sXh = reinterpret_cast<float *>(sp + eval_split_offset(T, d, R, nmp, n_in_max));
        m.sXl = m.sXh + (size_t)nmp * eval_plane_stride(T, d);
    }
    m.sS = reinterpret_cast<Real *>(sp);
    sp += (size_t)nmp * NS * sizeof(Real);
    m.sConst = reinterpret_cast<Real *>(sp);
    sp += 3 * (size_t)nmp * T * sizeof(Real);
    m.sRef = reinterpret_cast<Real *>(sp);
    sp += 2 * (size_t)nmp * sizeof(Real);
    m.sW = reinterpret_cast<Real *>(sp);
    sp += (size_t)n_in_max * nmp * sizeof(Real);
    m.sMh = reinterpret_cast<Real *>(sp);
    sp += (size_t)T * d * sizeof(Real);
    m.sMl = reinterpret_cast<Real *>(sp);
    sp += (size_t)T * d * sizeof(Real);
    m.sR = reinterpret_cast<Real *>(sp);
    sp += (size_t)T * d * sizeof(Real);
    m.sLo = reinterpret_cast<Real *>(sp);
    sp += (size_t)T * R * sizeof(Real);
    m.sHi = reinterpret_cast<Real *>(sp);
    sp += (size_t)T * R * sizeof(Real);
    m.sErr = reinterpret_cast<Real *>(sp);
    sp += (size_t)T * R * sizeof(Real);
    m.sIdx = reinterpret_cast<int64_t *>(sp);
    sp += (size_t)T * sizeof(int64_t);
    m.sRows = reinterpret_cast<int2 *>(sp);
    sp += (size_t)nmp * sizeof(int2);
    m.sRowIdx = reinterpret_cast<int *>(sp);
    sp += (size_t)nmp * sizeof(int);
    m.sLive = reinterpret_cast<int *>(sp);
    sp += (size_t)nmp * sizeof(int);
    m.sNRows = reinterpret_cast<int *>(sp);
    return m;
}

__device__ __forceinline__ int64_t source_count(const BoxSource &src) {
    int64_t n;
    if (src.index != nullptr) {
        n = (int64_t)*src.index_count;
    } else if (src.mode == 0) {
        n = (int64_t)*src.count;
    } else {
        n = src.n_explicit;
    }
    return n > src.cap ? src.cap : n;
}

// ---------------------------------------------------------------------------
// One tile: boxes base .. base + T - 1 of the source (n boxes in all).
// pass 0: working precision; writes the sound class and lists the undecided
//         boxes whose class depends on E (their optimistic class differs);
// pass 2: float64 with float-float hidden products (see contract_ff): writes
//         the class and lists the boxes whose class still depends on E;
// pass 1: re-check of such a list in the higher precision (writes the class,
//         counts the boxes still depending on E as ties).
// ---------------------------------------------------------------------------
// kPairs: pass 2 is compiled in (the single-problem float64 kernel).
template <typename Real, int T, int NT, int KI = 2, int CL = 1, int DC = 0, bool kPairs = false>
__device__ void eval_tile(const NetParams<Real> &net, const BoxSource &src, const EvalOutputs &out, const int pass,
                          const TileSmem<Real> &sm, const int64_t base, const int64_t n) {
    using A = Arith<Real>;
    using Tile = EvalTile<Real, T, NT, KI, DC>;
    const int d = Tile::dim_of(net);
    const int R = net.R;
    const int NS = state_stride(T, d);
    Real *sS = sm.sS, *sConst = sm.sConst, *sW = sm.sW, *sMh = sm.sMh, *sMl = sm.sMl, *sR = sm.sR;
    Real *sLo = sm.sLo, *sHi = sm.sHi, *sErr = sm.sErr;
    int64_t *sIdx = sm.sIdx;
    const int nb = (int)((n - base) < T ? (n - base) : T);
    if (threadIdx.x < T) {
        const int64_t k = base + (threadIdx.x < nb ? threadIdx.x : 0);
        sIdx[threadIdx.x] = src.index != nullptr ? src.index[k] : k;
    }
    for (int i = threadIdx.x; i < net.n_max_pad; i += NT) sm.sLive[i] = 0;
    __syncthreads();

    // ---- boxes: centre (hi + lo) and radius, outward ----------------------
    for (int item = threadIdx.x; item < T * d; item += NT) {
        const int b = item / d;
        const int i = item - b * d;
        const int64_t idx = sIdx[b];
        double m64, r64, pad;
        if (src.mode == 0) {
            // Sec. 2.2 bisection: dimension i split c times, half index k
            unsigned long long k;
            int c;
            code_dim(src, src.codes[idx], i, k, c);
            const double w = src.root_w[i];
            const double a = src.root_lo[i];
            r64 = ldexp(w, -(c + 1));
            m64 = a + w * ldexp((double)(2 * k + 1), -(c + 1));
            pad = ldexp(fabs(m64) + fabs(a) + w, -50);
        } else {
            const double lo = (double)src.lo[idx * d + i];
            const double hi = (double)src.hi[idx * d + i];
            m64 = 0.5 * (lo + hi);
            r64 = 0.5 * (hi - lo);
            pad = ldexp(fabs(m64) + fabs(r64), -52);
        }
        Real mh, ml, r;
        split_centre<Real>(m64, r64, pad, mh, ml, r);
        sMh[b * d + i] = mh;
        sMl[b * d + i] = ml;
        sR[b * d + i] = r;
    }
    __syncthreads();

    const SimtLayout<Real, T> lay{sS, NS};
    Tile::init_layer(lay, net, sMh, sMl, sR);
    __syncthreads();

    // float: hidden -> hidden constants as a reference box's plus offsets
    constexpr bool dconst = Tile::kCompensated;
    // reciprocals of the product tiles' column-quad counts (see item_tile)
    const uint32_t rW = Tile::recip32((d + 1) * T / 4), rA = Tile::recip32((d + 3) * T / 4);
    int alpha_off = 0;
    bool pdelta = false;
    // rounding bound of the last contraction (relative, absolute)
    Real gprev = gam<Real>(net.n[0]), aprev = 0;
    for (int k = 1; k < net.K; ++k) {
        // the tile's products sum over a list of input rows: only the rows
        // that are not zero in every box of the tile (inactive ReLUs with no
        // error: their products, constants and fold terms are exact zeros, so
        // every sum is unchanged)
        const bool lk = k + 1 < net.K;        // a hidden -> hidden product
        const int n_out = net.n[k + 1];
        const int Mpad = (n_out + 7) & ~7;
        // float: the property layer too, when its weight image holds the
        // fold's error bounds in its padding columns (at most 4 property rows)
        const bool pk = dconst && !lk && net.fold_pad != 0;
        const bool dk = dconst && (lk || pk);
        // float64 tile, pass 2: hidden -> hidden products as float-float pairs
        const bool ffk = kPairs && sizeof(Real) == 8 && CL == 1 && pass == 2 && lk;
        // sW is free (the last product ended with a barrier): its next image
        // lands while the epilogue runs
        if (ffk) Tile::stage_weights_async(sW, net.Wsf[k], net.n[k], Mpad);
        else Tile::stage_weights_async(sW, net.Ws[k], net.n[k], Mpad);
        Tile::hidden_epilogue(lay, sConst, net, k, gprev, src.alpha, src.alpha_ld, base, n, alpha_off, dconst,
                              CL == 1 ? sm.sLive : nullptr, aprev);
        alpha_off += net.n[k];
        Tile::stage_wait();
        pdelta = pk;
        if (CL == 1) {
            __syncthreads();
            if (threadIdx.x < 32) {
                // the live rows in order (the flags are cleared in the product phase)
                const int lane = threadIdx.x;
                int count = 0;
                for (int i0 = 0; i0 < net.n[k]; i0 += 32) {
                    const int i = i0 + lane;
                    const bool lv = i < net.n[k] && sm.sLive[i] != 0;
                    const unsigned bal = __ballot_sync(0xffffffffu, lv);
                    if (lv) {
                        const int at = count + __popc(bal & ((1u << lane) - 1u));
                        sm.sRows[at] = make_int2(i * Mpad * (int)sizeof(Real), i * NS * (int)sizeof(Real));
                        sm.sRowIdx[at] = i;
                    }
                    count += __popc(bal);
                }
                if (lane == 0) *sm.sNRows = count;
            }
            if (dk) Tile::delta_prep(lay, sm.sRef, net, k, sm.sLive);
            if (ffk) Tile::split_state(sS, sm.sXh, sm.sXl, net.n[k], NS, eval_plane_stride(T, d), d);
        }
        __syncthreads();
        // the flags for the next layer's epilogue (read above, before the barrier)
        if (CL == 1)
            for (int i = threadIdx.x; i < net.n[k]; i += NT) sm.sLive[i] = 0;
        // constants and products; barrier inside, then the in-place store
        if constexpr (CL > 1) {
            static_assert(!Tile::kCompensated, "the cluster tile is the float64 re-check's");
            Tile::template contract_cluster<CL>(lay, sConst, net, k, sS, sW, net.n[k], Mpad, d, NS, rW, rA);
        } else {
            if (ffk) {
                Tile::contract_ff(lay, sConst, net, k, sS, reinterpret_cast<const float *>(sW), sm.sXh, sm.sXl,
                                  net.n[k], Mpad, d, NS, eval_plane_stride(T, d), rW, rA, sm.sRowIdx, *sm.sNRows);
            } else {
                Tile::contract(lay, sConst, sm.sRef, net, k, sS, sW, net.n[k], Mpad, d, NS, dk, rW, rA, sm.sRows,
                               sm.sRowIdx, *sm.sNRows);
            }
        }
        if constexpr (sizeof(Real) == 8) {
            gprev = ffk ? (Real)gam_ff(net.n[k]) : gam<Real>(net.n[k]);
            aprev = ffk ? (Real)ff_abs(net.wabs[k], net.n[k], d) : (Real)0;
        } else {
            gprev = gam<Real>(net.n[k]);
        }
        __syncthreads();
    }
    Tile::final_rows(lay, sConst, net, gam<Real>(net.n[net.K - 1]), sLo, sHi, sErr, pdelta);
    __syncthreads();

    // ---- classify (Sec. 3) and write (one CTA of a cluster) ----------------
    if (threadIdx.x < nb && (CL == 1 || cluster_ctarank() == 0)) {
        const int b = threadIdx.x;
        const uint8_t cls = classify_rows<Real, T>(net, sLo, sHi, sErr, b, (Real)0);
        // optimistic bounds (raw +- E inward): the class the exact SLR could have
        const uint8_t opt = classify_rows<Real, T>(net, sLo, sHi, sErr, b, (Real)2);
        const bool near = (cls == kUndecided) && (opt != kUndecided);
        const int64_t idx = sIdx[b];
        const int64_t oidx = out.by_position ? base + b : idx;
        if (out.cls != nullptr) out.cls[oidx] = cls;
        if (out.row_lo != nullptr) {
            for (int r = 0; r < R; ++r) {
                out.row_lo[oidx * R + r] = to_lo<Real>(sLo[r * T + b]);
                out.row_hi[oidx * R + r] = to_hi<Real>(sHi[r * T + b]);
            }
        }
        if (out.row_err != nullptr) {
            for (int r = 0; r < R; ++r) out.row_err[oidx * R + r] = to_hi<Real>(sErr[r * T + b]);
        }
        if (near) {
            if ((pass == 0 || pass == 2) && out.near_list != nullptr) {
                const unsigned long long pos = atomicAdd(out.near_count, 1ull);
                if ((int64_t)pos < out.near_cap) {
                    out.near_list[pos] = idx;
                } else {
                    atomicOr(out.status, kStatusNearOverflow);
                }
            } else if (pass == 1 && out.tie_count != nullptr) {
                atomicAdd(out.tie_count, 1ull);
            }
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// The kernel: persistent over tiles of one problem's boxes.
// ---------------------------------------------------------------------------
// Resident CTAs per SM the register budget is sized for: two with two product
// tiles per thread; with one tile per thread (small T) three CTAs of 256 or
// six of 128 threads.
template <typename Real, int NT, int KI>
constexpr int eval_min_blocks() {
    return sizeof(Real) != 4 ? 1 : (KI == 2 ? 2 : (NT == 256 ? 3 : 6));
}

template <typename Real, int T, int NT, int KI = 2, int DC = 0>
__global__ void __launch_bounds__(NT, (eval_min_blocks<Real, NT, KI>()))
slr_eval_kernel(const NetParams<Real> net, const BoxSource src, const EvalOutputs out, const int pass) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TileSmem<Real> sm =
        carve_smem<Real, T>(smem_raw, net.n_max_pad, DC > 0 ? DC : net.d, net.n_in_max, net.R);
    const int64_t n = source_count(src);
    for (int64_t base = (int64_t)blockIdx.x * T; base < n; base += (int64_t)gridDim.x * T)
        eval_tile<Real, T, NT, KI, 1, DC, sizeof(Real) == 8>(net, src, out, pass, sm, base, n);
}

// The float64 re-check with each tile on a cluster of kRecheckCluster CTAs (one
// per SM): the few boxes of a level's re-check list then take several SMs'
// float64 units each instead of one.  Every CTA of a cluster runs the same
// tiles, so all reach the same cluster barriers; the last barrier keeps each
// CTA resident until no peer can still write to its shared memory.
template <typename Real, int T, int NT>
__global__ void __cluster_dims__(kRecheckCluster, 1, 1) __launch_bounds__(NT, 1)
slr_eval_cluster_kernel(const NetParams<Real> net, const BoxSource src, const EvalOutputs out, const int pass) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TileSmem<Real> sm = carve_smem<Real, T>(smem_raw, net.n_max_pad, net.d, net.n_in_max, net.R);
    const int64_t n = source_count(src);
    const int64_t c = cluster_index_x(), nc = cluster_count_x();
    for (int64_t base = c * T; base < n; base += nc * T)
        eval_tile<Real, T, NT, 2, kRecheckCluster>(net, src, out, pass, sm, base, n);
    cluster_barrier();
}

// ---------------------------------------------------------------------------
// Batched kernel: tiles of many problems in one persistent launch.  Tile g
// belongs to the problem p with tile_prefix[p] <= g < tile_prefix[p + 1]
// (tiles never mix problems); its network, source and outputs are copied to
// shared memory when the problem changes.
// ---------------------------------------------------------------------------
template <typename Real, int T, int NT>
__global__ void __launch_bounds__(NT, (eval_min_blocks<Real, NT, 2>()))
slr_eval_batch_kernel(const NetParams<Real> *__restrict__ nets, const BoxSource *__restrict__ srcs,
                      const EvalOutputs *__restrict__ outs, const int P, const long long *__restrict__ tile_prefix,
                      const BatchShape shape, const int pass) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ NetParams<Real> snet;
    __shared__ BoxSource ssrc;
    __shared__ EvalOutputs sout;
    __shared__ int s_p;
    __shared__ long long s_base;
    const TileSmem<Real> sm = carve_smem<Real, T>(smem_raw, shape.nmp, shape.d, shape.n_in_max, shape.R);
    const long long total = tile_prefix[P];
    int cur = -1;
    for (long long g = blockIdx.x; g < total; g += gridDim.x) {
        if (threadIdx.x == 0) {
            int lo = 0, hi = P;   // largest p with tile_prefix[p] <= g
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (tile_prefix[mid] <= g) lo = mid;
                else hi = mid;
            }
            s_p = lo;
            s_base = (g - tile_prefix[lo]) * T;
        }
        __syncthreads();
        const int p = s_p;
        if (p != cur) {
            const int *from = reinterpret_cast<const int *>(&nets[p]);
            int *to = reinterpret_cast<int *>(&snet);
            for (int i = threadIdx.x; i < (int)(sizeof(NetParams<Real>) / 4); i += NT) to[i] = from[i];
            if (threadIdx.x == 0) {
                ssrc = srcs[p];
                sout = outs[p];
            }
            cur = p;
            __syncthreads();
        }
        eval_tile<Real, T, NT>(snet, ssrc, sout, pass, sm, s_base, source_count(ssrc));
    }
}

}  // namespace slr
