// Fused SLR evaluation of a tile of boxes held in shared memory.
//
// One CTA takes a tile of T boxes and carries their symbolic state through all
// layers without leaving the SM:
//   decode     path code -> box centre m and radius r (outward to Real)
//   layer 1    C = [W_1 diag(r) | W_1 m + b_1], R = [0 | rounding error]
//   per hidden layer k:
//     widen    add the a-priori error of the contraction that produced it
//     bounds   concrete bounds of both equations over the box (Sec. 2.2):
//              max/min of (C +- R) = const +- sum_j |coeff_j|, directed rounding
//     relax    ReLU relaxation, Eq. 1 (per-equation or one-pair reading)
//     contract C' = W C + b, R' = |W| R (the per-layer symbolic matrix product)
//   last layer the property rows are folded into W_K; row bounds lo_r, hi_r
//   classify  Sec. 3 containment check: UNSAFE / SAFE / UNDECIDED, and flag
//              undecided boxes whose margins lie within the rounding budget.
//
// State layout in shared memory: element (row p, column c, box b) at
// S[p * NS + c * T + b] with NS = T * (2d + 3).  Columns 0..d hold C (d
// coefficients, then the constant), d+1..2d+1 hold R, 2d+2 holds the row
// magnitude N = sum |C| + sum |R| (used by the next layer's error bound).
// Boxes are the fastest index so that a warp reads one column of 32 boxes
// (or 32/T rows of T boxes; NS/T = 2d+3 is odd, so those rows fall in distinct
// banks) without bank conflicts.
#pragma once

#include "slr_device.cuh"

namespace slr {

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

// Concrete bounds of the raw equations U = C + R, L = C - R of one row over
// the box (Sec. 2.2: const +- sum_j |coeff_j| in the normalised input), with
// outward rounding so that they bound the stored equations exactly.
template <typename Real, int T>
struct RowBounds {
    Real uu, lu, ul, ll;   // max U, min U, max L, min L
    Real NC, NR;           // sum |C_j| over coefficients, sum |R_j| incl. its constant
    __device__ __forceinline__ void compute(const Real *row, int d, Real chi, Real clo) {
        using A = Arith<Real>;
        Real SU = 0, SL = 0;
        NC = 0;
        NR = 0;
        const Real *rr = row + (d + 1) * T;
        for (int j = 0; j < d; ++j) {
            const Real c = row[j * T];
            const Real r = rr[j * T];
            SU = A::add_up(SU, A::abs(c + r));
            SL = A::add_up(SL, A::abs(c - r));
            NC = A::add_up(NC, A::abs(c));
            NR = A::add_up(NR, A::abs(r));
        }
        const Real rd = rr[d * T];
        NR = A::add_up(NR, A::abs(rd));
        // |c +- r| <= |fl(c +- r)| (1 + u): cover the round-to-nearest of each term
        SU = A::mul_up(SU, (Real)1 + A::ulp2);
        SL = A::mul_up(SL, (Real)1 + A::ulp2);
        uu = A::add_up(A::add_up(A::add_up(chi, rd), clo), SU);
        lu = A::add_dn(A::add_dn(A::add_dn(chi, rd), clo), -SU);
        ul = A::add_up(A::add_up(A::add_up(chi, -rd), clo), SL);
        ll = A::add_dn(A::add_dn(A::add_dn(chi, -rd), clo), -SL);
    }
};

template <typename Real, int T, int NT>
struct EvalTile {
    using A = Arith<Real>;

    // Column offsets of one row (times T in memory): C coefficients [0, d),
    // C constant hi (d), R coefficients [d+1, 2d+1), R constant (2d+1),
    // N (2d+2), E (2d+3), C constant lo (2d+4).
    static __device__ __forceinline__ int cCh(int d) { return d; }
    static __device__ __forceinline__ int cR(int d) { return d + 1; }
    static __device__ __forceinline__ int cRd(int d) { return 2 * d + 1; }
    static __device__ __forceinline__ int cN(int d) { return 2 * d + 2; }
    static __device__ __forceinline__ int cE(int d) { return 2 * d + 3; }
    static __device__ __forceinline__ int cCl(int d) { return 2 * d + 4; }

    // Constant of one output row as an exact-product, compensated sum:
    // sum_i W[p][i] (hi_i + lo_i) + bias, returned as a normalised pair, and a
    // bound of its rounding error (2 gamma^2 sum |terms|, Ogita-Rump-Oishi).
    static __device__ __forceinline__ void const_dot(const Real *sW, int Mpad, int p, const Real *hcol,
                                                     const Real *lcol, int n_in, int NS, Real bias,
                                                     Real &chi, Real &clo, Real &err) {
        Real s = bias, e = 0, sabs = A::abs(bias);
        for (int i = 0; i < n_in; ++i) {
            const Real w = sW[i * Mpad + p];
            const Real h = hcol[i * NS];
            const Real l = lcol[i * NS];
            Real p1, pe, t, se;
            two_prod<Real>(w, h, p1, pe);
            two_sum<Real>(s, p1, t, se);
            s = t;
            e = A::fma_rn(w, l, e + (pe + se));
            sabs = sabs + A::abs(p1);
        }
        two_sum<Real>(s, e, chi, clo);
        const Real g = gam<Real>(n_in + 2);
        err = A::mul_up(A::mul_up((Real)2 * g, g), A::mul_up(sabs, (Real)1 + gam<Real>(n_in)));
    }

    // ---- layer 1: C = [W_1 diag(r) | W_1 m + b_1], R = 0 ------------------------
    static __device__ void init_layer(Real *S, const NetParams<Real> &net, const Real *sMh,
                                      const Real *sMl, const Real *sR, int NS) {
        const int d = net.d;
        const int n1 = net.n[1];
        for (int item = threadIdx.x; item < n1 * T; item += NT) {
            const int p = item / T;
            const int b = item - p * T;
            Real *row = S + p * NS + b;
            const Real *w = net.W0 + (size_t)p * d;
            const Real bp = net.b[0][p];
            Real S1 = 0, s = bp, e = 0, sabs = A::abs(bp);
            for (int j = 0; j < d; ++j) {
                const Real wj = w[j];
                const Real c = A::mul_rn(wj, sR[b * d + j]);
                row[j * T] = c;
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
            row[cCh(d) * T] = chi;
            row[cCl(d) * T] = clo;
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
            Real *rr = row + cR(d) * T;
            for (int j = 0; j <= d; ++j) rr[j * T] = 0;
            row[cN(d) * T] = S1;
            row[cE(d) * T] = E;
        }
    }

    // ---- add the contraction's constant and error; returns (chi, clo, E) -------
    static __device__ __forceinline__ void finish_contraction(Real *row, const Real *Sprev, const Real *sW, int Mpad,
                                                              int p, int b, int d, int n_in, int NS, Real bias,
                                                              Real &chi, Real &clo, Real &E) {
        Real cerr;
        const_dot(sW, Mpad, p, Sprev + cCh(d) * T + b, Sprev + cCl(d) * T + b, n_in, NS, bias, chi, clo, cerr);
        // coefficients: a-priori gamma_n (sum_i |W_pi| N_i) from the |W| N column
        const Real wN = row[cN(d) * T];
        const Real g = gam<Real>(n_in);
        Real eps = A::mul_up(g, A::mul_up(wN, (Real)1 + g));
        eps = A::add_up(A::add_up(eps, cerr), (Real)(n_in + 4) * A::tiny);
        // |W| E was summed in round-to-nearest from non-negative terms
        E = A::add_up(A::mul_up(row[cE(d) * T], (Real)1 + (Real)2 * g), eps);
    }

    // ---- one hidden layer: constant, error, concrete bounds, ReLU relaxation ----
    static __device__ void hidden_epilogue(Real *S, const Real *Sprev, const Real *sW, int Mpad,
                                           const NetParams<Real> &net, int layer, int NS) {
        const int d = net.d;
        const int nrows = net.n[layer];
        const int n_in = net.n[layer - 1];
        const Real *bias = net.b[layer - 1];
        for (int item = threadIdx.x; item < nrows * T; item += NT) {
            const int p = item / T;
            const int b = item - p * T;
            Real *row = S + p * NS + b;
            Real *rr = row + cR(d) * T;
            Real chi, clo, E;
            if (layer > 1) {
                finish_contraction(row, Sprev, sW, Mpad, p, b, d, n_in, NS, bias[p], chi, clo, E);
            } else {
                chi = row[cCh(d) * T];
                clo = row[cCl(d) * T];
                E = row[cE(d) * T];
            }
            RowBounds<Real, T> bd;
            bd.compute(row, d, chi, clo);
            if (bd.ll >= (Real)0) {
                // stable active: relu is the identity on [L - E, U + E] up to
                // U + E >= lu + E >= 0, so the equations and E carry over
                row[cCh(d) * T] = chi;
                row[cCl(d) * T] = clo;
                row[cN(d) * T] = A::add_up(bd.NC, bd.NR);
                row[cE(d) * T] = E;
                continue;
            }
            if (bd.uu <= (Real)0) {
                // stable inactive: relu(z) lies in [0, max(0, uu + E)]
                for (int j = 0; j < d; ++j) row[j * T] = 0;
                for (int j = 0; j <= d; ++j) rr[j * T] = 0;
                row[cCh(d) * T] = 0;
                row[cCl(d) * T] = 0;
                row[cN(d) * T] = 0;
                const Real top = A::add_up(bd.uu, E);
                row[cE(d) * T] = top > (Real)0 ? top : (Real)0;
                continue;
            }
            // unstable: U' = sig_u (U - l) and L' = sig_l L (Eq. 1).  Applied to
            // U + E over [lu + E, uu + E] the chord misses relu by (1 - sig_u) E
            // and shifts by sig_u E, and sig_l (L - E) <= relu(L - E): E carries over.
            Real sig_u, sig_l, h;
            if (net.relax_mode == kRelaxPaperLiteral) {
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
                sig_l = bd.ul <= (Real)0 ? (Real)0 : A::div_rn(bd.ul, bd.ul - bd.ll);
            }
            sig_l = sig_l < (Real)0 ? (Real)0 : (sig_l > (Real)1 ? (Real)1 : sig_l);
            // (C, R) <- ((U' + L') / 2, (U' - L') / 2)
            const Real pp = (sig_u + sig_l) * (Real)0.5;
            const Real qq = (sig_u - sig_l) * (Real)0.5;
            for (int j = 0; j < d; ++j) {
                const Real c = row[j * T];
                const Real r = rr[j * T];
                row[j * T] = A::fma_rn(pp, c, qq * r);
                rr[j * T] = A::fma_rn(qq, c, pp * r);
            }
            const Real rd = rr[d * T];
            const Real hh = h * (Real)0.5;
            Real ph, pe, nh, nl;
            two_prod<Real>(pp, chi, ph, pe);
            const Real rest = pe + A::fma_rn(pp, clo, A::fma_rn(qq, rd, hh));
            two_sum<Real>(ph, rest, nh, nl);
            row[cCh(d) * T] = nh;
            row[cCl(d) * T] = nl;
            rr[d * T] = A::fma_rn(qq, chi, A::fma_rn(qq, clo, A::fma_rn(pp, rd, hh)));
            const Real sig_max = sig_u > sig_l ? sig_u : sig_l;
            const Real tot = A::add_up(A::add_up(bd.NC, bd.NR), A::add_up(A::abs(chi), A::abs(clo)));
            const Real mag = A::add_up(A::mul_up(sig_max, tot), h);
            const Real err = A::add_up(A::mul_up((Real)8 * A::ulp2, mag), (Real)(2 * d + 8) * A::tiny);
            row[cE(d) * T] = A::add_up(E, err);
            row[cN(d) * T] = A::mul_up(A::add_up(mag, A::add_up(err, err)), (Real)1 + (Real)4 * A::ulp2);
        }
    }

    // ---- C' = W C, R' = |W| R over the coefficient, N and E columns ---------------
    // The constant of C is not part of this product: the epilogue computes it
    // with error-free transformations (const_dot).
    static __device__ void contract(const Real *__restrict__ sIn, Real *__restrict__ sOut,
                                    const Real *sW, int n_in, int Mpad, int d, int NS) {
        const int QW = d * T / 4;             // quads of C coefficient columns
        const int QA = (d + 3) * T / 4;       // quads of R, N, E columns
        const int Q = QW + QA;
        const int G = Mpad / 8;
        for (int item = threadIdx.x; item < G * Q; item += NT) {
            const int g = item / Q;
            const int q = item - g * Q;
            const int p0 = g * 8;
            const bool is_abs = q >= QW;
            const int j0 = is_abs ? (d + 1) * T + (q - QW) * 4 : q * 4;
            Real acc[8][4];
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = 0;
            const Real *wp = sW + p0;
            const Real *xp = sIn + j0;
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
#pragma unroll
            for (int r = 0; r < 8; ++r) V4<Real>::st(sOut + (p0 + r) * NS + j0, acc[r]);
        }
    }

    static __device__ void stage_weights(Real *sW, const Real *Wt, int n_in, int n_out, int Mpad) {
        for (int idx = threadIdx.x; idx < n_in * Mpad; idx += NT) {
            const int i = idx / Mpad;
            const int p = idx - i * Mpad;
            sW[idx] = p < n_out ? Wt[(size_t)i * n_out + p] : (Real)0;
        }
    }

    // ---- property rows: constant, error (incl. the fold), sound bounds ----------
    static __device__ void final_rows(Real *S, const Real *Sprev, const Real *sW, int Mpad,
                                      const NetParams<Real> &net, int NS, Real *sLo, Real *sHi, Real *sErr) {
        const int d = net.d;
        const int R = net.R;
        const int K = net.K;
        const int n_in = net.n[K - 1];
        const Real *bias = net.b[K - 1];
        for (int item = threadIdx.x; item < R * T; item += NT) {
            const int r = item / T;
            const int b = item - r * T;
            Real *row = S + r * NS + b;
            Real chi, clo, E;
            if (K > 1) {
                finish_contraction(row, Sprev, sW, Mpad, r, b, d, n_in, NS, bias[r], chi, clo, E);
                // rounding of the folded property layer: |z_i| <= N_i + |C_i const| + E_i
                Real fe = net.fold_berr[r];
                const Real *pv = Sprev + b;
                for (int i = 0; i < n_in; ++i) {
                    const Real *q = pv + i * NS;
                    Real z = A::add_up(A::add_up(q[cN(d) * T], A::abs(q[cCh(d) * T])),
                                       A::add_up(A::abs(q[cCl(d) * T]), q[cE(d) * T]));
                    fe = A::add_up(fe, A::mul_up(net.fold_err[r * n_in + i], z));
                }
                E = A::add_up(E, fe);
            } else {
                chi = row[cCh(d) * T];
                clo = row[cCl(d) * T];
                E = row[cE(d) * T];
            }
            RowBounds<Real, T> bd;
            bd.compute(row, d, chi, clo);
            sLo[r * T + b] = A::add_dn(bd.ll, -E);
            sHi[r * T + b] = A::add_up(bd.uu, E);
            sErr[r * T + b] = E;
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
// The kernel: persistent over tiles of the level's boxes.
// pass 0: working precision; writes the sound class and lists the undecided
//         boxes whose class depends on E (their optimistic class differs);
// pass 1: re-check of such a list in the higher precision (writes the class,
//         counts the boxes still depending on E as ties).
// ---------------------------------------------------------------------------
template <typename Real, int T, int NT>
__global__ void __launch_bounds__(NT)
slr_eval_kernel(const NetParams<Real> net, const BoxSource src, const EvalOutputs out, const int pass) {
    using A = Arith<Real>;
    using Tile = EvalTile<Real, T, NT>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int d = net.d;
    const int R = net.R;
    const int NS = T * state_cols(d);
    const int nmp = net.n_max_pad;

    unsigned char *sp = smem_raw;
    Real *sA = reinterpret_cast<Real *>(sp);
    sp += (size_t)nmp * NS * sizeof(Real);
    Real *sB = reinterpret_cast<Real *>(sp);
    sp += (size_t)nmp * NS * sizeof(Real);
    Real *sW = reinterpret_cast<Real *>(sp);
    sp += (size_t)net.n_in_max * nmp * sizeof(Real);
    sp += (size_t)nmp * sizeof(Real);   // (bias slot, unused: biases enter the constant)
    Real *sMh = reinterpret_cast<Real *>(sp);
    sp += (size_t)T * d * sizeof(Real);
    Real *sMl = reinterpret_cast<Real *>(sp);
    sp += (size_t)T * d * sizeof(Real);
    Real *sR = reinterpret_cast<Real *>(sp);
    sp += (size_t)T * d * sizeof(Real);
    Real *sLo = reinterpret_cast<Real *>(sp);
    sp += (size_t)T * R * sizeof(Real);
    Real *sHi = reinterpret_cast<Real *>(sp);
    sp += (size_t)T * R * sizeof(Real);
    Real *sErr = reinterpret_cast<Real *>(sp);
    sp += (size_t)T * R * sizeof(Real);
    int64_t *sIdx = reinterpret_cast<int64_t *>(sp);

    int64_t n;
    if (src.index != nullptr) {
        n = (int64_t)*src.index_count;
    } else if (src.mode == 0) {
        n = (int64_t)*src.count;
    } else {
        n = src.n_explicit;
    }
    if (n > src.cap) n = src.cap;

    for (int64_t base = (int64_t)blockIdx.x * T; base < n; base += (int64_t)gridDim.x * T) {
        const int nb = (int)((n - base) < T ? (n - base) : T);
        if (threadIdx.x < T) {
            const int64_t k = base + (threadIdx.x < nb ? threadIdx.x : 0);
            sIdx[threadIdx.x] = src.index != nullptr ? src.index[k] : k;
        }
        __syncthreads();

        // ---- boxes: centre (hi + lo) and radius, outward ----------------------
        for (int item = threadIdx.x; item < T * d; item += NT) {
            const int b = item / d;
            const int i = item - b * d;
            const int64_t idx = sIdx[b];
            double m64, r64, pad;
            if (src.mode == 0) {
                // Sec. 2.2 bisection: dimension i split c times, half index k
                const unsigned long long code = src.codes[idx];
                const unsigned long long mask = src.dim_mask[i] >> (src.D - src.t);
                const unsigned long long k = pext64(code, mask);
                const int c = __popcll(mask);
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

        Tile::init_layer(sA, net, sMh, sMl, sR, NS);
        __syncthreads();

        Real *cur = sA;
        Real *nxt = sB;
        int Mpad_prev = 0;
        for (int k = 1; k < net.K; ++k) {
            Tile::hidden_epilogue(cur, nxt, sW, Mpad_prev, net, k, NS);
            __syncthreads();
            const int n_out = net.n[k + 1];
            const int Mpad = (n_out + 7) & ~7;
            Tile::stage_weights(sW, net.Wt[k], net.n[k], n_out, Mpad);
            __syncthreads();
            Tile::contract(cur, nxt, sW, net.n[k], Mpad, d, NS);
            __syncthreads();
            Real *t = cur;
            cur = nxt;
            nxt = t;
            Mpad_prev = Mpad;
        }
        Tile::final_rows(cur, nxt, sW, Mpad_prev, net, NS, sLo, sHi, sErr);
        __syncthreads();

        // ---- classify (Sec. 3) and write ------------------------------------
        if (threadIdx.x < nb) {
            const int b = threadIdx.x;
            const uint8_t cls = classify_rows<Real, T>(net, sLo, sHi, sErr, b, (Real)0);
            // optimistic bounds (raw +- E inward): the class the exact SLR could have
            const uint8_t opt = classify_rows<Real, T>(net, sLo, sHi, sErr, b, (Real)2);
            const bool near = (cls == kUndecided) && (opt != kUndecided);
            const int64_t idx = sIdx[b];
            if (out.cls != nullptr) out.cls[idx] = cls;
            if (out.row_lo != nullptr) {
                for (int r = 0; r < R; ++r) {
                    out.row_lo[idx * R + r] = to_lo<Real>(sLo[r * T + b]);
                    out.row_hi[idx * R + r] = to_hi<Real>(sHi[r * T + b]);
                }
            }
            if (out.row_err != nullptr) {
                for (int r = 0; r < R; ++r) out.row_err[idx * R + r] = to_hi<Real>(sErr[r * T + b]);
            }
            if (near) {
                if (pass == 0 && out.near_list != nullptr) {
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
}

}  // namespace slr
