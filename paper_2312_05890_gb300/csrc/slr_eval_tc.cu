// Fused SLR evaluation with the symbolic contraction on the 5th-generation
// tensor cores (tcgen05, kind::tf32, three-term split precision).
//
// Same tile algorithm as slr_eval.cuh (decode, layer 1, per layer: error,
// bounds, ReLU relaxation, contraction; property rows; classification), but
// the state of a tile of T boxes lives directly in the layout of the MMA's B
// operand, and the per-layer product
//     D[m][n] = sum_k A[m][k] B[n][k],   A = [W ; |W|] (128 x K),
//     B[n][k] = state column n (box b, GEMM column c, n = b NCg + c) of neuron k
// runs on the tensor core with the accumulator in tensor memory.  Rows 0..63
// of D give W C on the C-coefficient columns, rows 64..127 give |W| R on the
// R, N and E columns.  Operands are split x = hi + lo into TF32 pieces and the
// product is hi*lo + lo*hi + hi*hi (lower-order passes first), accumulated in
// FP32: about 22 correct bits per product, covered in E by the bound
// gamma_tc = (K + 8) 2^-23 + 3 2^-22 of sum |A||B| per output.
//
// The weights of each layer ([A hi | A lo | W^T float]) are pre-formatted on
// the host in the exact shared-memory image and brought in by one TMA bulk
// copy per layer that overlaps the previous epilogue.  The constants of C
// (float-float, error-free) are computed on the CUDA cores while the MMA runs.
//
// Shared-memory operand layout (K-major, no swizzle): element (row r, k) at
//     (r / 8) SBO + (k / 4) 144 + (r % 8) 16 + (k % 4) 4,
// i.e. 8-row x 16-byte core matrices, 144 bytes apart along K (one 16-byte
// pad per core matrix so that 32 consecutive k of one row hit distinct banks),
// SBO = (K / 4) 144 between 8-row groups.
#include "slr_eval.cuh"
#include "slr_kernels.h"
#include "slr_tc_util.cuh"

namespace slr {

using namespace tc;

namespace {

constexpr int kTcThreads = 256;

__device__ __forceinline__ int boff(int n, int k, int sbo) {
    return (n >> 3) * sbo + (k >> 2) * kTcLbo + (n & 7) * 16 + (k & 3) * 4;
}

}  // namespace

// State of a tile in the B-operand images: GEMM columns of row (neuron) p and
// box b in the hi image (raw FP32 between the contraction and the epilogue,
// TF32 hi piece after finish_row), the constants of C in `cst`.
template <int T>
struct TcLayout {
    unsigned char *bhi;
    unsigned char *blo;
    float *cst;
    int d, NCg, sbo, nmpT;
    struct Row {
        unsigned char *bhi;
        float *cst;
        int p, b, d, NCg, sbo, nmpT;
        __device__ __forceinline__ float &operator()(int c) const {
            if (c == d) return cst[p * T + b];
            if (c == 2 * d + 4) return cst[nmpT + p * T + b];
            const int n = b * NCg + c - (c > d ? 1 : 0);
            return *reinterpret_cast<float *>(bhi + boff(n, p, sbo));
        }
    };
    __device__ __forceinline__ Row row(int p, int b) const { return Row{bhi, cst, p, b, d, NCg, sbo, nmpT}; }
    // |value| bound of a column once the row is split into TF32 pieces
    __device__ __forceinline__ float mag(int p, int b, int c) const {
        if (c == d || c == 2 * d + 4) return fabsf(row(p, b)(c));
        const int n = b * NCg + c - (c > d ? 1 : 0);
        const int o = boff(n, p, sbo);
        const float h = *reinterpret_cast<const float *>(bhi + o);
        const float l = *reinterpret_cast<const float *>(blo + o);
        return __fmul_ru(__fadd_ru(fabsf(h), fabsf(l)), 1.0f + 0x1p-20f);
    }
    // split every GEMM column of the row into TF32 hi + lo for the next product
    __device__ __forceinline__ void finish_row(int p, int b) const {
        for (int c = 0; c < NCg; ++c) {
            const int o = boff(b * NCg + c, p, sbo);
            const float v = *reinterpret_cast<const float *>(bhi + o);
            const float h = tf32_rna(v);
            *reinterpret_cast<float *>(bhi + o) = h;
            *reinterpret_cast<float *>(blo + o) = tf32_rna(v - h);
        }
    }
};

template <int T>
__global__ void __launch_bounds__(kTcThreads, 1)
slr_eval_tc_kernel(const NetParams<float> net, const TcParams tc, const BoxSource src, const EvalOutputs out,
                   const int pass) {
    using A = Arith<float>;
    using Tile = EvalTile<float, T, kTcThreads>;
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    const int d = net.d;
    const int R = net.R;
    const int nmp = net.n_max_pad;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;

    unsigned char *sp = smem_tc;
    unsigned char *sBhi = sp;
    sp += tc.b_bytes;
    unsigned char *sBlo = sp;
    sp += tc.b_bytes;
    unsigned char *sAhi = sp;          // [A hi | A lo | W^T float] of the current layer, one bulk copy
    unsigned char *sAlo = sp + tc.a_bytes;
    float *sW = reinterpret_cast<float *>(sp + 2 * tc.a_bytes);
    sp += tc.img_max;
    float *sConst = reinterpret_cast<float *>(sp);
    sp += 3 * (size_t)nmp * T * sizeof(float);
    float *sCst = reinterpret_cast<float *>(sp);
    sp += 2 * (size_t)nmp * T * sizeof(float);
    float *sMh = reinterpret_cast<float *>(sp);
    sp += (size_t)T * d * sizeof(float);
    float *sMl = reinterpret_cast<float *>(sp);
    sp += (size_t)T * d * sizeof(float);
    float *sR = reinterpret_cast<float *>(sp);
    sp += (size_t)T * d * sizeof(float);
    float *sLo = reinterpret_cast<float *>(sp);
    sp += (size_t)T * R * sizeof(float);
    float *sHi = reinterpret_cast<float *>(sp);
    sp += (size_t)T * R * sizeof(float);
    float *sErr = reinterpret_cast<float *>(sp);
    sp += (size_t)T * R * sizeof(float);
    sp = reinterpret_cast<unsigned char *>(((uintptr_t)sp + 15) & ~(uintptr_t)15);
    int64_t *sIdx = reinterpret_cast<int64_t *>(sp);
    sp += (size_t)T * sizeof(int64_t);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sp);   // [0] MMA done, [1] weights landed
    sp += 2 * sizeof(uint64_t);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sp);
    int *sAbort = reinterpret_cast<int *>(sp + 4);

    // operand padding (rows and columns beyond the network) must hold finite values
    for (int i = tid; i < 2 * tc.b_bytes / 16; i += kTcThreads) reinterpret_cast<int4 *>(sBhi)[i] = make_int4(0, 0, 0, 0);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
        *sAbort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTcTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    uint32_t ph_mma = 0, ph_w = 0;
    const int wait_limit = 1 << 24;

    int64_t n;
    if (src.index != nullptr) {
        n = (int64_t)*src.index_count;
    } else if (src.mode == 0) {
        n = (int64_t)*src.count;
    } else {
        n = src.n_explicit;
    }
    if (n > src.cap) n = src.cap;

    const TcLayout<T> lay{sBhi, sBlo, sCst, d, tc.NCg, tc.sbo, nmp * T};
    for (int64_t base = (int64_t)blockIdx.x * T; base < n; base += (int64_t)gridDim.x * T) {
        if (*sAbort) break;
        const int nb = (int)((n - base) < T ? (n - base) : T);
        if (tid < T) {
            const int64_t k = base + (tid < nb ? tid : 0);
            sIdx[tid] = src.index != nullptr ? src.index[k] : k;
        }
        __syncthreads();
        for (int item = tid; item < T * d; item += kTcThreads) {
            const int b = item / d;
            const int i = item - b * d;
            const int64_t idx = sIdx[b];
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
            float mh, ml, r;
            split_centre<float>(m64, r64, pad, mh, ml, r);
            sMh[b * d + i] = mh;
            sMl[b * d + i] = ml;
            sR[b * d + i] = r;
        }
        __syncthreads();
        Tile::init_layer(lay, net, sMh, sMl, sR);
        __syncthreads();

        bool ok = true;
        for (int k = 1; k < net.K; ++k) {
            const int n_in = net.n[k];
            const int n_out = net.n[k + 1];
            const int Mpad = (n_out + 7) & ~7;
            const int kp = tc.k_pad[k];
            // weights of layer k: one bulk copy, overlapping the epilogue below
            if (tid == 0) {
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&mbar[1])),
                             "r"(tc.img_bytes[k])
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(sAhi)),
                    "l"(tc.img[k]), "r"(tc.img_bytes[k]), "r"(smem_u32(&mbar[1]))
                    : "memory");
            }
            Tile::hidden_epilogue(lay, sConst, net, k, tc_gamma(tc.k_pad[k - 1]));
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (!mbar_wait(smem_u32(&mbar[1]), ph_w, wait_limit)) ok = false;
            ph_w ^= 1u;
            __syncthreads();
            if (tid == 0 && ok) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t a_hi = smem_u32(sAhi), a_lo = smem_u32(sAlo);
                const uint32_t b_hi = smem_u32(sBhi), b_lo = smem_u32(sBlo);
                const uint32_t pa[3] = {a_hi, a_lo, a_hi};
                const uint32_t pb[3] = {b_lo, b_hi, b_hi};
                int first = 1;
                for (int ps = 0; ps < 3; ++ps) {
                    for (int s = 0; s < kp / 8; ++s) {
                        const uint64_t da = umma_desc(pa[ps] + s * 2 * kTcLbo, kTcLbo, tc.sbo);
                        const uint64_t db = umma_desc(pb[ps] + s * 2 * kTcLbo, kTcLbo, tc.sbo);
                        const uint32_t acc = first ? 0u : 1u;
                        first = 0;
                        asm volatile(
                            "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
                            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(tmem),
                            "l"(da), "l"(db), "r"(tc.idesc), "r"(acc));
                    }
                }
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&mbar[0]))
                    : "memory");
            }
            // constants of layer k+1 on the CUDA cores while the tensor core runs
            Tile::const_phase(lay, sConst, sW, Mpad, net, k);
            if (ok && !mbar_wait(smem_u32(&mbar[0]), ph_mma, wait_limit)) ok = false;
            ph_mma ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (!ok) atomicExch(sAbort, 1);
            __syncthreads();
            if (*sAbort) break;
            // tensor memory -> raw FP32 state: rows 0..63 hold W C, rows 64..127 |W| (R, N, E)
            {
                const int quad = warp & 3;
                const int half = warp >> 2;
                const int m = quad * 32 + lane;
                const bool cpart = m < 64;
                const int p = cpart ? m : m - 64;
                const int ncols = tc.Npad / 2;
                const int c0 = half * ncols;
                for (int cc = 0; cc < ncols; cc += 8) {
                    uint32_t r[8];
                    const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(c0 + cc);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                          "=r"(r[7])
                        : "r"(taddr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (p < n_out) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int col = c0 + cc + j;
                            const int b = col / tc.NCg;
                            const int gc = col - b * tc.NCg;
                            if (b < T && (cpart ? gc < d : gc >= d))
                                *reinterpret_cast<float *>(sBhi + boff(col, p, tc.sbo)) = __uint_as_float(r[j]);
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            (void)n_in;
        }
        if (*sAbort) break;
        Tile::final_rows(lay, sConst, net, tc_gamma(tc.k_pad[net.K - 1]), sLo, sHi, sErr);
        __syncthreads();

        if (tid < nb) {
            const int b = tid;
            const uint8_t cls = classify_rows<float, T>(net, sLo, sHi, sErr, b, 0.0f);
            const uint8_t opt = classify_rows<float, T>(net, sLo, sHi, sErr, b, 2.0f);
            const bool near = (cls == kUndecided) && (opt != kUndecided);
            const int64_t idx = sIdx[b];
            if (out.cls != nullptr) out.cls[idx] = cls;
            if (out.row_lo != nullptr) {
                for (int r = 0; r < R; ++r) {
                    out.row_lo[idx * R + r] = sLo[r * T + b];
                    out.row_hi[idx * R + r] = sHi[r * T + b];
                }
            }
            if (out.row_err != nullptr)
                for (int r = 0; r < R; ++r) out.row_err[idx * R + r] = sErr[r * T + b];
            if (near && out.near_list != nullptr) {
                const unsigned long long pos = atomicAdd(out.near_count, 1ull);
                if ((int64_t)pos < out.near_cap) out.near_list[pos] = idx;
                else atomicOr(out.status, kStatusNearOverflow);
            } else if (near && out.tie_count != nullptr) {
                atomicAdd(out.tie_count, 1ull);
            }
        }
        __syncthreads();
    }
    if (*sAbort && tid == 0) atomicOr(out.status, kStatusTimeout);
    // a timed-out MMA may still be running: give it a bounded chance to finish
    if (*sAbort) mbar_wait(smem_u32(&mbar[0]), ph_mma, wait_limit);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols));
}

size_t eval_tc_smem_bytes(int T, const NetParams<float> &net, const TcParams &tc) {
    size_t s = 2 * (size_t)tc.b_bytes + (size_t)tc.img_max;
    s += 5 * (size_t)net.n_max_pad * T * sizeof(float);
    s += 3 * (size_t)T * net.d * sizeof(float) + 3 * (size_t)T * net.R * sizeof(float);
    s = (s + 15) & ~(size_t)15;
    s += (size_t)T * sizeof(int64_t) + 2 * sizeof(uint64_t) + 16;
    return (s + 127) & ~(size_t)127;
}

template <int T>
static cudaError_t launch_tc_t(int grid, size_t smem, cudaStream_t s, const NetParams<float> &net, const TcParams &tc,
                               const BoxSource &src, const EvalOutputs &out, int pass) {
    auto k = slr_eval_tc_kernel<T>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kTcThreads, smem, s>>>(net, tc, src, out, pass);
    return cudaGetLastError();
}

cudaError_t launch_eval_tc(int T, int grid, size_t smem, cudaStream_t s, const NetParams<float> &net,
                           const TcParams &tc, const BoxSource &src, const EvalOutputs &out, int pass) {
    switch (T) {
        case 64: return launch_tc_t<64>(grid, smem, s, net, tc, src, out, pass);
        case 32: return launch_tc_t<32>(grid, smem, s, net, tc, src, out, pass);
        case 16: return launch_tc_t<16>(grid, smem, s, net, tc, src, out, pass);
        case 8: return launch_tc_t<8>(grid, smem, s, net, tc, src, out, pass);
        case 4: return launch_tc_t<4>(grid, smem, s, net, tc, src, out, pass);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace slr
