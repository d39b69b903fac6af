// FP32 instantiations of the fused SLR evaluation kernel.
#include "slr_eval.cuh"
#include "slr_kernels.h"

namespace slr {

template <int T, int NT, int KI, int DC = 0>
static cudaError_t launch_t(int grid, size_t smem, cudaStream_t s, const NetParams<float> &net,
                            const BoxSource &src, const EvalOutputs &out, int pass) {
    auto k = slr_eval_kernel<float, T, NT, KI, DC>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, smem, s>>>(net, src, out, pass);
    return cudaGetLastError();
}

template <int T, int NT, int KI>
static int occ_t(size_t smem) {
    auto k = slr_eval_kernel<float, T, NT, KI>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, smem) != cudaSuccess) return 0;
    return nb;
}

// Tiles of 8 or fewer boxes whose product tiles fit one per thread run the
// one-tile-per-thread instantiation (fewer registers, more resident CTAs).
static int items_per_thread(int T, int NT, int items) { return (T <= 8 && items <= NT) ? 1 : 2; }

#define SLR_DISPATCH(NT_, CALL)                                                                \
    switch (T * 10 + KI) {                                                                     \
        case 642: return CALL<64, NT_, 2>(grid, smem, s, net, src, out, pass);                 \
        case 322: return CALL<32, NT_, 2>(grid, smem, s, net, src, out, pass);                 \
        case 202: return CALL<20, NT_, 2>(grid, smem, s, net, src, out, pass);                 \
        case 122: return CALL<12, NT_, 2>(grid, smem, s, net, src, out, pass);                 \
        case 162: return CALL<16, NT_, 2>(grid, smem, s, net, src, out, pass);                 \
        case 82: return CALL<8, NT_, 2>(grid, smem, s, net, src, out, pass);                   \
        case 81: return CALL<8, NT_, 1>(grid, smem, s, net, src, out, pass);                   \
        case 42: return CALL<4, NT_, 2>(grid, smem, s, net, src, out, pass);                   \
        case 41: return CALL<4, NT_, 1>(grid, smem, s, net, src, out, pass);                   \
        default: break;                                                                        \
    }

// Networks with five inputs (the collision-avoidance shape) on the two-tile,
// 256-thread tiles: the input count as a compile-time constant.
static cudaError_t launch_d5(int T, int grid, size_t smem, cudaStream_t s, const NetParams<float> &net,
                             const BoxSource &src, const EvalOutputs &out, int pass) {
    switch (T) {
        case 32: return launch_t<32, 256, 2, 5>(grid, smem, s, net, src, out, pass);
        case 20: return launch_t<20, 256, 2, 5>(grid, smem, s, net, src, out, pass);
        case 16: return launch_t<16, 256, 2, 5>(grid, smem, s, net, src, out, pass);
        case 12: return launch_t<12, 256, 2, 5>(grid, smem, s, net, src, out, pass);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_eval_f32(int T, int NT, int grid, size_t smem, cudaStream_t s, const NetParams<float> &net,
                            const BoxSource &src, const EvalOutputs &out, int pass) {
    const int KI = items_per_thread(T, NT, eval_gemm_items(T, net.d, net.n_max_pad));
    if (net.d == 5 && NT == 256 && KI == 2 && (T == 32 || T == 20 || T == 16 || T == 12))
        return launch_d5(T, grid, smem, s, net, src, out, pass);
    if (NT == 256) {
        SLR_DISPATCH(256, launch_t)
    } else if (NT == 128) {
        SLR_DISPATCH(128, launch_t)
    }
    return cudaErrorInvalidValue;
}

int eval_blocks_per_sm_f32(int T, int NT, size_t smem, int items) {
    const int KI = items_per_thread(T, NT, items);
    switch (NT * 1000 + T * 10 + KI) {
        case 256642: return occ_t<64, 256, 2>(smem);
        case 256322: return occ_t<32, 256, 2>(smem);
        case 256202: return occ_t<20, 256, 2>(smem);
        case 256162: return occ_t<16, 256, 2>(smem);
        case 256122: return occ_t<12, 256, 2>(smem);
        case 256082: return occ_t<8, 256, 2>(smem);
        case 256081: return occ_t<8, 256, 1>(smem);
        case 256042: return occ_t<4, 256, 2>(smem);
        case 256041: return occ_t<4, 256, 1>(smem);
        case 128642: return occ_t<64, 128, 2>(smem);
        case 128322: return occ_t<32, 128, 2>(smem);
        case 128202: return occ_t<20, 128, 2>(smem);
        case 128162: return occ_t<16, 128, 2>(smem);
        case 128122: return occ_t<12, 128, 2>(smem);
        case 128082: return occ_t<8, 128, 2>(smem);
        case 128081: return occ_t<8, 128, 1>(smem);
        case 128042: return occ_t<4, 128, 2>(smem);
        case 128041: return occ_t<4, 128, 1>(smem);
        default: return 0;
    }
}

template <int T>
static cudaError_t launch_batch_t(int grid, size_t smem, cudaStream_t s, const NetParams<float> *nets,
                                  const BoxSource *srcs, const EvalOutputs *outs, int P, const long long *prefix,
                                  const BatchShape &shape, int pass) {
    auto k = slr_eval_batch_kernel<float, T, 256>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, 256, smem, s>>>(nets, srcs, outs, P, prefix, shape, pass);
    return cudaGetLastError();
}

template <int T>
static int occ_batch_t(size_t smem) {
    auto k = slr_eval_batch_kernel<float, T, 256>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 256, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_eval_batch_f32(int T, int grid, size_t smem, cudaStream_t s, const NetParams<float> *nets,
                                  const BoxSource *srcs, const EvalOutputs *outs, int P, const long long *prefix,
                                  const BatchShape &shape, int pass) {
    switch (T) {
        case 64: return launch_batch_t<64>(grid, smem, s, nets, srcs, outs, P, prefix, shape, pass);
        case 32: return launch_batch_t<32>(grid, smem, s, nets, srcs, outs, P, prefix, shape, pass);
        case 16: return launch_batch_t<16>(grid, smem, s, nets, srcs, outs, P, prefix, shape, pass);
        case 8: return launch_batch_t<8>(grid, smem, s, nets, srcs, outs, P, prefix, shape, pass);
        case 4: return launch_batch_t<4>(grid, smem, s, nets, srcs, outs, P, prefix, shape, pass);
        default: return cudaErrorInvalidValue;
    }
}

int eval_batch_blocks_per_sm_f32(int T, size_t smem) {
    switch (T) {
        case 64: return occ_batch_t<64>(smem);
        case 32: return occ_batch_t<32>(smem);
        case 16: return occ_batch_t<16>(smem);
        case 8: return occ_batch_t<8>(smem);
        case 4: return occ_batch_t<4>(smem);
        default: return 0;
    }
}

}  // namespace slr
