// FP32 instantiation of the fused SLR evaluation kernel.
#include "slr_eval.cuh"
#include "slr_kernels.h"

namespace slr {

template <int T>
static cudaError_t launch_t(int grid, size_t smem, cudaStream_t s, const NetParams<float> &net,
                            const BoxSource &src, const EvalOutputs &out, int pass) {
    auto k = slr_eval_kernel<float, T, kEvalThreads>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kEvalThreads, smem, s>>>(net, src, out, pass);
    return cudaGetLastError();
}

template <int T>
static int occ_t(size_t smem) {
    auto k = slr_eval_kernel<float, T, kEvalThreads>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kEvalThreads, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_eval_f32(int T, int grid, size_t smem, cudaStream_t s, const NetParams<float> &net,
                            const BoxSource &src, const EvalOutputs &out, int pass) {
    switch (T) {
        case 64: return launch_t<64>(grid, smem, s, net, src, out, pass);
        case 32: return launch_t<32>(grid, smem, s, net, src, out, pass);
        case 16: return launch_t<16>(grid, smem, s, net, src, out, pass);
        case 8: return launch_t<8>(grid, smem, s, net, src, out, pass);
        case 4: return launch_t<4>(grid, smem, s, net, src, out, pass);
        default: return cudaErrorInvalidValue;
    }
}

int eval_blocks_per_sm_f32(int T, size_t smem) {
    switch (T) {
        case 64: return occ_t<64>(smem);
        case 32: return occ_t<32>(smem);
        case 16: return occ_t<16>(smem);
        case 8: return occ_t<8>(smem);
        case 4: return occ_t<4>(smem);
        default: return 0;
    }
}

}  // namespace slr
