// FP32 instantiations of the fused SLR evaluation kernel.
#include "slr_eval.cuh"
#include "slr_kernels.h"

namespace slr {

template <int T, int NT>
static cudaError_t launch_t(int grid, size_t smem, cudaStream_t s, const NetParams<float> &net,
                            const BoxSource &src, const EvalOutputs &out, int pass) {
    auto k = slr_eval_kernel<float, T, NT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, smem, s>>>(net, src, out, pass);
    return cudaGetLastError();
}

template <int T, int NT>
static int occ_t(size_t smem) {
    auto k = slr_eval_kernel<float, T, NT>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, smem) != cudaSuccess) return 0;
    return nb;
}

#define SLR_DISPATCH(NT_, CALL)          \
    switch (T) {                          \
        case 64: return CALL<64, NT_>(grid, smem, s, net, src, out, pass);    \
        case 32: return CALL<32, NT_>(grid, smem, s, net, src, out, pass);    \
        case 16: return CALL<16, NT_>(grid, smem, s, net, src, out, pass);    \
        case 8: return CALL<8, NT_>(grid, smem, s, net, src, out, pass);      \
        case 4: return CALL<4, NT_>(grid, smem, s, net, src, out, pass);      \
        default: break;                   \
    }

cudaError_t launch_eval_f32(int T, int NT, int grid, size_t smem, cudaStream_t s, const NetParams<float> &net,
                            const BoxSource &src, const EvalOutputs &out, int pass) {
    if (NT == 256) {
        SLR_DISPATCH(256, launch_t)
    } else if (NT == 128) {
        SLR_DISPATCH(128, launch_t)
    }
    return cudaErrorInvalidValue;
}

int eval_blocks_per_sm_f32(int T, int NT, size_t smem) {
    switch (NT * 100 + T) {
        case 25664: return occ_t<64, 256>(smem);
        case 25632: return occ_t<32, 256>(smem);
        case 25616: return occ_t<16, 256>(smem);
        case 25608: return occ_t<8, 256>(smem);
        case 25604: return occ_t<4, 256>(smem);
        case 12864: return occ_t<64, 128>(smem);
        case 12832: return occ_t<32, 128>(smem);
        case 12816: return occ_t<16, 128>(smem);
        case 12808: return occ_t<8, 128>(smem);
        case 12804: return occ_t<4, 128>(smem);
        default: return 0;
    }
}

}  // namespace slr
