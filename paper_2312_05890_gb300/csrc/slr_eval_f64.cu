// FP64 instantiations of the fused SLR evaluation kernel (re-check of near-decided boxes).
#include "slr_eval.cuh"
#include "slr_kernels.h"

namespace slr {

template <int T, int NT>
static cudaError_t launch_t(int grid, size_t smem, cudaStream_t s, const NetParams<double> &net,
                            const BoxSource &src, const EvalOutputs &out, int pass) {
    auto k = slr_eval_kernel<double, T, NT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, smem, s>>>(net, src, out, pass);
    return cudaGetLastError();
}

template <int T, int NT>
static int occ_t(size_t smem) {
    auto k = slr_eval_kernel<double, T, NT>;
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

// Two-box tiles for the short re-check lists (odd input counts only: the
// products take the columns four at a time, (d + 1) T and (d + 3) T must be
// multiples of 4, and a row of the state must start on 16 bytes).
static bool f64_pair_tile_ok(int d) { return d % 2 == 1; }

cudaError_t launch_eval_f64(int T, int NT, int grid, size_t smem, cudaStream_t s, const NetParams<double> &net,
                            const BoxSource &src, const EvalOutputs &out, int pass) {
    if (NT == 256) {
        SLR_DISPATCH(256, launch_t)
        if (T == 2 && f64_pair_tile_ok(net.d)) return launch_t<2, 256>(grid, smem, s, net, src, out, pass);
    } else if (NT == 128) {
        SLR_DISPATCH(128, launch_t)
    }
    return cudaErrorInvalidValue;
}

int eval_blocks_per_sm_f64(int T, int NT, size_t smem) {
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
        case 25602: return occ_t<2, 256>(smem);
        default: return 0;
    }
}

int eval_f64_pair_tile_ok(int d) { return f64_pair_tile_ok(d) ? 1 : 0; }

// The re-check with each tile on a cluster of kRecheckCluster CTAs of 256 threads.
template <int T>
static cudaError_t launch_cluster_t(int grid, size_t smem, cudaStream_t s, const NetParams<double> &net,
                                    const BoxSource &src, const EvalOutputs &out, int pass) {
    auto k = slr_eval_cluster_kernel<double, T, 256>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, 256, smem, s>>>(net, src, out, pass);
    return cudaGetLastError();
}

template <int T>
static int cluster_max_t(size_t smem) {
    auto k = slr_eval_cluster_kernel<double, T, 256>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kRecheckCluster * 256, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return nc;
}

cudaError_t launch_eval_f64_cluster(int T, int grid, size_t smem, cudaStream_t s, const NetParams<double> &net,
                                    const BoxSource &src, const EvalOutputs &out, int pass) {
    if (grid <= 0 || grid % kRecheckCluster != 0) return cudaErrorInvalidValue;
    if (T == 4) return launch_cluster_t<4>(grid, smem, s, net, src, out, pass);
    if (T == 2 && f64_pair_tile_ok(net.d)) return launch_cluster_t<2>(grid, smem, s, net, src, out, pass);
    return cudaErrorInvalidValue;
}

int eval_f64_cluster_max(int T, size_t smem) {
    if (T == 4) return cluster_max_t<4>(smem);
    if (T == 2) return cluster_max_t<2>(smem);
    return 0;
}


template <int T>
static cudaError_t launch_batch_t(int grid, size_t smem, cudaStream_t s, const NetParams<double> *nets,
                                  const BoxSource *srcs, const EvalOutputs *outs, int P, const long long *prefix,
                                  const BatchShape &shape, int pass) {
    auto k = slr_eval_batch_kernel<double, T, 256>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, 256, smem, s>>>(nets, srcs, outs, P, prefix, shape, pass);
    return cudaGetLastError();
}

template <int T>
static int occ_batch_t(size_t smem) {
    auto k = slr_eval_batch_kernel<double, T, 256>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 256, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_eval_batch_f64(int T, int grid, size_t smem, cudaStream_t s, const NetParams<double> *nets,
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

int eval_batch_blocks_per_sm_f64(int T, size_t smem) {
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
