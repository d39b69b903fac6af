// Host-side launch wrappers of the SLR kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "slr_device.cuh"

namespace slr {

// Tile sizes (boxes per CTA) the evaluation kernel is built for.
constexpr int kTileSizes[] = {64, 32, 16, 8, 4};
constexpr int kThreadCounts[] = {256, 128};

// Fused evaluation (kernel (b) plus its contraction); one instantiation per
// working precision.  `T` must be one of kTileSizes and `NT` of kThreadCounts.
cudaError_t launch_eval_f32(int T, int NT, int grid, size_t smem, cudaStream_t s, const NetParams<float> &net,
                            const BoxSource &src, const EvalOutputs &out, int pass);
cudaError_t launch_eval_f64(int T, int NT, int grid, size_t smem, cudaStream_t s, const NetParams<double> &net,
                            const BoxSource &src, const EvalOutputs &out, int pass);
// Resident CTAs per SM of the evaluation kernel at tile size T, NT threads and this smem.
int eval_blocks_per_sm_f32(int T, int NT, size_t smem);
int eval_blocks_per_sm_f64(int T, int NT, size_t smem);

// Tensor-core evaluation (FP32 state, split-TF32 contraction on tcgen05).
size_t eval_tc_smem_bytes(int T, const NetParams<float> &net, const TcParams &tc);
cudaError_t launch_eval_tc(int T, int grid, size_t smem, cudaStream_t s, const NetParams<float> &net,
                           const TcParams &tc, const BoxSource &src, const EvalOutputs &out, int pass);

// Batched count (many problems, one persistent launch per step).
struct CompactArgs {
    const uint64_t *codes_in;
    const uint8_t *cls;
    uint64_t *codes_out;
    LevelCounters *ctr;
    int64_t cap;
    int D;
};
cudaError_t launch_eval_batch_f32(int T, int grid, size_t smem, cudaStream_t s, const NetParams<float> *nets,
                                  const BoxSource *srcs, const EvalOutputs *outs, int P, const long long *prefix,
                                  const BatchShape &shape, int pass);
cudaError_t launch_eval_batch_f64(int T, int grid, size_t smem, cudaStream_t s, const NetParams<double> *nets,
                                  const BoxSource *srcs, const EvalOutputs *outs, int P, const long long *prefix,
                                  const BatchShape &shape, int pass);
int eval_batch_blocks_per_sm_f32(int T, size_t smem);
int eval_batch_blocks_per_sm_f64(int T, size_t smem);
cudaError_t launch_tile_prefix(const BoxSource *srcs, int P, int T, long long *prefix, cudaStream_t s);
cudaError_t launch_compact_batch(const CompactArgs *args, int P, int t, unsigned int *status, int blocks_per_problem,
                                 cudaStream_t s);
cudaError_t launch_init_batch(const CompactArgs *args, int P, cudaStream_t s);

cudaError_t launch_init_count(uint64_t *codes0, LevelCounters *ctr, cudaStream_t s);
cudaError_t launch_compact(const uint64_t *codes_in, const uint8_t *cls, uint64_t *codes_out,
                           LevelCounters *ctr, unsigned int *status, int64_t cap, int t, int D,
                           uint64_t *leaf_codes, uint8_t *leaf_depth, uint8_t *leaf_cls,
                           int64_t leaf_cap, int grid, cudaStream_t s);

}  // namespace slr
