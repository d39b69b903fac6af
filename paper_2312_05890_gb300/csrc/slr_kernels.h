// Host-side launch wrappers of the SLR kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "slr_device.cuh"

namespace slr {

// Tile sizes (boxes per CTA) the evaluation kernel is built for.
constexpr int kTileSizes[] = {64, 32, 20, 16, 12, 8, 4};
// Tile sizes of the tensor-core tile kernel.
constexpr int kTcTileSizes[] = {64, 32, 16, 8, 4};
constexpr int kThreadCounts[] = {256, 128};

// Fused evaluation (kernel (b) plus its contraction); one instantiation per
// working precision.  `T` must be one of kTileSizes and `NT` of kThreadCounts
// (tiles of 20 and 12 boxes exist in FP32 only).
cudaError_t launch_eval_f32(int T, int NT, int grid, size_t smem, cudaStream_t s, const NetParams<float> &net,
                            const BoxSource &src, const EvalOutputs &out, int pass);
cudaError_t launch_eval_f64(int T, int NT, int grid, size_t smem, cudaStream_t s, const NetParams<double> &net,
                            const BoxSource &src, const EvalOutputs &out, int pass);
// Resident CTAs per SM of the evaluation kernel at tile size T, NT threads and
// this smem; `items` = eval_gemm_items of the network (selects the
// one-product-tile-per-thread instantiation where it fits).
int eval_blocks_per_sm_f32(int T, int NT, size_t smem, int items);
int eval_blocks_per_sm_f64(int T, int NT, size_t smem);
// 1 when the FP64 kernel can take tiles of two boxes for d inputs.
int eval_f64_pair_tile_ok(int d);
// FP64 re-check with each tile on a cluster of kRecheckCluster CTAs (256
// threads each, T = 2 for odd d or T = 4); grid a multiple of kRecheckCluster.
cudaError_t launch_eval_f64_cluster(int T, int grid, size_t smem, cudaStream_t s, const NetParams<double> &net,
                                    const BoxSource &src, const EvalOutputs &out, int pass);
// Clusters of that kernel the GPU holds at once (0: cannot run it).
int eval_f64_cluster_max(int T, size_t smem);

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

// Adjoint of the SLR pass (gradients of a linear loss of the row bounds) and
// projected Adam on the lower ReLU slopes; one box per CTA.
enum { kAlphaDefault = 0, kAlphaFree = 1, kAlphaInit = 2 };
struct AdjArgs {
    NetParams<float> net;
    BoxSource src;                  // boxes at positions 0..n-1
    int64_t n;                      // positions (an upper bound when `count` is set)
    const unsigned long long *count;  // optional device count of positions
    int64_t H;                      // hidden neurons (row length of the slope arrays)
    int n_max;                      // widest layer n[1..K]
    int nck;                        // hidden layers whose equations stay in shared memory
    int boxes_per_cta;              // boxes a CTA works on together
    float *gscratch;                // optional: per-CTA box state in global memory (networks whose
                                    // state exceeds shared memory); CTA c uses boxes_per_cta slots
                                    // from gscratch + c * boxes_per_cta * (floats per box)
    int alpha_mode;                 // kAlphaDefault: u/(u-l), differentiated through; kAlphaFree: read;
                                    // kAlphaInit: write u/(u-l) to alpha, then treat it as free
    float *alpha;                   // n x H
    const float *g_lo, *g_hi;       // n x R upstream adjoints; null: in-kernel decision loss
    int8_t *dir;                    // decision loss direction per position (1 safe, 2 unsafe)
    float *row_lo, *row_hi;         // optional: the float32 row bounds (not widened)
    float *d_alpha;                 // optional n x H
    float *d_lo, *d_hi;             // optional n x d
    float *dW[kMaxLayers];          // optional, accumulated: network layout n[k+1] x n[k], last unfolded
    float *db[kMaxLayers];
    const float *Cprop;             // property rows (R x n_out) for unfolding the last layer
    int n_out;
    int adam_t;                     // > 0: take Adam step t on the slopes
    float *adam_m, *adam_v;         // n x H
    float lr, beta1, beta2, eps, beta1_t, beta2_t;
    float *d_r;                     // optional n x d: gradient with respect to the box radius
    // gradient split rule: for each position whose box split_cls (indexed like
    // the source) still holds UNDECIDED, store in the box's code in split_codes
    // the position in split_dims of the dimension i with the largest
    // |dM/dr_i| r_i (the first on ties); split_codes null: no choice
    uint64_t *split_codes;
    const uint8_t *split_cls;
    const int *split_dims;
    int n_split;
};
size_t adjoint_smem_bytes(const AdjArgs &a);
size_t adjoint_box_bytes(const AdjArgs &a);
int adjoint_blocks_per_sm(size_t smem);
cudaError_t launch_adjoint(const AdjArgs &a, int grid, cudaStream_t s);
// The adjoint on the wide path (per-layer tensor-core products; slr_wide_adj.cu).
cudaError_t launch_wadj_box(const BoxSource &src, int64_t pos0, int nb, int d, float *m, float *r, int sms,
                            cudaStream_t s);
cudaError_t launch_wadj_layer1(const NetParams<float> &net, const float *W0t, int nb, int NP, const float *m,
                               const float *r, float *C, cudaStream_t s);
cudaError_t launch_wadj_fwd(const AdjArgs &a, int layer, int64_t pos0, int nb, int NP, float *C, const float *R,
                            const float *bias, float *sc, int64_t sstride, float *Pc, float *Pr, cudaStream_t s);
cudaError_t launch_wadj_rows(const AdjArgs &a, int64_t pos0, int nb, int NP, const float *C, const float *R,
                             const float *bias, float *gC, float *gR, cudaStream_t s);
cudaError_t launch_wadj_bwd(const AdjArgs &a, int layer, int64_t pos0, int nb, int NP, const float *C, const float *R,
                            const float *sc, int64_t sstride, const float *gPc, const float *gPr, float *gC, float *gR,
                            cudaStream_t s);
cudaError_t launch_wadj_boxgrad(const AdjArgs &a, int64_t pos0, int nb, int NP, const float *W0t, const float *gC1,
                                float *gr, int sms, cudaStream_t s);
cudaError_t launch_wadj_split(const AdjArgs &a, int64_t pos0, int nb, const float *gr, const float *r, int sms,
                              cudaStream_t s);
cudaError_t launch_merge_bounds(const NetParams<float> &net, int64_t n, const unsigned long long *count,
                                const float *lo_new, const float *hi_new, float *lo_best, float *hi_best,
                                uint8_t *cls_pos, uint8_t *cls_idx, const int64_t *index, int first,
                                unsigned long long *decided, cudaStream_t s);
cudaError_t launch_margin_filter(const NetParams<float> &net, const float *lo, const float *hi,
                                 const unsigned long long *n_in, int64_t cap, const int64_t *list_in,
                                 int64_t *list_out, unsigned long long *n_out, float tau, int grid, cudaStream_t s);
cudaError_t launch_gather_undecided(const uint8_t *cls, const unsigned long long *n, int64_t cap, int64_t *list,
                                    unsigned long long *list_n, int64_t list_cap, int grid, cudaStream_t s);

// Wide networks: per-box state in HBM, one tensor-core product per layer.
struct WideGemm {
    const float *Ahi, *Alo;   // TF32 pieces of W (or |W|), Mpad x Kpad row-major, zero padded
    const float *B;           // column col, element k at B[col * ldb + k] (k < K)
    float *D;                 // D[col * ldd + m] for m < M
    int M, K, Kpad, ncols, ldb, ldd;
};
struct WideGemmArgs {
    WideGemm g[2];
    unsigned int *status;
};
size_t wide_gemm_smem_bytes();
cudaError_t launch_wide_gemm(const WideGemmArgs &args, int nprob, cudaStream_t s);
cudaError_t launch_wait_selfcheck(unsigned int *status, int limit, cudaStream_t s);
// The property layer (R <= 16 rows) of the wide path on the CUDA cores.
cudaError_t launch_wide_rows_product(const float *Wt, int n_in, int R, const float *B, int ldb, float *D, int ldd,
                                     int64_t ncols, bool abs_w, int sms, cudaStream_t s);
cudaError_t launch_wide_box(const BoxSource &src, int64_t base, int nb, int d, float *mh, float *ml, float *rr,
                            int64_t *bidx, int sms, cudaStream_t s);
// Wide row kernels: `alpha` (nullable) holds the lower slopes of the chunk's
// boxes, box b (0-based in the chunk) at row (base + b) * alpha_ld.
cudaError_t launch_wide_init(const NetParams<float> &net, const float *W0t, int nb, int NP, const float *mh,
                             const float *ml, const float *rr, float *C, float *Rr, float *Ch, float *Cl,
                             const float *alpha, int64_t alpha_ld, int64_t base, cudaStream_t s);
cudaError_t launch_wide_const(const NetParams<float> &net, int k, int nb, int NP, const float *Ch, const float *Cl,
                              const float *Rr, float *Kh, float *Kl, float *Ke, int sms, cudaStream_t s);
cudaError_t launch_wide_hidden(const NetParams<float> &net, int layer, int nb, int NP, float gcoef, float *C, float *Rr,
                               float *Ch, float *Cl, const float *Kh, const float *Kl, const float *Ke,
                               const float *alpha, int64_t alpha_ld, int64_t base, cudaStream_t s);
cudaError_t launch_wide_final(const NetParams<float> &net, int nb, int NP, float gcoef, float *C, float *Rr, float *Ch,
                              float *Cl, const float *Kh, const float *Kl, const float *Ke, float *lo, float *hi,
                              float *err, cudaStream_t s);
cudaError_t launch_wide_classify(const NetParams<float> &net, int nb, int64_t base, const float *lo, const float *hi,
                                 const float *err, const int64_t *bidx, const EvalOutputs &out, int sms,
                                 cudaStream_t s);

cudaError_t launch_init_count(uint64_t *codes0, LevelCounters *ctr, cudaStream_t s);
cudaError_t launch_compact(const uint64_t *codes_in, const uint8_t *cls, uint64_t *codes_out,
                           LevelCounters *ctr, unsigned int *status, int64_t cap, int t, int D,
                           uint64_t *leaf_codes, uint8_t *leaf_depth, uint8_t *leaf_cls,
                           int64_t leaf_cap, int grid, cudaStream_t s, uint64_t path_mask = ~0ull,
                           bool add_volume = true);
// Keep shard `index` of `count` of level t's frontier (every count-th box from index).
cudaError_t launch_shard_level(uint64_t *codes, uint64_t *scratch, LevelCounters *ctr, int t, int count, int index,
                               int64_t cap, int sms, cudaStream_t s);

}  // namespace slr
