// Device-side structures and arithmetic shared by the SLR kernels.
//
// The symbolic state of one box is kept in centre/radius form over the
// normalised input xi in [-1, 1]^d (x = m + r * xi):
//   upper equation  U(xi) = C(xi) + R(xi),   lower equation  L(xi) = C(xi) - R(xi),
// with C and R affine in xi (d coefficients + constant).  This is the pair of
// linear equations per neuron of Sec. 3; the affine step of the symbolic
// propagation U' = W+ U + W- L + b, L' = W+ L + W- U + b becomes
//   C' = W C + b,   R' = |W| R,
// which is the same map (W+ (C+R) + W- (C-R) = W C + |W| R).
//
// Precision.  The equations are the plain ("raw") SLR of the paper computed in
// the working precision: ReLU cases and slopes are decided from the raw
// concrete bounds, as the FP64 oracle decides them.  Soundness is kept by a
// separate per-neuron scalar E >= 0 with
//     C - R - E  <=  true neuron value  <=  C + R + E    on the box,
// bounded a priori: every rounding adds its bound to E, the affine step maps E
// to |W| E, and a ReLU maps E to at most E (see the epilogue).  The constant
// of C (about the network's value at the box centre, large next to the
// coefficients once boxes are small) is carried as an unevaluated sum of two
// numbers (hi + lo) and propagated with error-free products and sums, so its
// rounding does not dominate E.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace slr {

constexpr int kMaxLayers = 16;
constexpr int kMaxRows = 64;      // property rows
constexpr int kMaxWidth = 1024;   // neurons per layer
constexpr int kMaxDepth = 62;
// Per-box split dimensions (gradient split rule): a path code keeps the halves
// taken in its low kSplitPathBits bits (split j in bit t-1-j) and, above them,
// one 4-bit position in the split set (at most kSplitSetMax dimensions) per
// level, for at most kSplitMaxDepth levels.
constexpr int kSplitPathBits = 16;
constexpr int kSplitSetMax = 16;
constexpr int kSplitMaxDepth = 12;
// CTAs (on as many SMs) of the thread-block cluster that evaluates one tile of
// the FP64 re-check together.
constexpr int kRecheckCluster = 4;

enum : uint8_t { kSafe = 0, kUnsafe = 1, kUndecided = 2 };
enum : int { kRelaxNeurify = 0, kRelaxPaperLiteral = 1, kRelaxInterval = 2 };
// Activation after a hidden layer.
enum : int { kActRelu = 0, kActTanh = 1, kActSigmoid = 2 };

enum : uint32_t {
    kStatusOverflow = 1u,      // a level exceeded the frontier capacity
    kStatusNearOverflow = 2u,  // the FP64 re-check list overflowed
    kStatusLeafOverflow = 4u,  // leaf recording overflowed
    kStatusTimeout = 8u,       // a bounded wait on the tensor core gave up
};

// Tensor-core path: operand layout constants and per-layer weight images.
constexpr int kTcLbo = 144;       // bytes between core matrices along K (128 + 16 pad)
constexpr int kTcTmemCols = 256;  // accumulator columns allocated per CTA
constexpr int kTcMaxWidth = 64;   // widest layer the [W ; |W|] stacking in M = 128 allows

struct TcParams {
    const unsigned char *img[kMaxLayers];  // layer k >= 1: [A hi | A lo | W^T float], shared-memory image
    int img_bytes[kMaxLayers];
    int k_pad[kMaxLayers];                 // K of layer k's product: n[k] rounded up to 8
    int a_bytes;                           // bytes of one A image (128 rows)
    int img_max;                           // largest image, bytes
    int b_bytes;                           // bytes of one B image (Npad rows)
    int sbo;                               // bytes between 8-row groups of A and B
    int NCg;                               // GEMM columns per box: 2d + 3
    int Npad;                              // NCg * T rounded up to 16
    uint32_t idesc;                        // tcgen05 instruction descriptor (tf32, M = 128, N = Npad)
};

// Relative rounding bound of one output of the split-TF32 product:
// dropped lo*lo and TF32 rounding of the lo pieces (3 2^-22) plus FP32
// accumulation, modelled as one 2^-23 rounding per product of the K terms.
__host__ __device__ inline float tc_gamma(int k_pad) {
    return (float)(k_pad + 8) * 0x1p-23f + 3.0f * 0x1p-22f;
}

// Directed-rounding arithmetic, one specialisation per working precision.
template <typename Real> struct Arith;

template <> struct Arith<float> {
    static __device__ __forceinline__ float add_up(float a, float b) { return __fadd_ru(a, b); }
    static __device__ __forceinline__ float add_dn(float a, float b) { return __fadd_rd(a, b); }
    static __device__ __forceinline__ float mul_up(float a, float b) { return __fmul_ru(a, b); }
    static __device__ __forceinline__ float mul_dn(float a, float b) { return __fmul_rd(a, b); }
    static __device__ __forceinline__ float div_up(float a, float b) { return __fdiv_ru(a, b); }
    static __device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float abs(float a) { return fabsf(a); }
    // 2^-23: twice the unit roundoff of round-to-nearest.
    static constexpr float ulp2 = 1.1920928955078125e-07f;
    // Smallest normal number: bounds the absolute error of a subnormal result.
    static constexpr float tiny = 1.1754943508222875e-38f;
};

template <> struct Arith<double> {
    static __device__ __forceinline__ double add_up(double a, double b) { return __dadd_ru(a, b); }
    static __device__ __forceinline__ double add_dn(double a, double b) { return __dadd_rd(a, b); }
    static __device__ __forceinline__ double mul_up(double a, double b) { return __dmul_ru(a, b); }
    static __device__ __forceinline__ double mul_dn(double a, double b) { return __dmul_rd(a, b); }
    static __device__ __forceinline__ double div_up(double a, double b) { return __ddiv_ru(a, b); }
    static __device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double abs(double a) { return fabs(a); }
    static constexpr double ulp2 = 2.220446049250313e-16;    // 2^-52
    static constexpr double tiny = 2.2250738585072014e-308;  // DBL_MIN
};

// Network, property and option parameters, passed by value to the kernels.
// Layer k (0-based) maps n[k] -> n[k+1]; the last layer is already folded
// with the property rows (W' = C W_K, b' = C b_K + e), so n[K] = R.
template <typename Real>
struct NetParams {
    int K;                       // affine layers
    int d;                       // inputs
    int R;                       // property rows
    int n[kMaxLayers + 1];
    int n_max_pad;               // max over n[1..K] rounded up to 8
    int n_in_max;                // max over n[0..K-1]
    const Real *W0;              // layer 0, row-major n[1] x d
    const Real *Wt[kMaxLayers];  // layer k >= 1, transposed: n[k] x n[k+1] row-major
    const Real *Ws[kMaxLayers];  // layer k >= 1, the tile's shared-memory image of Wt[k]:
                                 // n[k] x Mpad_k, Mpad_k = n[k+1] rounded up to 8, padding 0
    int fold_pad;                // 1: Ws[K-1] holds fold_err[p][i] in column n[K] + p
    // float64 tile, hidden -> hidden layers k (1 <= k < K-1): the same weights
    // as float (exact: the network's weights are float32), for the re-check's
    // float-float products, and wabs[k] >= max_p sum_i |W_k[p][i]|
    const float *Wsf[kMaxLayers];
    double wabs[kMaxLayers];
    const Real *b[kMaxLayers];   // biases, b[K-1] folded
    const Real *fold_err;        // R x n[K-1]: bound on |W'_fp - C W_K|
    const Real *fold_berr;       // R:          bound on |b'_fp - (C b_K + e)|
    int n_clauses;
    int clause_end[kMaxRows];    // exclusive end row of each clause
    uint8_t strict[kMaxRows];
    int relax_mode;
    uint8_t act[kMaxLayers];     // activation after layer k (k < K - 1): kAct*
};

// Where the boxes of one evaluation come from.
struct BoxSource {
    // mode 0: depth-t path codes decoded against the root box and split schedule
    // mode 1: explicit float32 endpoints lo/hi (n x d)
    int mode;
    const uint64_t *codes;
    const unsigned long long *count;  // device counter holding n (mode 0)
    int64_t n_explicit;               // mode 1
    const float *lo;
    const float *hi;
    const int64_t *index;             // optional indirection: box k is index[k]
    const unsigned long long *index_count;
    int t;                            // depth of the codes
    int D;                            // depth cap (mask shift)
    const unsigned long long *dim_mask;  // per input dim: bits of the splits on it, full depth D
    const int8_t *split_of;           // per input dim: position in the split set, or -1; non-null
                                      // for per-box split dimensions carried in the codes
    const double *root_lo;            // float64 root box
    const double *root_w;             // float64 root widths
    int64_t cap;                      // upper bound on n (buffer capacity)
    // optional lower ReLU slopes (Eq. 1 lower line, any value in [0, 1] is
    // sound): the box at position k (before indirection) reads row
    // alpha[k * alpha_ld + ...], one entry per hidden neuron, layers in order
    const float *alpha;
    int64_t alpha_ld;
};

struct EvalOutputs {
    uint8_t *cls;                 // per box (indexed like the source before indirection)
    float *row_lo;                // optional, n x R (sound)
    float *row_hi;
    float *row_err;               // optional, n x R: E of the row (rigorous rounding bound)
    int64_t *near_list;           // FP32 pass: undecided boxes within the re-check margin
    unsigned long long *near_count;
    int64_t near_cap;
    unsigned long long *tie_count;  // FP64 pass: boxes whose class still depends on E
    unsigned int *status;
    int by_position;              // cls/row outputs at the position in the source, not at the index
};

// Blocks of the order-preserving compaction (each takes one contiguous range).
constexpr int kCompactBlocks = 1024;

struct LevelCounters {
    unsigned long long unsafe_lo;
    unsigned long long undecided_at_D;
    unsigned long long boxes;
    unsigned long long rechecked;
    unsigned long long ties;
    unsigned long long leaves;
    unsigned long long level_boxes[kMaxDepth + 2];
    unsigned long long level_safe[kMaxDepth + 2];
    unsigned long long level_unsafe[kMaxDepth + 2];
    unsigned long long level_undecided[kMaxDepth + 2];
    unsigned long long frontier_n[kMaxDepth + 2];   // boxes at each level
    unsigned long long near_n[kMaxDepth + 2];       // re-check list length at each level
    unsigned long long near2_n[kMaxDepth + 2];      // second re-check list (tensor-core path)
    unsigned long long near3_n[kMaxDepth + 2];      // boxes the float-float re-check left to plain FP64
    unsigned int block_count[kCompactBlocks];       // order-preserving compaction: per-block undecided
};

// Largest shapes of the problems of one batched launch (shared-memory carve).
struct BatchShape {
    int nmp, d, n_in_max, R;
};

// Columns of one row of the state (see slr_eval.cuh): C coefficients, C
// constant (hi), R coefficients, R constant, N, E, C constant (lo).
__host__ __device__ inline int state_cols(int d) { return 2 * d + 5; }

// Row stride of a tile's state: T (2d + 5) floats padded so that it is T modulo
// 32, i.e. a warp's (row, box) items of consecutive rows fall in distinct banks.
__host__ __device__ inline int state_stride(int T, int d) {
    const int ns = T * state_cols(d);
    return ns + (((T - ns) % 32) + 32) % 32;
}

// Contraction tiles (8 rows x 4 columns) per CTA of the fused kernel; each of
// its threads holds at most two in registers, so this must not exceed 2 x 256.
__host__ __device__ inline int eval_gemm_items(int T, int d, int n_max_pad) {
    return (n_max_pad / 8) * ((2 * d + 4) * T / 4);
}

// Row stride (floats) of the float64 tile's float-float planes: NS rounded up
// to 4, so that every row starts on 16 bytes.
__host__ __device__ inline int eval_plane_stride(int T, int d) { return (state_stride(T, d) + 3) & ~3; }

// Shared-memory footprint of the fused evaluation kernel for a tile of T boxes;
// `pairs` (float64): with the planes of the float-float re-check stage.
template <typename Real>
__host__ __device__ inline size_t eval_smem_bytes(int T, int d, int R, int n_max_pad, int n_in_max,
                                                  bool pairs = false) {
    const int NS = state_stride(T, d);
    size_t s = 0;
    s += (size_t)n_max_pad * NS * sizeof(Real);            // state, updated in place
    s += 3 * (size_t)n_max_pad * T * sizeof(Real);         // next layer's constants (hi, lo, error)
    s += 2 * (size_t)n_max_pad * sizeof(Real);             // reference box's constants
    s += (size_t)n_in_max * n_max_pad * sizeof(Real);      // staged weights (transposed)
    s += 3 * (size_t)T * d * sizeof(Real);                 // box centres (hi, lo) and radii
    s += 3 * (size_t)T * R * sizeof(Real);                 // row lo / hi / E
    s += (size_t)T * sizeof(int64_t);                      // box indices
    s += (size_t)n_max_pad * (sizeof(int2) + 2 * sizeof(int)) + 16;   // live-row list, indices, flags, length
    s = (s + 15) & ~(size_t)15;
    // float64: the state split into float hi and lo planes for the float-float products
    if (sizeof(Real) == 8 && pairs) s += 2 * (size_t)n_max_pad * eval_plane_stride(T, d) * sizeof(float);
    return s;
}

// Offset of the float-float planes in the float64 tile's shared memory (they
// follow everything else).
__host__ __device__ inline size_t eval_split_offset(int T, int d, int R, int n_max_pad, int n_in_max) {
    return eval_smem_bytes<double>(T, d, R, n_max_pad, n_in_max, false);
}

}  // namespace slr
