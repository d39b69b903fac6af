/*
 * slrcount.h - C ABI of the GB300 exact #DNN-Verification counter.
 *
 * The counter follows the problem statement T = <N, P, Q> of Sec. 2.1: a ReLU
 * network N, an input box P (a hyperrectangle) and an output property Q.
 * It bounds every box of one branch-and-bound level at once (Sec. 3) with
 * Symbolic Linear Relaxation (Sec. 2.2, Eq. 1; two linear equations per
 * neuron, Sec. 3), checks the unsafe set against the output bounds (Sec. 3
 * containment check), counts the unsafe volume of decided boxes and bisects
 * the undecided ones (Alg. 1), down to a depth cap D.
 *
 * Conventions for every call:
 *   - Every function returns an slr_status (0 = SLR_OK, negative = error); on
 *     error slr_last_error() holds a one-line message.  No call aborts, throws
 *     or exits across the ABI.
 *   - Inputs are copied; the caller keeps ownership of every buffer it passes.
 *   - Outputs are written into caller buffers.  Pointer arguments are host
 *     pointers unless a call says otherwise.
 *   - One context serves one problem on one GPU and is not thread-safe; use one
 *     context per host thread.
 *   - All device work runs on the context's CUDA stream; every call that
 *     returns results synchronises that stream before returning.
 */
#ifndef SLRCOUNT_H
#define SLRCOUNT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slr_ctx slr_ctx;

typedef enum {
    SLR_OK = 0,
    SLR_EINVAL = -1,       /* bad argument: sizes, lo > hi, non-finite values, D out of range */
    SLR_ENOMEM = -2,       /* device or host allocation failed */
    SLR_ECUDA = -3,        /* a CUDA runtime call failed (message names it) */
    SLR_ESTATE = -4,       /* call order: count/bounds before network, box and property are set */
    SLR_EOVERFLOW = -5,    /* a level produced more boxes than frontier_cap */
    SLR_ETIMEOUT = -6,     /* a bounded device wait gave up */
    SLR_EUNSUPPORTED = -7  /* shape or option not supported by this build */
} slr_status;

/* Box classes (Sec. 3): the reachable set R of the box is inside the unsafe
 * set Y (UNSAFE), disjoint from it (SAFE), or neither (UNDECIDED). */
enum { SLR_SAFE = 0, SLR_UNSAFE = 1, SLR_UNDECIDED = 2 };

/* Reading of Eq. 1 (Sec. 2.2).
 * NEURIFY: the upper line uses the bounds (l_u, u_u) of the upper equation and
 *   the lower slope those (l_l, u_l) of the lower equation (default).
 * PAPER_LITERAL: one pair (l, u) = (min of Eq_l, max of Eq_u) serves both.
 * INTERVAL: no relaxation: every hidden neuron keeps only its interval
 *   [relu(min), relu(max)] (Moore interval propagation, the paper's naive
 *   "Exact Count" baseline of Sec. 4), for comparing split counts. */
enum { SLR_RELAX_NEURIFY = 0, SLR_RELAX_PAPER_LITERAL = 1, SLR_RELAX_INTERVAL = 2 };

/* Arithmetic of the symbolic contraction U' = W+ U + W- L + b, L' = W+ L + W- U + b.
 * FP32: IEEE FP32 FMA on the CUDA cores (the constant terms as float-float
 *   pairs); every rounding is bounded a priori and the bounds are widened
 *   outward by that amount, so every bound stays sound.
 * TC_TF32: the contraction on the tensor cores (tcgen05) with operands split
 *   into two TF32 pieces (three products, FP32 accumulation), widened by its
 *   own a-priori bound; boxes whose class depends on that widening are
 *   re-bounded by the FP32 path (and, if still needed, in FP64).  Needs every
 *   layer and the property at most 64 wide (SLR_EUNSUPPORTED otherwise). */
enum { SLR_PREC_FP32 = 0, SLR_PREC_TC_TF32 = 1 };

/* Which side an UNDECIDED box is bisected along (Sec. 2.2 splits a box into two
 * halves of one input interval and leaves the dimension open).
 * WIDEST: the widest side, ties to the lowest index.  All boxes of a level then
 *   split the same dimension (one schedule, slr_schedule).
 * GRADIENT: per box.  A split set S of at most 16 input dimensions is fixed at
 *   the root: those with the largest |dM/dr_i| w_i, where M is the decision loss
 *   of the slope optimisation at the fixed slopes u/(u-l), r the box radius and
 *   w the root widths (ties to the lowest index).  Each UNDECIDED box then
 *   splits the dimension of S with the largest |dM/dr_i| r_i for its own
 *   radius, the gradient taken by the adjoint at the slopes of its bounds (the
 *   optimised ones when alpha_steps > 0); ties go to the first in S.  Counts
 *   to depth 12 at most; needs relax_mode NEURIFY and every UNDECIDED box of a
 *   level within alpha_cap (SLR_EOVERFLOW otherwise).  slr_split_set returns S. */
enum { SLR_SPLIT_WIDEST = 0, SLR_SPLIT_GRADIENT = 1 };

typedef struct {
    int32_t precision;      /* SLR_PREC_*; default SLR_PREC_FP32 */
    int32_t relax_mode;     /* SLR_RELAX_*; default SLR_RELAX_NEURIFY */
    int32_t fp64_recheck;   /* 1: re-bound in FP64 the undecided boxes that the FP32
                               bounds would decide without their widening; default 1 */
    int32_t record_leaves;  /* 1: keep the leaves of the last count for slr_leaves(); default 0 */
    int32_t profile;        /* 1: time each kernel of a count with CUDA events (kernel_ms); default 0 */
    int32_t split_rule;     /* SLR_SPLIT_*; default SLR_SPLIT_WIDEST */
    int64_t frontier_cap;   /* most boxes one level may hold; default 1<<24 */
    int64_t leaf_cap;       /* most leaves recorded when record_leaves; default 1<<22 */
    int32_t alpha_steps;    /* slr_count: projected-Adam steps on the lower ReLU slopes of the
                               boxes a level leaves UNDECIDED (0 = fixed slopes u/(u-l)); default 0 */
    float alpha_lr;         /* Adam step size of those steps; default 0.1 */
    int64_t alpha_cap;      /* most UNDECIDED boxes per level whose slopes are optimised
                               (the rest keep fixed slopes); default 1<<16 */
    int32_t tile_boxes;     /* FP32 evaluation kernel: boxes per CTA (64, 32, 16, 8 or 4) and */
    int32_t tile_threads;   /* threads per CTA (256 or 128); 0, 0 = chosen by timing (default).
                               A pair the network cannot run with gives SLR_EUNSUPPORTED. */
    int32_t wide;           /* 1: always use the wide path (per-box state in GPU memory, each
                               layer one tensor-core product, no FP64 re-check); 0 (default):
                               only for networks whose per-box state does not fit the fused
                               shared-memory kernel */
    int32_t shard_count;    /* N > 1: this context counts one of N shards of the tree (default 1) */
    int32_t shard_index;    /* which shard, 0..N-1: the level-g boxes whose frontier position
                               is congruent to it modulo N, and everything below them */
    int32_t shard_level;    /* g: every shard evaluates levels 0..g-1 in full, then keeps its
                               share of level g (0 <= g <= D); the unsafe volume of levels
                               below g is added by shard 0 only, so the sums of unsafe_lo and
                               of unsafe_hi over the N shards are the whole count's */
    int32_t recheck_cluster; /* FP64 re-check: 0 (default) = each tile on one CTA; 1 = each tile
                               on a cluster of 4 CTAs (4 SMs) where the GPU can run one, its
                               products dealt over them and exchanged through distributed
                               shared memory.  Both are sound; the products' inputs are summed
                               in another order, so a bound may differ in its last float64 bits */
    float alpha_margin;     /* alpha_steps > 0: optimise only the UNDECIDED boxes whose decision gap
                               at the fixed slopes (the smaller of the SAFE gap sum_c max(0, min_r hi_r)
                               and the UNSAFE gap min_c max(0, -min_r lo_r)) is at most alpha_margin
                               times the box's widest row bound hi_r - lo_r; the others keep fixed
                               slopes (most boxes far from a decision stay undecided whatever the
                               slopes).  0: every UNDECIDED box up to alpha_cap.  Default 0.2.
                               Not applied under SLR_SPLIT_GRADIENT, whose split choices need the
                               optimised slopes of every UNDECIDED box */
    int32_t recheck_pairs;  /* FP64 re-check (one CTA per tile): 1 (default) = in two stages, the first
                               with the hidden-layer products as float-float pairs on the FP32 units
                               (float64 state, constants and relaxation; the pairs' rounding bound,
                               a few 1e-11 relative at 50 inputs, joins the error bound E), the second, with plain
                               FP64 products, on the boxes whose class the first left depending on E;
                               0 = plain FP64 products only.  Both give the same classes: a box is
                               decided by the first stage only when its bound is sound */
} slr_options;

#define SLR_MAX_LEVELS 63

/* Result of slr_count.  Volumes are exact integers in units of 2^-D of the root
 * box volume; the violation rate lies in [unsafe_lo, unsafe_hi] / 2^D. */
typedef struct {
    uint64_t unsafe_lo;     /* volume of the boxes proved UNSAFE */
    uint64_t unsafe_hi;     /* unsafe_lo + boxes still UNDECIDED at depth D */
    uint64_t boxes;         /* boxes bounded over all levels */
    uint64_t rechecked;     /* boxes re-bounded in FP64 (see recheck_pairs) */
    uint64_t tie_leaves;    /* re-bounded boxes whose FP64 class still depends on its widening */
    int32_t depth;          /* D */
    int32_t levels;         /* levels evaluated (D + 1 unless the frontier emptied first) */
    uint64_t level_boxes[SLR_MAX_LEVELS + 1];
    uint64_t level_safe[SLR_MAX_LEVELS + 1];
    uint64_t level_unsafe[SLR_MAX_LEVELS + 1];
    uint64_t level_undecided[SLR_MAX_LEVELS + 1];
    double device_ms;       /* device time of the count (CUDA events on the context stream) */
    double kernel_ms[3];    /* with profile: summed device time of the FP32 evaluation,
                               the FP64 re-check and the compaction kernels */
    int64_t launches;       /* kernels launched by the count */
    int64_t h2d_bytes;      /* host-to-device bytes copied by the count (inputs, schedule) */
    int64_t d2h_bytes;      /* device-to-host bytes copied by the count (counters, status) */
    int32_t tile_boxes;     /* boxes per CTA of the FP32 evaluation kernel (chosen by timing) */
    int32_t tile_threads;   /* threads per CTA of the FP32 evaluation kernel */
    uint64_t rechecked_fp32; /* TC_TF32: boxes re-bounded by the FP32 path */
    uint64_t alpha_boxes;   /* alpha_steps > 0: boxes whose slopes were optimised */
    uint64_t alpha_decided; /* of those, boxes that the optimised slopes decided */
    double alpha_ms;        /* with profile: device time of the slope optimisation */
    double gemm_ms;         /* with profile, wide path: device time of the tensor-core products */
    int64_t gemm_launches;  /* wide path: product launches */
    double gemm_flop;       /* wide path: algorithmic FLOP of those products (2 M N K each) */
    double completion_ms;   /* slr_count_batch: device time from the start of the batch to the end
                               of this problem's last level (0 for slr_count) */
    uint64_t rechecked_fp64; /* of `rechecked`: boxes re-bounded with plain FP64 products (with
                               recheck_pairs, those the float-float stage left depending on E) */
} slr_result;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t to
 * run on, or NULL for a stream the context creates and owns.  *out receives the
 * context (NULL on error). */
int slr_create(slr_ctx **out, int device, void *cuda_stream);

/* Free every device and host resource of the context.  NULL is accepted. */
int slr_destroy(slr_ctx *ctx);

/* Default options (see slr_options). */
void slr_default_options(slr_options *opt);

/* Set options; takes effect at the next count or bounds call. */
int slr_set_options(slr_ctx *ctx, const slr_options *opt);

/* The network N (Sec. 2.1): K affine layers (1 <= K <= 16), widths[0..K] with
 * widths[0] = d inputs and widths[K] outputs (each 1..1024).  W[k] points to a
 * row-major widths[k+1] x widths[k] float32 matrix and b[k] to widths[k+1]
 * float32 biases; ReLU follows every layer except the last (slr_set_activations
 * changes that).  All values must be finite.  Copied to the device. */
int slr_load_network(slr_ctx *ctx, int K, const int32_t *widths,
                     const float *const *W, const float *const *b);

/* Activation after each hidden layer.  Sec. 3 relaxes ReLU (Eq. 1) and names
 * other activations only as an extension; the S-shaped ones here are relaxed
 * by lines over the pre-activation's concrete interval [l, u]:
 *   l >= 0 (concave side): upper = tangent at (l + u) / 2, lower = chord;
 *   u <= 0 (convex side):  upper = chord, lower = tangent at (l + u) / 2;
 *   l < 0 < u:             slope min(s'(l), s'(u)) through (u, s(u)) above
 *                          and through (l, s(l)) below;
 * with every intercept rounded outward by a bound of the error of CUDA's
 * tanh/exp (their documented ulp accuracy), so the bounds stay sound.
 * RELAX_INTERVAL keeps [s(l), s(u)].  Networks with S-shaped activations
 * take no slopes (alpha_steps, slr_margin_backward, slr_optimize_alpha,
 * supplied slopes) and no gradient split rule: SLR_EUNSUPPORTED. */
enum { SLR_ACT_RELU = 0, SLR_ACT_TANH = 1, SLR_ACT_SIGMOID = 2 };

/* Activations of the loaded network's K - 1 hidden layers: act[k] follows
 * layer k (SLR_ACT_*); n must be K - 1.  slr_load_network resets every
 * hidden layer to ReLU.  SLR_ESTATE before a network is loaded, SLR_EINVAL
 * for a wrong n or an unknown value. */
int slr_set_activations(slr_ctx *ctx, int n, const int32_t *act);

/* The input box P (Sec. 2.1): d float32 endpoints with lo[i] <= hi[i], finite. */
int slr_set_box(slr_ctx *ctx, int d, const float *lo, const float *hi);

/* The unsafe set Y, i.e. the negated postcondition Q (Sec. 3): an OR over
 * n_clauses clauses, clause c being an AND over rows_per_clause[c] rows; row r
 * holds when C[r] . y + e[r] >= 0 (> 0 if strict[r]).  C is row-major
 * R x n_out float32 with R = sum(rows_per_clause) <= 64 and n_out equal to the
 * network's output width.  e is float32[R], strict uint8[R]. */
int slr_set_property(slr_ctx *ctx, int n_clauses, const int32_t *rows_per_clause,
                     int n_out, const float *C, const float *e, const uint8_t *strict);

/* Count to depth D (0 <= D <= 62): Alg. 1 level by level (Sec. 3), bisecting the
 * widest side of each undecided box (ties to the lowest index).  An UNSAFE box
 * at depth t adds 2^(D-t) to unsafe_lo; an UNDECIDED box at depth D adds 1 to
 * unsafe_hi - unsafe_lo.  Needs network, box and property (SLR_ESTATE). */
int slr_count(slr_ctx *ctx, int D, slr_result *out);

/* Bound n boxes given by float32 endpoints box_lo/box_hi (n x d, row-major) and
 * write, for each box, the SLR lower/upper bound of every property row
 * (row_lo/row_hi, n x R), the rigorous bound E of the rounding error of that
 * row (row_err, n x R) and the box class (cls, n bytes).  Any output may be
 * NULL, but row_lo and row_hi go together.  `on_device` = 1 means every
 * pointer is a device pointer (CUDA global memory of the context's device); 0
 * means host memory.  row_lo/row_hi are sound for the float32 network: they
 * are the FP32 SLR bounds widened outward by E, so row_lo + row_err and
 * row_hi - row_err are the FP32 SLR bounds themselves.  No FP64 re-check is
 * applied here.  `alpha` (nullable, n x H with H from slr_alpha_width) gives
 * the lower slope of every hidden neuron of every box, clamped to [0, 1]
 * (relax mode NEURIFY, FP32 precision); NULL uses u_l / (u_l - l_l).  Needs
 * network and property (SLR_ESTATE); with host pointers lo > hi or non-finite
 * endpoints give SLR_EINVAL. */
int slr_bounds(slr_ctx *ctx, int64_t n, const float *box_lo, const float *box_hi,
               const float *alpha, float *row_lo, float *row_hi, float *row_err, uint8_t *cls,
               int on_device);

/* Hidden neurons of the loaded network, H = widths[1] + ... + widths[K-1]: the
 * row length of every slope array below. */
int slr_alpha_width(slr_ctx *ctx, int64_t *H);

/* Reverse mode of the SLR pass (Sec. 2.2, Eq. 1; Sec. 3) for n boxes.  With
 * lo, hi the float32 SLR row bounds of each box (round to nearest, not widened),
 * the loss is J = sum over boxes b and rows r of g_lo[b,r] lo[b,r] + g_hi[b,r]
 * hi[b,r] (g_lo, g_hi: n x R, required).  Writes, each output optional (NULL):
 *   row_lo, row_hi  n x R: lo and hi;
 *   d_alpha         n x H: dJ/d(slope) of every hidden neuron, the slopes
 *                   being free variables; 0 for neurons whose lower line is
 *                   not a slope line (stable, or u_l <= 0);
 *   d_box_lo, d_box_hi  n x d: dJ/d(box endpoints);
 *   d_W, d_b        K pointers each (NULL, or all K set): dJ/dW_k
 *                   (widths[k+1] x widths[k], row-major) and dJ/db_k, summed
 *                   over the boxes and overwritten.  The last layer's
 *                   gradients are those of the network's own W_K, b_K (the
 *                   property rows C are folded in as C W_K).
 * `alpha` (n x H, nullable) gives the lower slopes; entries are clamped to
 * [0, 1] (any slope in [0, 1] is sound: relu(z) >= a z >= a Eq_l).  NULL uses
 * u_l / (u_l - l_l) and then the gradients also flow through that formula
 * (d_alpha is then dJ/d(slope) at those slopes, holding the box fixed).
 * Gradients are those of the piecewise-smooth bounds: at a kink (a ReLU case
 * or a coefficient sign changing) they are one-sided.  Relax mode NEURIFY
 * only (SLR_EUNSUPPORTED otherwise).  `on_device` as in slr_bounds, for every
 * pointer; float32 atomics make d_W and d_b vary in the last bits run to run. */
int slr_margin_backward(slr_ctx *ctx, int64_t n, const float *box_lo, const float *box_hi,
                        const float *alpha, const float *g_lo, const float *g_hi,
                        float *row_lo, float *row_hi, float *d_alpha,
                        float *d_box_lo, float *d_box_hi, float *const *d_W,
                        float *const *d_b, int on_device);

/* Tighten the bounds of n boxes by `steps` projected-Adam steps on their lower
 * ReLU slopes (lr = step size; betas 0.9, 0.999), starting from u_l/(u_l - l_l).
 * Each step differentiates the nearer decision's loss (the SAFE loss
 * sum_c max(0, min_{r in c} hi_r) or the UNSAFE loss min_c max(0, -min_{r in c}
 * lo_r), chosen per box at the first step), moves the slopes and clips them
 * to [0, 1]; then the sound FP32 bounds at the new slopes are intersected with
 * the best so far.  Writes the intersected sound bounds (row_lo/row_hi, n x R,
 * including the starting slopes), the class they give (cls), and the final
 * slopes (alpha, n x H); each output optional.  on_device as in slr_bounds. */
int slr_optimize_alpha(slr_ctx *ctx, int64_t n, const float *box_lo, const float *box_hi,
                       int steps, float lr, float *alpha, float *row_lo, float *row_hi,
                       uint8_t *cls, int on_device);

/* Leaves of the last slr_count when record_leaves was set: for each leaf its
 * path code (bit t-1-j = half taken at split j, 1 = upper), depth and class.
 * Under SLR_SPLIT_GRADIENT the path takes the low 16 bits and bits 16+4j ..
 * 19+4j hold the position in the split set of the dimension split j took.
 * Leaves are the SAFE and UNSAFE boxes of every level and the UNDECIDED boxes of
 * depth D, in no particular order.  Writes at most `cap` entries and sets *n to
 * the total number recorded (SLR_EOVERFLOW if leaf_cap was exceeded). */
int slr_leaves(slr_ctx *ctx, int64_t cap, uint64_t *codes, uint8_t *depth,
               uint8_t *cls, int64_t *n);

/* The split dimension of each of the first D levels of the last count (the
 * widest-side schedule), D entries.  SLR_ESTATE after a SLR_SPLIT_GRADIENT count. */
int slr_schedule(slr_ctx *ctx, int D, int32_t *dims);

/* The split set S of the last SLR_SPLIT_GRADIENT count, ascending: writes *n <= 16
 * dimensions to dims (room for 16).  SLR_ESTATE after a widest-side count. */
int slr_split_set(slr_ctx *ctx, int32_t *dims, int32_t *n);

/* Failure detection check (no paper counterpart): runs, on the context's
 * device and stream, the bounded wait that the tensor-core kernels use, on a
 * barrier phase that nothing completes, giving up after `limit` polls
 * (1..2^20).  Returns SLR_ETIMEOUT, as every count does when one of its waits
 * gives up, and leaves the context usable; SLR_OK would mean the wait did not
 * give up. */
int slr_wait_selfcheck(slr_ctx *ctx, int32_t limit);

/* One problem of a batch: a network, an input box, a property (as in
 * slr_load_network, slr_set_box and slr_set_property) and its depth cap. */
typedef struct {
    int32_t K;                        /* affine layers */
    const int32_t *widths;            /* widths[0..K] */
    const float *const *W;            /* W[k]: widths[k+1] x widths[k], row-major */
    const float *const *b;            /* b[k]: widths[k+1] */
    const float *lo;                  /* box: widths[0] endpoints, lo <= hi */
    const float *hi;
    int32_t n_clauses;                /* property: OR over clauses of AND over rows */
    const int32_t *rows_per_clause;
    const float *C;                   /* R x widths[K], row-major */
    const float *e;                   /* R */
    const uint8_t *strict;            /* R */
    int32_t depth;                    /* D of this problem, 0..62 */
} slr_problem;

/* Count n problems of uneven size together (Alg. 1 for each, Sec. 3 level
 * evaluation across all of them): every level step bounds the current level
 * of every unfinished problem, tiles never mixing problems; problems with
 * smaller depth caps simply finish earlier.  Problems are grouped by the
 * largest tile (32, 16, 8 or 4 boxes) their shape fits, one persistent launch
 * per group and step.  The step loop is captured once as a CUDA graph and
 * replayed while later calls keep the batch's shape (same widths, rows,
 * clauses and depths; weights, boxes and properties may change).  Problems
 * too wide for any tile are counted on the wide path in the same call, after
 * the tiled ones, four at a time (host threads, each with a helper context
 * and stream of its own).  results[i] receives problem i's count as
 * slr_count would return it (device_ms is the time of the whole batch,
 * completion_ms the time from its start to the end of problem i's last level;
 * tile_boxes the problem's tile).
 * Inputs are copied.  Each problem's frontier holds up to min(2^depth,
 * frontier_cap) boxes (SLR_EOVERFLOW beyond).  Uses the context's options
 * (relax_mode, fp64_recheck, frontier_cap) and stream; FP32 arithmetic with
 * the FP64 re-check; the widest-side split rule only (SLR_EUNSUPPORTED under
 * SLR_SPLIT_GRADIENT). */
int slr_count_batch(slr_ctx *ctx, int n, const slr_problem *problems, slr_result *results);

/* slr_count for callers that cannot allocate GPU memory.  The paper has no
 * counterpart: this entry exists for programs that set the library up once
 * and then count from code where cudaMalloc/cudaFree are not allowed (while a
 * framework's caching allocator holds the device memory, or inside a
 * real-time loop that must not stall on allocation, which can synchronise the
 * whole device).
 *
 * It runs the FP32 tile path with fixed slopes and the one-CTA FP64 re-check:
 * a context set to the wide path, alpha_steps > 0, precision TC_TF32,
 * recheck_cluster, the gradient split rule or sharding gets SLR_EUNSUPPORTED.
 * Otherwise it takes the same arguments and gives the same result and
 * classification as slr_count, but every scratch
 * buffer (two frontiers of path codes, class bytes, the FP64 re-check list,
 * level counters, root box and split masks) lives in one fixed device array
 * of about 4.8 MB that the library defines at file scope: each GPU that loads
 * the library holds it until the process exits.  Limits: at most 262144
 * boxes per level and 65536 re-checked boxes per level; a count that needs
 * more returns SLR_EOVERFLOW (its result is then incomplete).  Leaves are not
 * recorded, slr_schedule is not updated and profile timing is not taken.
 *
 * The network and property must already be on the device: call slr_count (or
 * slr_bounds with n >= 1) once after setting them, else SLR_ESTATE.  The
 * first call on a device looks up the array's device address (a CUDA runtime
 * query, no allocation); make that first call before any stream capture.
 * All calls share the one array: calls that overlap on the GPU (two contexts
 * or streams at once on one device) race and give wrong counts; run them one
 * after another.  Each call clears the counters it needs before use. */
int slr_count_noalloc(slr_ctx *ctx, int D, slr_result *out);

/* Checkpoint and resume of a count at a level boundary.  Alg. 1 evaluates
 * the tree level by level (Sec. 3), so between levels t and t + 1 the whole
 * state of a count is the frontier F_{t+1} (the path codes of the boxes that
 * level t left UNDECIDED) and the counters of levels 0..t.
 *
 * slr_count_checkpoint runs levels 0..t (0 <= t < D) of a count to depth D
 * and writes that state into the caller's host buffer buf of cap bytes: a
 * self-describing blob (format tag, D, t, a fingerprint of the network, box,
 * property and the options that change results, the counters, then the
 * frontier's 8-byte codes in frontier order).  *used receives its size in
 * bytes.  If buf is NULL or cap < *used, nothing is written and SLR_EINVAL is
 * returned with *used set: call again with a buffer that large (the levels
 * are recomputed, with the same result).  The blob is plain host memory owned
 * by the caller; it may be written to a file and resumed in another process
 * on a GPU of the same kind.
 *
 * slr_count_resume continues such a count from level t + 1 to its depth D and
 * fills out as slr_count would for the whole count (counts and per-level
 * statistics of every level; device_ms, launches and kernel_ms cover the
 * resumed levels only).  The context must hold the same network, box,
 * property and result options (precision, relax_mode, fp64_recheck,
 * recheck_cluster, recheck_pairs, wide), else SLR_EINVAL; a blob that is truncated or not a
 * checkpoint gives SLR_EINVAL.  The blob also records the FP32 tile (boxes
 * and threads per CTA) of the checkpointed levels: the resumed levels run
 * that tile, whatever the context's own choice, because the tile fixes the
 * order of the FP32 sums and so which boxes take the FP64 re-check.  Neither call supports record_leaves, alpha_steps > 0, the
 * gradient split rule or sharding (SLR_EUNSUPPORTED). */
int slr_count_checkpoint(slr_ctx *ctx, int D, int t, void *buf, size_t cap, size_t *used);
int slr_count_resume(slr_ctx *ctx, const void *buf, size_t bytes, slr_result *out);

/* Approximate counter CountingProVe_SLR (Sec. 2.3; Sec. 4, Table 1's
 * "Approximations" block).  Each of `trials` independent trials starts from
 * the context's box and makes up to `splits` balanced splits: it samples
 * `samples` points uniformly in the current box (SplitMix64, Steele, Lea and
 * Flood 2014, as a counter-based generator keyed by seed, trial, split, point
 * and coordinate), evaluates the network in float64 at each one, and splits
 * the widest side (ties to the lowest index) at the lower median of the
 * sampled unsafe points' coordinates on that side (rounded to the nearest
 * float32; the midpoint when no sample is unsafe), so that the sampled
 * violations are shared evenly by the halves; a fair coin (one more draw)
 * keeps one half.  A side too narrow to split ends the trial's splitting.
 * The final leaf is counted exactly, as slr_count does with the context's
 * options, to depth leaf_depth: [lo_l, hi_l] in units of 2^-leaf_depth of the
 * leaf.  The trial's estimate of the violation rate is
 *     X = 2^s lo_l 2^-leaf_depth vol(leaf) / vol(root)   (s: splits made).
 * Since the coin picks each half with probability 1/2, E[X] is at most the
 * violation rate VR; by Markov's inequality P(X >= 2^beta VR) <= 2^-beta, so
 *     vr_lower = 2^-beta min_i X_i <= VR   with probability >= 1 - 2^(-beta trials)
 * (the confidence reported).  The library computes this guarantee; the
 * paper states it for CountingProVe without the derivation.  Volumes of
 * zero-width root sides are left out of vol(.).  Needs network, box and
 * property (SLR_ESTATE); SLR_EINVAL for options out of range; sharded
 * contexts get SLR_EUNSUPPORTED.  leaf_lo, leaf_hi (nullable, trials x d
 * float32) receive each trial's leaf box. */
#define SLR_APPROX_MAX_TRIALS 64
typedef struct {
    int32_t trials;      /* 1..64; default 8 */
    int32_t splits;      /* balanced splits per trial before the exact count, 0..62; default 10 */
    int32_t samples;     /* points sampled per split, 1 .. 2^24 - 2; default 4096 */
    int32_t leaf_depth;  /* depth of the exact count of the final leaf, 0..62; default 12 */
    double beta;         /* tolerance > 0 of the lower bound; default 1 */
    uint64_t seed;       /* generator seed; default 0 */
} slr_approx_options;

typedef struct {
    double vr_lower;                                   /* 2^-beta min over trials of X_i */
    double confidence;                                 /* 1 - 2^(-beta trials) */
    double vr_mean;                                    /* mean of the X_i */
    int32_t trials;
    int32_t splits_done[SLR_APPROX_MAX_TRIALS];        /* s of each trial */
    uint64_t leaf_unsafe_lo[SLR_APPROX_MAX_TRIALS];    /* exact count of the leaf, units 2^-leaf_depth */
    uint64_t leaf_unsafe_hi[SLR_APPROX_MAX_TRIALS];
    double leaf_volume[SLR_APPROX_MAX_TRIALS];         /* vol(leaf) / vol(root) */
    double estimate[SLR_APPROX_MAX_TRIALS];            /* X_i */
    double estimate_hi[SLR_APPROX_MAX_TRIALS];         /* X_i with hi_l in place of lo_l */
    uint64_t boxes;                                    /* boxes bounded by the leaves' exact counts */
    uint64_t samples_unsafe;                           /* sampled points found unsafe */
    double device_ms;                                  /* device time of sampling and leaf counts */
} slr_approx_result;

void slr_default_approx_options(slr_approx_options *opt);
int slr_count_approx(slr_ctx *ctx, const slr_approx_options *opt, slr_approx_result *out, float *leaf_lo,
                     float *leaf_hi);

/* Measurement aid (no paper counterpart): the FP32 fused multiply-add rate of
 * CUDA device `device` in TFLOP/s (2 FLOP per FMA), the roofline denominator
 * of the CUDA-core kernels.  Runs, on a stream of its own, a kernel in which
 * every thread of 8 CTAs of 256 threads per SM issues 16 independent FMA
 * chains of `iters` steps (>= 1; 1 << 19 takes about 70 ms on a GB300), four
 * times, and reports the fastest of the last three: *tflops (required) and
 * its duration in ms (*ms, nullable).  SLR_EINVAL for a NULL tflops or
 * iters < 1, SLR_ECUDA if a CUDA call fails. */
int slr_measure_fp32_peak(int device, int iters, double *tflops, double *ms);

/* Message of the last failed call on this context ("" if none).  With a NULL
 * context, the message of the last failed slr_create on this thread. */
const char *slr_last_error(const slr_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SLRCOUNT_H */
