// C ABI of the SLR counter: context, validation, device copies of the
// network and the level loop of the count (Alg. 1, Sec. 3).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "slrcount.h"
#include "slr_approx.h"
#include "slr_kernels.h"
#include "slr_noalloc.h"

namespace {

thread_local std::string g_create_error;

constexpr size_t kAlign = 256;
constexpr int kMaxSmem = 232448;   // 227 KB of dynamic shared memory per CTA

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

float round_up_to_float(double x) {
    float f = (float)x;
    if ((double)f < x) f = std::nextafter(f, INFINITY);
    return f;
}

template <typename Real>
struct HostLayers {
    // layer 0 row-major, layers >= 1 transposed, the last folded with the property
    std::vector<std::vector<Real>> W;
    std::vector<std::vector<Real>> b;
    std::vector<Real> fold_err, fold_berr;
    // layers >= 1: the fused tile's shared-memory image of W (rows padded to a
    // multiple of 8 columns); float, at most 4 property rows: the fold's error
    // bounds in the last image's padding columns R .. 2R - 1
    std::vector<std::vector<Real>> Ws;
    bool fold_pad = false;
};

}  // namespace

// Device state of the last batched count, reused while the batch keeps its shape.
struct BatchState {
    std::string key;
    void *arena = nullptr;
    size_t upload_bytes = 0;             // weights, network params, roots and masks (re-uploaded per call)
    unsigned char *h_upload = nullptr;   // pinned staging of the upload region
    cudaGraphExec_t graph = nullptr;
    int P = 0, Dmax = 0;
    slr::LevelCounters *ctrs = nullptr;  // P counters
    unsigned int *status = nullptr;
    slr::LevelCounters *h_ctrs = nullptr;
    std::vector<int64_t> near_cap;
    int64_t launches = 0;
    int T32 = 0, T64 = 0;
    std::vector<int> tile_of;            // per problem: boxes per tile of its class
    std::vector<cudaEvent_t> step_ev;    // recorded at the end of each level step (graph nodes)
};

struct slr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    slr_options opt{};

    int K = 0;
    std::vector<int> widths;
    std::vector<std::vector<float>> W, b;
    std::vector<float> lo, hi;
    int n_clauses = 0;
    std::vector<int> rpc;
    std::vector<float> C, e;
    std::vector<uint8_t> strict;
    std::vector<int> act;                 // activation after each hidden layer (empty: ReLU)
    bool has_net = false, has_box = false, has_prop = false;

    bool dev_dirty = true;
    void *net_buf = nullptr;
    slr::NetParams<float> nf{};
    slr::NetParams<double> nd{};
    int T32 = 0, T64 = 0, NT32 = 0, NT64 = 0;
    bool pairs_fit = false;   // the FP64 tile's footprint holds the float-float stage's planes
    size_t smem32 = 0, smem64 = 0;
    int grid32 = 0, grid64 = 0;
    int grid64c = 0;   // > 0: the FP64 re-check on clusters (grid of that many CTAs)
    void *tc_buf = nullptr;               // tensor-core weight images
    slr::TcParams tcp{};
    int T_tc = 0, grid_tc = 0;
    size_t smem_tc = 0;
    bool tc_ok = false;
    int64_t *near_list2 = nullptr;
    BatchState *batch = nullptr;
    std::vector<slr_ctx *> wide_helpers;  // batched counts: problems too wide for a tile (own streams)
    void *split_buf = nullptr;            // gradient split rule: set, dimension map, root gradient
    cudaGraphExec_t count_graph = nullptr;  // the tile path's level loop, captured once per configuration
    std::string count_graph_key;
    int64_t count_graph_launches = 0;
    std::vector<int> split_set;           // split set of the last count (ascending); empty: widest side
    std::string tuned_key;                // network shape the FP32 tile choice was timed for
    int tuned_T = 0, tuned_NT = 0;
    const float *dC = nullptr;            // property rows on the device (inside net_buf)
    int64_t H = 0;                        // hidden neurons (slope row length)
    int adj_nck = 0, adj_grid = 0, adj_nmax = 0, adj_boxes = 1;
    bool adj_gmem = false;                // adjoint state in global memory (wide networks)
    void *adj_scratch = nullptr;
    size_t adj_scratch_bytes = 0;
    size_t adj_smem = 0;
    void *alpha_buf = nullptr;            // slope optimisation during a count
    size_t alpha_buf_bytes = 0;
    unsigned long long *alpha_ctr = nullptr;  // per level: undecided list length, then decided
    bool wide = false;                    // per-box state in HBM, one tensor-core product per layer
    int wide_NP = 0, wide_Bc = 0;
    void *wide_img = nullptr;             // TF32 pieces of W and |W| per layer
    const float *w_hi[slr::kMaxLayers] = {}, *w_lo[slr::kMaxLayers] = {};
    const float *wa_hi[slr::kMaxLayers] = {}, *wa_lo[slr::kMaxLayers] = {};
    const float *w0t = nullptr;           // layer 1 transposed (d x n_1)
    int w_Kpad[slr::kMaxLayers] = {};
    // transposed pieces (W_k^T, |W_k|^T) for the adjoint's backward products
    const float *wt_hi[slr::kMaxLayers] = {}, *wt_lo[slr::kMaxLayers] = {};
    const float *wta_hi[slr::kMaxLayers] = {}, *wta_lo[slr::kMaxLayers] = {};
    int wt_Kpad[slr::kMaxLayers] = {};
    void *wadj_buf = nullptr;             // the wide adjoint's chunk state
    size_t wadj_bytes = 0;
    int wadj_Bc = 0;
    void *approx_buf = nullptr;           // approximate counter: box, sampled coordinates, count
    size_t approx_bytes = 0;
    void *wide_buf = nullptr;             // chunk state
    size_t wide_buf_bytes = 0;
    std::vector<cudaEvent_t> gemm_ev;     // profile: a pair around each product launch
    size_t gemm_ev_used = 0;
    int64_t gemm_launches = 0;
    double gemm_flop = 0;

    int64_t cap = 0, near_cap = 0;
    uint64_t *codes[2] = {nullptr, nullptr};
    uint8_t *cls = nullptr;
    int64_t *near_list = nullptr;
    slr::LevelCounters *ctr = nullptr;
    unsigned int *status = nullptr;
    double *root = nullptr;
    unsigned long long *masks = nullptr;
    int root_d = 0;

    int64_t leaf_cap_alloc = 0;
    uint64_t *leaf_codes = nullptr;
    uint8_t *leaf_depth = nullptr, *leaf_cls = nullptr;
    bool leaves_valid = false;
    int64_t n_leaves = 0;
    std::vector<int> sched;

    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    int sm_count = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<cudaEvent_t> prof_ev;   // profile: one event before and after each launch
    slr::LevelCounters *h_ctr = nullptr;
    unsigned int *h_status = nullptr;
    unsigned char *h_stage = nullptr;     // pinned staging for host-to-device copies
    size_t h_stage_bytes = 0;
    int64_t h2d_pending = 0;              // bytes uploaded since the last count returned
};

namespace {

int fail(slr_ctx *ctx, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    else g_create_error = buf;
    return code;
}

int cuda_fail(slr_ctx *ctx, cudaError_t e, const char *what) {
    const int code = e == cudaErrorMemoryAllocation ? SLR_ENOMEM : SLR_ECUDA;
    return fail(ctx, code, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(ctx, call)                                              \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
    } while (0)

bool finite_all(const float *p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// Fold the property rows into the last layer in float64 (Sec. 3 check on the
// rows C y + e): W' = C W_K, b' = C b_K + e, with a bound on the float64
// rounding error, then round to the working precision and add that rounding.
template <typename Real, typename Src>
void build_layers(const Src *ctx, HostLayers<Real> &L) {
    const int K = ctx->K;
    const int R = (int)ctx->e.size();
    const int n_out = ctx->widths[K];
    const int n_prev = ctx->widths[K - 1];
    const double g64 = (double)(n_out + 3) * std::ldexp(1.0, -52);
    std::vector<double> Wf((size_t)R * n_prev), Wf_err((size_t)R * n_prev), bf(R), bf_err(R);
    const std::vector<float> &WK = ctx->W[K - 1];
    const std::vector<float> &bK = ctx->b[K - 1];
    for (int r = 0; r < R; ++r) {
        for (int i = 0; i < n_prev; ++i) {
            double s = 0.0, a = 0.0;
            for (int o = 0; o < n_out; ++o) {
                const double c = ctx->C[(size_t)r * n_out + o];
                const double w = WK[(size_t)o * n_prev + i];
                s += c * w;
                a += std::fabs(c * w);
            }
            Wf[(size_t)r * n_prev + i] = s;
            Wf_err[(size_t)r * n_prev + i] = g64 * a;
        }
        double s = ctx->e[r], a = std::fabs((double)ctx->e[r]);
        for (int o = 0; o < n_out; ++o) {
            const double c = ctx->C[(size_t)r * n_out + o];
            s += c * (double)bK[o];
            a += std::fabs(c * (double)bK[o]);
        }
        bf[r] = s;
        bf_err[r] = g64 * a;
    }
    L.W.assign(K, {});
    L.b.assign(K, {});
    for (int k = 0; k < K; ++k) {
        const int ni = ctx->widths[k];
        const bool last = k == K - 1;
        const int no = last ? R : ctx->widths[k + 1];
        std::vector<Real> &w = L.W[k];
        w.resize((size_t)ni * no);
        for (int p = 0; p < no; ++p) {
            for (int i = 0; i < ni; ++i) {
                const Real v = last ? (Real)Wf[(size_t)p * ni + i] : (Real)ctx->W[k][(size_t)p * ni + i];
                if (k == 0) w[(size_t)p * ni + i] = v;       // row-major
                else w[(size_t)i * no + p] = v;              // transposed
            }
        }
        L.b[k].resize(no);
        for (int p = 0; p < no; ++p) L.b[k][p] = last ? (Real)bf[p] : (Real)ctx->b[k][p];
    }
    L.fold_err.resize((size_t)R * n_prev);
    L.fold_berr.resize(R);
    for (size_t i = 0; i < (size_t)R * n_prev; ++i) {
        const double rounded = (double)(Real)Wf[i];
        const double tot = std::fabs(rounded - Wf[i]) + Wf_err[i];
        L.fold_err[i] = sizeof(Real) == 4 ? (Real)round_up_to_float(tot * (1 + 1e-15)) : (Real)(tot * (1 + 1e-15));
    }
    for (int r = 0; r < R; ++r) {
        const double rounded = (double)(Real)bf[r];
        const double tot = std::fabs(rounded - bf[r]) + bf_err[r];
        L.fold_berr[r] = sizeof(Real) == 4 ? (Real)round_up_to_float(tot * (1 + 1e-15)) : (Real)(tot * (1 + 1e-15));
    }
    L.Ws.assign(K, {});
    for (int k = 1; k < K; ++k) {
        const int ni = ctx->widths[k];
        const int no = k == K - 1 ? R : ctx->widths[k + 1];
        const int mp = (no + 7) & ~7;
        std::vector<Real> &img = L.Ws[k];
        img.assign((size_t)ni * mp, (Real)0);
        for (int i = 0; i < ni; ++i)
            for (int p = 0; p < no; ++p) img[(size_t)i * mp + p] = L.W[k][(size_t)i * no + p];
    }
    L.fold_pad = sizeof(Real) == 4 && K > 1 && 2 * R <= ((R + 7) & ~7);
    if (L.fold_pad) {
        const int mp = (R + 7) & ~7;
        for (int p = 0; p < R; ++p)
            for (int i = 0; i < n_prev; ++i) L.Ws[K - 1][(size_t)i * mp + R + p] = L.fold_err[(size_t)p * n_prev + i];
    }
}

template <typename Real>
size_t layers_bytes(const HostLayers<Real> &L) {
    size_t s = 0;
    for (auto &w : L.W) s += align_up(w.size() * sizeof(Real));
    for (auto &b : L.b) s += align_up(b.size() * sizeof(Real));
    for (auto &w : L.Ws) s += align_up(w.size() * sizeof(Real));
    s += align_up(L.fold_err.size() * sizeof(Real)) + align_up(L.fold_berr.size() * sizeof(Real));
    return s;
}

template <typename Real, typename Src>
void layout_params(const Src *ctx, const HostLayers<Real> &L, unsigned char *dev, unsigned char *host,
                   size_t &off, slr::NetParams<Real> &p) {
    auto put = [&](const std::vector<Real> &v) -> const Real * {
        const Real *dp = reinterpret_cast<const Real *>(dev + off);
        std::memcpy(host + off, v.data(), v.size() * sizeof(Real));
        off += align_up(v.size() * sizeof(Real));
        return dp;
    };
    const int K = ctx->K;
    std::memset(&p, 0, sizeof p);
    p.K = K;
    p.d = ctx->widths[0];
    p.R = (int)ctx->e.size();
    for (int k = 0; k < K; ++k) p.n[k] = ctx->widths[k];
    p.n[K] = p.R;
    int nmax = 0, nin = 0;
    for (int k = 1; k <= K; ++k) nmax = std::max(nmax, p.n[k]);
    for (int k = 1; k < K; ++k) nin = std::max(nin, p.n[k]);
    p.n_max_pad = (nmax + 7) & ~7;
    p.n_in_max = std::max(nin, 1);
    p.W0 = put(L.W[0]);
    for (int k = 1; k < K; ++k) p.Wt[k] = put(L.W[k]);
    for (int k = 1; k < K; ++k) p.Ws[k] = put(L.Ws[k]);
    p.fold_pad = L.fold_pad ? 1 : 0;
    // hidden -> hidden: max_p sum_i |W[p][i]| (float64 sums of float weights, widened)
    for (int k = 1; k + 1 < K; ++k) {
        const int ni = p.n[k], no = p.n[k + 1];
        double m = 0.0;
        for (int q = 0; q < no; ++q) {
            double a = 0.0;
            for (int i = 0; i < ni; ++i) a += std::fabs((double)L.W[k][(size_t)i * no + q]);
            m = std::max(m, a);
        }
        p.wabs[k] = m * (1.0 + 1e-12) + 1e-300;
    }
    for (int k = 0; k < K; ++k) p.b[k] = put(L.b[k]);
    p.fold_err = put(L.fold_err);
    p.fold_berr = put(L.fold_berr);
    p.n_clauses = ctx->n_clauses;
    int end = 0;
    for (int c = 0; c < ctx->n_clauses; ++c) {
        end += ctx->rpc[c];
        p.clause_end[c] = end;
    }
    for (int r = 0; r < p.R; ++r) p.strict[r] = ctx->strict[r];
    p.relax_mode = ctx->opt.relax_mode;
    for (int k = 0; k + 1 < K; ++k) p.act[k] = (uint8_t)(k < (int)ctx->act.size() ? ctx->act[k] : slr::kActRelu);
}

struct TileChoice {
    int T = 0, NT = 0, blocks = 0;
    size_t smem = 0;
};

// Every (boxes per CTA, threads per CTA) the fused kernel can run this network with.
// pairs (float64): with the planes of the float-float re-check stage.
template <typename Real>
std::vector<TileChoice> tile_candidates(const slr::NetParams<Real> &p, bool pairs = false) {
    std::vector<TileChoice> out;
    for (int NT : slr::kThreadCounts) {
        for (int T : slr::kTileSizes) {
            TileChoice c;
            c.T = T;
            c.NT = NT;
            c.smem = slr::eval_smem_bytes<Real>(T, p.d, p.R, p.n_max_pad, p.n_in_max, pairs);
            if (c.smem > (size_t)kMaxSmem) continue;
            if (slr::eval_gemm_items(T, p.d, p.n_max_pad) > 2 * NT) continue;
            c.blocks = sizeof(Real) == 4 ? slr::eval_blocks_per_sm_f32(T, NT, c.smem,
                                                                       slr::eval_gemm_items(T, p.d, p.n_max_pad))
                                         : slr::eval_blocks_per_sm_f64(T, NT, c.smem);
            if (c.blocks <= 0) continue;
            out.push_back(c);
        }
    }
    return out;
}

int ensure_stage(slr_ctx *ctx, size_t bytes) {
    if (ctx->h_stage_bytes >= bytes) return SLR_OK;
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    ctx->h_stage = nullptr;
    ctx->h_stage_bytes = 0;
    CK(ctx, cudaMallocHost(&ctx->h_stage, bytes));
    ctx->h_stage_bytes = bytes;
    return SLR_OK;
}

float tf32_host(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;
    u = (u + 0x1000u) & 0xffffe000u;   // nearest, ties away from zero, 10 fraction bits
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// Weight images of the tensor-core path (see slr_eval_tc.cu): for each layer
// k >= 1, A = [W ; |W|] split into TF32 hi and lo in the K-major shared-memory
// layout, then the float W^T used by the constant dot products.
int build_tc(slr_ctx *ctx, const HostLayers<float> &L) {
    ctx->tc_ok = false;
    const slr::NetParams<float> &nf = ctx->nf;
    const int K = nf.K;
    if (K < 2) return fail(ctx, SLR_EUNSUPPORTED, "the tensor-core path needs at least one hidden layer");
    int kmax = 8;
    for (int k = 1; k < K; ++k) {
        if (nf.n[k] > slr::kTcMaxWidth || nf.n[k + 1] > slr::kTcMaxWidth)
            return fail(ctx, SLR_EUNSUPPORTED, "the tensor-core path needs layers and property at most %d wide",
                        slr::kTcMaxWidth);
        // B holds the inputs of layer k and, after the product, its outputs
        kmax = std::max(kmax, std::max((nf.n[k] + 7) & ~7, (nf.n[k + 1] + 7) & ~7));
    }
    slr::TcParams &tp = ctx->tcp;
    std::memset(&tp, 0, sizeof tp);
    tp.sbo = (kmax / 4) * slr::kTcLbo;
    tp.a_bytes = 16 * tp.sbo;
    tp.NCg = 2 * nf.d + 3;
    auto boff = [&](int r, int kk) { return (r / 8) * tp.sbo + (kk / 4) * slr::kTcLbo + (r % 8) * 16 + (kk % 4) * 4; };
    std::vector<size_t> offs(K, 0);
    size_t total = 0;
    for (int k = 1; k < K; ++k) {
        const int n_in = nf.n[k], n_out = nf.n[k + 1], Mpad = (n_out + 7) & ~7;
        const size_t wb = ((size_t)n_in * Mpad * 4 + 15) & ~(size_t)15;
        tp.img_bytes[k] = (int)(2 * (size_t)tp.a_bytes + wb);
        tp.k_pad[k] = (n_in + 7) & ~7;
        tp.img_max = std::max(tp.img_max, tp.img_bytes[k]);
        offs[k] = total;
        total += ((size_t)tp.img_bytes[k] + 255) & ~(size_t)255;
    }
    tp.k_pad[0] = (nf.n[0] + 7) & ~7;
    std::vector<unsigned char> img(total, 0);
    for (int k = 1; k < K; ++k) {
        const int n_in = nf.n[k], n_out = nf.n[k + 1], Mpad = (n_out + 7) & ~7;
        unsigned char *hi = img.data() + offs[k];
        unsigned char *lo = hi + tp.a_bytes;
        float *w = reinterpret_cast<float *>(hi + 2 * tp.a_bytes);
        const std::vector<float> &Wt = L.W[k];   // transposed: [i * n_out + p]
        for (int p = 0; p < n_out; ++p) {
            for (int i = 0; i < n_in; ++i) {
                const float v = Wt[(size_t)i * n_out + p];
                const float h = tf32_host(v);
                const float l = tf32_host(v - h);
                const float ah = std::fabs(h);
                const float al = v >= 0.f ? l : -l;
                std::memcpy(hi + boff(p, i), &h, 4);
                std::memcpy(lo + boff(p, i), &l, 4);
                std::memcpy(hi + boff(64 + p, i), &ah, 4);
                std::memcpy(lo + boff(64 + p, i), &al, 4);
                w[(size_t)i * Mpad + p] = v;
            }
        }
    }
    if (ctx->tc_buf) {
        cudaFree(ctx->tc_buf);
        ctx->tc_buf = nullptr;
    }
    CK(ctx, cudaMalloc(&ctx->tc_buf, total));
    CK(ctx, cudaMemcpy(ctx->tc_buf, img.data(), total, cudaMemcpyHostToDevice));
    ctx->h2d_pending += (int64_t)total;
    for (int k = 1; k < K; ++k) tp.img[k] = (const unsigned char *)ctx->tc_buf + offs[k];
    // the most boxes per CTA whose B operand fits N <= 256 and shared memory
    ctx->T_tc = 0;
    for (int T : slr::kTcTileSizes) {
        slr::TcParams t2 = tp;
        t2.Npad = (tp.NCg * T + 15) & ~15;
        if (t2.Npad > 256) continue;
        t2.b_bytes = (t2.Npad / 8) * tp.sbo;
        const size_t smem = slr::eval_tc_smem_bytes(T, nf, t2);
        if (smem > (size_t)kMaxSmem) continue;
        tp = t2;
        ctx->T_tc = T;
        ctx->smem_tc = smem;
        break;
    }
    if (!ctx->T_tc) return fail(ctx, SLR_EUNSUPPORTED, "no tensor-core tile fits (d=%d)", nf.d);
    tp.idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(tp.Npad >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    ctx->grid_tc = ctx->sm_count * (ctx->smem_tc * 2 <= (size_t)kMaxSmem ? 2 : 1);
    ctx->tc_ok = true;
    return SLR_OK;
}

int ensure_scratch(slr_ctx *ctx, size_t bytes);

// Time every tile choice of the FP32 kernel on a fixed set of boxes (sides 1/16
// of the root box, or of [-0.05, 0.05]^d without one) and keep the fastest.
// The result is kept per network shape, so new weights of the same shape reuse it.
int autotune(slr_ctx *ctx, const std::vector<TileChoice> &cands, TileChoice &best) {
    char key[256];
    int kl = std::snprintf(key, sizeof key, "R%d r%d", (int)ctx->e.size(), ctx->opt.relax_mode);
    for (int w : ctx->widths) kl += std::snprintf(key + kl, sizeof key - kl, " %d", w);
    if (ctx->tuned_key == key) {
        for (const TileChoice &c : cands)
            if (c.T == ctx->tuned_T && c.NT == ctx->tuned_NT) {
                best = c;
                return SLR_OK;
            }
    }
    const int d = ctx->widths[0];
    int64_t n = 16384;
    while (n > 1024 && (size_t)n * d * 8 > ((size_t)64 << 20)) n /= 2;
    const size_t need = align_up((size_t)n * d * 2 * sizeof(float)) + align_up((size_t)n);
    int rc = ensure_scratch(ctx, need);
    if (rc) return rc;
    std::vector<float> h((size_t)n * d * 2);
    uint64_t st = 0x9e3779b97f4a7c15ull;
    auto rnd = [&]() {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        return (double)(st >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int64_t k = 0; k < n; ++k) {
        for (int i = 0; i < d; ++i) {
            double a = -0.05, w = 0.1;
            if (ctx->has_box && (int)ctx->lo.size() == d) {
                a = ctx->lo[i];
                w = (double)ctx->hi[i] - ctx->lo[i];
            }
            const double side = w / 16.0;
            const double lo = a + (w - side) * rnd();
            h[(size_t)k * d + i] = (float)lo;
            h[(size_t)n * d + (size_t)k * d + i] = (float)(lo + side);
        }
    }
    float *dlo = (float *)ctx->scratch;
    float *dhi = dlo + (size_t)n * d;
    uint8_t *dcls = (uint8_t *)ctx->scratch + align_up((size_t)n * d * 2 * sizeof(float));
    CK(ctx, cudaMemcpyAsync(dlo, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    slr::BoxSource src{};
    src.mode = 1;
    src.n_explicit = n;
    src.lo = dlo;
    src.hi = dhi;
    src.cap = n;
    slr::EvalOutputs o{};
    o.cls = dcls;
    if (!ctx->status) {
        CK(ctx, cudaMalloc(&ctx->status, sizeof(unsigned int)));
        CK(ctx, cudaMallocHost(&ctx->h_status, sizeof(unsigned int)));
    }
    o.status = ctx->status;
    float best_ms = 1e30f;
    for (const TileChoice &c : cands) {
        const int grid = (int)std::min<int64_t>((n + c.T - 1) / c.T, (int64_t)c.blocks * ctx->sm_count);
        float ms = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            CK(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
            CK(ctx, slr::launch_eval_f32(c.T, c.NT, grid, c.smem, ctx->stream, ctx->nf, src, o, 0));
            CK(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
            CK(ctx, cudaEventSynchronize(ctx->ev1));
            float t = 0.f;
            cudaEventElapsedTime(&t, ctx->ev0, ctx->ev1);
            if (rep > 0) ms += t;     // the first run warms the caches
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    ctx->tuned_key = key;
    ctx->tuned_T = best.T;
    ctx->tuned_NT = best.NT;
    return SLR_OK;
}

// Wide path: TF32 pieces of W and |W| of every layer k >= 1 (the last one
// folded with the property), zero padded to multiples of 128 rows and 32
// columns, and the chunk size for the per-box state.
int build_wide(slr_ctx *ctx, const HostLayers<float> &L) {
    const slr::NetParams<float> &nf = ctx->nf;
    const int K = nf.K;
    const int d = nf.d;
    int np = 32;
    for (int k = 1; k <= K; ++k) np = std::max(np, (nf.n[k] + 31) & ~31);
    ctx->wide_NP = np;
    std::vector<size_t> offs(K, 0), offs_t(K, 0);
    size_t total = align_up((size_t)d * nf.n[1] * sizeof(float));   // W_1 transposed first
    for (int k = 1; k < K; ++k) {
        const int Mpad = (nf.n[k + 1] + 127) & ~127, Kpad = (nf.n[k] + 31) & ~31;
        ctx->w_Kpad[k] = Kpad;
        offs[k] = total;
        total += 4 * align_up((size_t)Mpad * Kpad * sizeof(float));
        const int MpadT = (nf.n[k] + 127) & ~127, KpadT = (nf.n[k + 1] + 31) & ~31;
        ctx->wt_Kpad[k] = KpadT;
        offs_t[k] = total;
        total += 4 * align_up((size_t)MpadT * KpadT * sizeof(float));
    }
    if (ctx->wide_img) cudaFree(ctx->wide_img);
    ctx->wide_img = nullptr;
    {
        std::vector<unsigned char> host(total, 0);
        float *w0t = (float *)host.data();
        for (int p = 0; p < nf.n[1]; ++p)
            for (int j = 0; j < d; ++j) w0t[(size_t)j * nf.n[1] + p] = L.W[0][(size_t)p * d + j];
        for (int k = 1; k < K; ++k) {
            const int n_in = nf.n[k], n_out = nf.n[k + 1];
            const int Mpad = (n_out + 127) & ~127, Kpad = ctx->w_Kpad[k];
            const size_t one = align_up((size_t)Mpad * Kpad * sizeof(float));
            float *hi = (float *)(host.data() + offs[k]);
            float *lo = (float *)(host.data() + offs[k] + one);
            float *ahi = (float *)(host.data() + offs[k] + 2 * one);
            float *alo = (float *)(host.data() + offs[k] + 3 * one);
            const int KpadT = ctx->wt_Kpad[k];
            const size_t oneT = align_up((size_t)((n_in + 127) & ~127) * KpadT * sizeof(float));
            float *thi = (float *)(host.data() + offs_t[k]);
            float *tlo = (float *)(host.data() + offs_t[k] + oneT);
            float *tahi = (float *)(host.data() + offs_t[k] + 2 * oneT);
            float *talo = (float *)(host.data() + offs_t[k] + 3 * oneT);
            for (int p = 0; p < n_out; ++p) {
                for (int i = 0; i < n_in; ++i) {
                    const float v = L.W[k][(size_t)i * n_out + p];   // transposed float weights
                    const float h = tf32_host(v);
                    const float l = tf32_host(v - h);
                    const size_t o = (size_t)p * Kpad + i;
                    hi[o] = h;
                    lo[o] = l;
                    ahi[o] = std::fabs(h);
                    alo[o] = v >= 0.f ? l : -l;
                    const size_t ot = (size_t)i * KpadT + p;
                    thi[ot] = h;
                    tlo[ot] = l;
                    tahi[ot] = std::fabs(h);
                    talo[ot] = v >= 0.f ? l : -l;
                }
            }
        }
        CK(ctx, cudaMalloc(&ctx->wide_img, total));
        CK(ctx, cudaMemcpy(ctx->wide_img, host.data(), total, cudaMemcpyHostToDevice));
        ctx->h2d_pending += (int64_t)total;
        ctx->w0t = (const float *)ctx->wide_img;
        for (int k = 1; k < K; ++k) {
            const int Mpad = (nf.n[k + 1] + 127) & ~127;
            const size_t one = align_up((size_t)Mpad * ctx->w_Kpad[k] * sizeof(float));
            const unsigned char *b = (const unsigned char *)ctx->wide_img + offs[k];
            ctx->w_hi[k] = (const float *)b;
            ctx->w_lo[k] = (const float *)(b + one);
            ctx->wa_hi[k] = (const float *)(b + 2 * one);
            ctx->wa_lo[k] = (const float *)(b + 3 * one);
            const size_t oneT = align_up((size_t)((nf.n[k] + 127) & ~127) * ctx->wt_Kpad[k] * sizeof(float));
            const unsigned char *bt = (const unsigned char *)ctx->wide_img + offs_t[k];
            ctx->wt_hi[k] = (const float *)bt;
            ctx->wt_lo[k] = (const float *)(bt + oneT);
            ctx->wta_hi[k] = (const float *)(bt + 2 * oneT);
            ctx->wta_lo[k] = (const float *)(bt + 3 * oneT);
        }
    }
    // chunk: the boxes whose state fits about 3 GB
    const int R = nf.R;
    const size_t per_box = sizeof(float) * ((size_t)np * (2 * (size_t)d + 2 * (size_t)(d + 3) + 5) + 3 * (size_t)d +
                                            3 * (size_t)R) + sizeof(int64_t) + 64;
    int64_t bc = (int64_t)(((size_t)3 << 30) / per_box);
    bc = std::max<int64_t>(1, std::min<int64_t>(bc, 8192));
    while (bc > 1 && (int64_t)bc * (d + 3) > ((int64_t)1 << 30)) bc /= 2;
    ctx->wide_Bc = (int)bc;
    return SLR_OK;
}

int ensure_wide_buf(slr_ctx *ctx) {
    const int d = ctx->nf.d, np = ctx->wide_NP, R = ctx->nf.R;
    const size_t bc = (size_t)ctx->wide_Bc;
    const size_t need = 2 * align_up(bc * d * np * 4) + 2 * align_up(bc * (d + 3) * np * 4) + 5 * align_up(bc * np * 4) +
                        3 * align_up(bc * d * 4) + 3 * align_up(bc * R * 4) + align_up(bc * 8);
    if (ctx->wide_buf_bytes >= need) return SLR_OK;
    cudaFree(ctx->wide_buf);
    ctx->wide_buf = nullptr;
    ctx->wide_buf_bytes = 0;
    CK(ctx, cudaMalloc(&ctx->wide_buf, need));
    CK(ctx, cudaMemsetAsync(ctx->wide_buf, 0, need, ctx->stream));
    ctx->wide_buf_bytes = need;
    return SLR_OK;
}

// Bound positions [0, n) of `src` on the wide path, chunk by chunk.
int run_wide(slr_ctx *ctx, const slr::BoxSource &src, int64_t n, const slr::EvalOutputs &out, int64_t *launches) {
    int rc = ensure_wide_buf(ctx);
    if (rc) return rc;
    const slr::NetParams<float> &nf = ctx->nf;
    const int K = nf.K, d = nf.d, np = ctx->wide_NP, R = nf.R, sms = ctx->sm_count;
    const size_t bc = (size_t)ctx->wide_Bc;
    unsigned char *p = (unsigned char *)ctx->wide_buf;
    auto take = [&](size_t bytes) {
        float *q = (float *)p;
        p += align_up(bytes);
        return q;
    };
    float *Cb[2] = {take(bc * d * np * 4), take(bc * d * np * 4)};
    float *Rb[2] = {take(bc * (d + 3) * np * 4), take(bc * (d + 3) * np * 4)};
    float *Ch = take(bc * np * 4), *Cl = take(bc * np * 4);
    float *Kh = take(bc * np * 4), *Kl = take(bc * np * 4), *Ke = take(bc * np * 4);
    float *mh = take(bc * d * 4), *ml = take(bc * d * 4), *rr = take(bc * d * 4);
    float *lo = take(bc * R * 4), *hi = take(bc * R * 4), *er = take(bc * R * 4);
    int64_t *bidx = (int64_t *)take(bc * 8);
    for (int64_t base = 0; base < n; base += (int64_t)bc) {
        const int nb = (int)std::min<int64_t>((int64_t)bc, n - base);
        CK(ctx, slr::launch_wide_box(src, base, nb, d, mh, ml, rr, bidx, sms, ctx->stream));
        int cur = 0;
        CK(ctx, slr::launch_wide_init(nf, ctx->w0t, nb, np, mh, ml, rr, Cb[cur], Rb[cur], Ch, Cl, src.alpha,
                                      src.alpha_ld, base, ctx->stream));
        *launches += 2;
        for (int k = 1; k < K; ++k) {
            const int nxt = cur ^ 1;
            if (k + 1 == K && nf.R <= 16) {
                // the property layer: a few rows, on the CUDA cores (FP32 FMA
                // chains, rounding bound gamma_{n_in} like the tile kernel's)
                CK(ctx, slr::launch_wide_rows_product(nf.Wt[k], nf.n[k], nf.R, Cb[cur], np, Cb[nxt], np,
                                                      (int64_t)nb * d, false, sms, ctx->stream));
                CK(ctx, slr::launch_wide_rows_product(nf.Wt[k], nf.n[k], nf.R, Rb[cur], np, Rb[nxt], np,
                                                      (int64_t)nb * (d + 3), true, sms, ctx->stream));
                CK(ctx, slr::launch_wide_const(nf, k, nb, np, Ch, Cl, Rb[cur], Kh, Kl, Ke, sms, ctx->stream));
                const float gf = (float)(nf.n[k] + 2) * 0x1p-24f;
                CK(ctx, slr::launch_wide_final(nf, nb, np, gf, Cb[nxt], Rb[nxt], Ch, Cl, Kh, Kl, Ke, lo, hi, er,
                                               ctx->stream));
                *launches += 4;
                cur = nxt;
                continue;
            }
            slr::WideGemmArgs ga{};
            ga.status = out.status;
            ga.g[0] = slr::WideGemm{ctx->w_hi[k], ctx->w_lo[k], Cb[cur], Cb[nxt], nf.n[k + 1], nf.n[k], ctx->w_Kpad[k],
                                    nb * d, np, np};
            ga.g[1] = slr::WideGemm{ctx->wa_hi[k], ctx->wa_lo[k], Rb[cur], Rb[nxt], nf.n[k + 1], nf.n[k],
                                    ctx->w_Kpad[k], nb * (d + 3), np, np};
            const bool prof = ctx->opt.profile != 0;
            if (prof) {
                while (ctx->gemm_ev.size() < ctx->gemm_ev_used + 2) {
                    cudaEvent_t e;
                    CK(ctx, cudaEventCreate(&e));
                    ctx->gemm_ev.push_back(e);
                }
                CK(ctx, cudaEventRecord(ctx->gemm_ev[ctx->gemm_ev_used], ctx->stream));
            }
            CK(ctx, slr::launch_wide_gemm(ga, 2, ctx->stream));
            if (prof) {
                CK(ctx, cudaEventRecord(ctx->gemm_ev[ctx->gemm_ev_used + 1], ctx->stream));
                ctx->gemm_ev_used += 2;
            }
            ctx->gemm_launches += 1;
            ctx->gemm_flop += 2.0 * nf.n[k + 1] * nf.n[k] * ((double)nb * (2 * d + 1));
            CK(ctx, slr::launch_wide_const(nf, k, nb, np, Ch, Cl, Rb[cur], Kh, Kl, Ke, sms, ctx->stream));
            const float g = slr::tc_gamma(ctx->w_Kpad[k]);
            if (k + 1 < K) {
                CK(ctx, slr::launch_wide_hidden(nf, k + 1, nb, np, g, Cb[nxt], Rb[nxt], Ch, Cl, Kh, Kl, Ke, src.alpha,
                                                src.alpha_ld, base, ctx->stream));
            } else {
                CK(ctx, slr::launch_wide_final(nf, nb, np, g, Cb[nxt], Rb[nxt], Ch, Cl, Kh, Kl, Ke, lo, hi, er,
                                               ctx->stream));
            }
            *launches += 3;
            cur = nxt;
        }
        if (K == 1) {
            CK(ctx, slr::launch_wide_final(nf, nb, np, 0.f, Cb[cur], Rb[cur], Ch, Cl, Kh, Kl, Ke, lo, hi, er,
                                           ctx->stream));
            *launches += 1;
        }
        CK(ctx, slr::launch_wide_classify(nf, nb, base, lo, hi, er, bidx, out, sms, ctx->stream));
        *launches += 1;
    }
    return SLR_OK;
}

// The adjoint on the wide path for positions [0, n) of a.src (the device count
// when a.count is set): per chunk, the forward products keeping each hidden
// layer's pre-activation equations, the rows and their adjoints, the backward
// products through W^T and |W|^T with the relaxations between them, and the
// box gradient and split choice.
int run_wide_adjoint(slr_ctx *ctx, const slr::AdjArgs &a, int64_t *launches) {
    const slr::NetParams<float> &nf = ctx->nf;
    const int K = nf.K, d = nf.d, Q = d + 1, np = ctx->wide_NP, sms = ctx->sm_count;
    int64_t n = a.n;
    if (a.count != nullptr) {
        unsigned long long c = 0;
        CK(ctx, cudaMemcpyAsync(&c, a.count, sizeof c, cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        n = std::min<int64_t>(n, (int64_t)c);
    }
    if (n <= 0) return SLR_OK;
    // chunk: the boxes whose state fits about 6 GB
    const size_t eq = (size_t)Q * np;
    const size_t per_box = sizeof(float) * (eq * (size_t)(2 * (K - 1) - 1 + 6) + 5 * (size_t)(K - 1) * np +
                                            3 * (size_t)d) + 64 * 16;
    const int64_t bc = std::max<int64_t>(1, std::min<int64_t>(4096, (int64_t)(((size_t)6 << 30) / per_box)));
    const size_t need = per_box * (size_t)bc + ((size_t)64 << 10);
    if (ctx->wadj_bytes < need) {
        cudaFree(ctx->wadj_buf);
        ctx->wadj_buf = nullptr;
        ctx->wadj_bytes = 0;
        CK(ctx, cudaMalloc(&ctx->wadj_buf, need));
        ctx->wadj_bytes = need;
    }
    unsigned char *p = (unsigned char *)ctx->wadj_buf;
    auto take = [&](size_t floats) {
        float *q = (float *)p;
        p += align_up(floats * sizeof(float));
        return q;
    };
    float *m = take((size_t)bc * d), *r = take((size_t)bc * d), *gr = take((size_t)bc * d);
    float *Cl[slr::kMaxLayers] = {}, *Rl[slr::kMaxLayers] = {};
    for (int k = 1; k < K; ++k) {
        Cl[k] = take((size_t)bc * eq);
        Rl[k] = k > 1 ? take((size_t)bc * eq) : nullptr;   // layer 1: U = L
    }
    float *Cf = take((size_t)bc * eq), *Rf = take((size_t)bc * eq);
    float *Pc = take((size_t)bc * eq), *Pr = take((size_t)bc * eq);
    float *gC = take((size_t)bc * eq), *gR = take((size_t)bc * eq);
    const int64_t sstride = bc * np;
    float *sc = take((size_t)5 * (K - 1) * sstride);
    for (int64_t pos0 = 0; pos0 < n; pos0 += bc) {
        const int nb = (int)std::min<int64_t>(bc, n - pos0);
        CK(ctx, slr::launch_wadj_box(a.src, pos0, nb, d, m, r, sms, ctx->stream));
        CK(ctx, slr::launch_wadj_layer1(nf, ctx->w0t, nb, np, m, r, Cl[1], ctx->stream));
        *launches += 2;
        for (int k = 1; k < K; ++k) {
            float *sck = sc + (size_t)(k - 1) * 5 * sstride;
            CK(ctx, slr::launch_wadj_fwd(a, k, pos0, nb, np, Cl[k], Rl[k], k > 1 ? nf.b[k - 1] : nullptr, sck,
                                         sstride, Pc, Pr, ctx->stream));
            float *oc = k + 1 < K ? Cl[k + 1] : Cf, *orr = k + 1 < K ? Rl[k + 1] : Rf;
            if (k + 1 == K && nf.R <= 16) {
                // the property layer's few rows on the CUDA cores
                CK(ctx, slr::launch_wide_rows_product(nf.Wt[k], nf.n[k], nf.R, Pc, np, oc, np, (int64_t)nb * Q, false,
                                                      sms, ctx->stream));
                CK(ctx, slr::launch_wide_rows_product(nf.Wt[k], nf.n[k], nf.R, Pr, np, orr, np, (int64_t)nb * Q, true,
                                                      sms, ctx->stream));
                *launches += 3;
                continue;
            }
            slr::WideGemmArgs ga{};
            ga.status = ctx->status;
            ga.g[0] = slr::WideGemm{ctx->w_hi[k], ctx->w_lo[k], Pc, oc, nf.n[k + 1], nf.n[k], ctx->w_Kpad[k],
                                    nb * Q, np, np};
            ga.g[1] = slr::WideGemm{ctx->wa_hi[k], ctx->wa_lo[k], Pr, orr, nf.n[k + 1], nf.n[k], ctx->w_Kpad[k],
                                    nb * Q, np, np};
            CK(ctx, slr::launch_wide_gemm(ga, 2, ctx->stream));
            *launches += 2;
        }
        CK(ctx, slr::launch_wadj_rows(a, pos0, nb, np, Cf, Rf, nf.b[K - 1], gC, gR, ctx->stream));
        *launches += 1;
        for (int k = K - 1; k >= 1; --k) {
            slr::WideGemmArgs ga{};
            ga.status = ctx->status;
            ga.g[0] = slr::WideGemm{ctx->wt_hi[k], ctx->wt_lo[k], gC, Pc, nf.n[k], nf.n[k + 1], ctx->wt_Kpad[k],
                                    nb * Q, np, np};
            ga.g[1] = slr::WideGemm{ctx->wta_hi[k], ctx->wta_lo[k], gR, Pr, nf.n[k], nf.n[k + 1], ctx->wt_Kpad[k],
                                    nb * Q, np, np};
            CK(ctx, slr::launch_wide_gemm(ga, 2, ctx->stream));
            const float *sck = sc + (size_t)(k - 1) * 5 * sstride;
            CK(ctx, slr::launch_wadj_bwd(a, k, pos0, nb, np, Cl[k], Rl[k], sck, sstride, Pc, Pr, gC,
                                         k > 1 ? gR : nullptr, ctx->stream));
            *launches += 2;
        }
        if (a.d_lo != nullptr || a.d_r != nullptr || a.split_codes != nullptr) {
            CK(ctx, slr::launch_wadj_boxgrad(a, pos0, nb, np, ctx->w0t, gC, gr, sms, ctx->stream));
            *launches += 1;
            if (a.split_codes != nullptr) {
                CK(ctx, slr::launch_wadj_split(a, pos0, nb, gr, r, sms, ctx->stream));
                *launches += 1;
            }
        }
    }
    return SLR_OK;
}

// The adjoint of `a`: on the wide path by per-layer products (no weight
// gradients there), else the one-box-per-CTA kernel.
int run_adjoint(slr_ctx *ctx, const slr::AdjArgs &a, int grid, int64_t *launches) {
    bool weights = false;
    for (int k = 0; k < ctx->nf.K; ++k) weights = weights || a.dW[k] != nullptr || a.db[k] != nullptr;
    if (ctx->wide && ctx->nf.K > 1 && !weights) return run_wide_adjoint(ctx, a, launches);
    CK(ctx, slr::launch_adjoint(a, grid, ctx->stream));
    *launches += 1;
    return SLR_OK;
}

// FP64 re-check of a list of boxes at level t: on clusters where chosen (pass
// 1); else, with recheck_pairs, the float-float stage (pass 2) lists the
// boxes it leaves depending on E in the other re-check list, and pass 1
// re-bounds those with plain FP64 products.  Returns the launches in *n.
cudaError_t launch_recheck(slr_ctx *ctx, const slr::BoxSource &src, const slr::EvalOutputs &out, int t,
                           int64_t *n) {
    *n = 1;
    if (ctx->grid64c > 0)
        return slr::launch_eval_f64_cluster(ctx->T64, ctx->grid64c, ctx->smem64, ctx->stream, ctx->nd, src, out, 1);
    if (ctx->opt.recheck_pairs && ctx->pairs_fit) {
        int64_t *rest = src.index == ctx->near_list ? ctx->near_list2 : ctx->near_list;
        slr::EvalOutputs oa = out;
        oa.near_list = rest;
        oa.near_count = &ctx->ctr->near3_n[t];
        oa.near_cap = ctx->near_cap;
        oa.tie_count = nullptr;
        cudaError_t e =
            slr::launch_eval_f64(ctx->T64, ctx->NT64, ctx->grid64, ctx->smem64, ctx->stream, ctx->nd, src, oa, 2);
        if (e != cudaSuccess) return e;
        slr::BoxSource sb = src;
        sb.index = rest;
        sb.index_count = &ctx->ctr->near3_n[t];
        sb.cap = ctx->near_cap;
        *n = 2;
        return slr::launch_eval_f64(ctx->T64, ctx->NT64, ctx->grid64, ctx->smem64, ctx->stream, ctx->nd, sb, out, 1);
    }
    return slr::launch_eval_f64(ctx->T64, ctx->NT64, ctx->grid64, ctx->smem64, ctx->stream, ctx->nd, src, out, 1);
}

// FP64 re-check: short lists, so the smallest tiles spread them over the
// most SMs, with the most threads (a tile's products then split their inputs
// over lane pairs: the per-level latency is what counts).  T64 = 0 when no
// FP64 tile holds the network.  The footprint includes the float-float
// stage's planes where some tile holds them (pairs_fit), else not.
std::vector<TileChoice> recheck_candidates(slr_ctx *ctx, bool pairs) {
    std::vector<TileChoice> c64 = tile_candidates(ctx->nd, pairs);
    if (slr::eval_f64_pair_tile_ok(ctx->nd.d)) {
        TileChoice c;
        c.T = 2;
        c.NT = 256;
        c.smem = slr::eval_smem_bytes<double>(2, ctx->nd.d, ctx->nd.R, ctx->nd.n_max_pad, ctx->nd.n_in_max, pairs);
        if (c.smem <= (size_t)kMaxSmem && slr::eval_gemm_items(2, ctx->nd.d, ctx->nd.n_max_pad) <= 2 * 256) {
            c.blocks = slr::eval_blocks_per_sm_f64(2, 256, c.smem);
            if (c.blocks > 0) c64.push_back(c);
        }
    }
    return c64;
}

void choose_recheck_tile(slr_ctx *ctx) {
    std::vector<TileChoice> c64 = recheck_candidates(ctx, true);
    ctx->pairs_fit = !c64.empty();
    if (!ctx->pairs_fit) c64 = recheck_candidates(ctx, false);
    ctx->T64 = 0;
    for (const TileChoice &c : c64) {
        if (ctx->T64 == 0 || c.T < ctx->T64 || (c.T == ctx->T64 && c.NT > ctx->NT64)) {
            ctx->T64 = c.T;
            ctx->NT64 = c.NT;
            ctx->smem64 = c.smem;
            ctx->grid64 = c.blocks * ctx->sm_count;
        }
    }
    // on request, the same tile on a cluster of CTAs (products dealt over their
    // SMs) where the GPU runs such clusters
    ctx->grid64c = 0;
    if (ctx->T64 > 0 && ctx->T64 <= 4 && ctx->NT64 == 256 && ctx->opt.recheck_cluster == 1 &&
        slr::eval_gemm_items(ctx->T64, ctx->nd.d, ctx->nd.n_max_pad) <= slr::kRecheckCluster * 256) {
        const int nc = slr::eval_f64_cluster_max(ctx->T64, ctx->smem64);
        if (nc > 0) ctx->grid64c = nc * slr::kRecheckCluster;
    }
}

int prepare_device(slr_ctx *ctx) {
    if (!ctx->dev_dirty) return SLR_OK;
    if (ctx->widths.back() != (int)(ctx->C.size() / std::max<size_t>(1, ctx->e.size())))
        return fail(ctx, SLR_EINVAL, "property has %zu outputs per row but the network has %d outputs",
                    ctx->C.size() / std::max<size_t>(1, ctx->e.size()), ctx->widths.back());
    HostLayers<float> Lf;
    HostLayers<double> Ld;
    build_layers(ctx, Lf);
    build_layers(ctx, Ld);
    const size_t c_bytes = align_up(ctx->C.size() * sizeof(float));
    const size_t bytes = layers_bytes(Lf) + layers_bytes(Ld) + c_bytes;
    if (ctx->net_buf) {
        cudaFree(ctx->net_buf);
        ctx->net_buf = nullptr;
    }
    CK(ctx, cudaMalloc(&ctx->net_buf, bytes));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    int rc = ensure_stage(ctx, bytes);
    if (rc) return rc;
    std::memset(ctx->h_stage, 0, bytes);
    size_t off = 0;
    layout_params(ctx, Lf, (unsigned char *)ctx->net_buf, ctx->h_stage, off, ctx->nf);
    layout_params(ctx, Ld, (unsigned char *)ctx->net_buf, ctx->h_stage, off, ctx->nd);
    for (int k = 1; k + 1 < ctx->K; ++k) ctx->nd.Wsf[k] = ctx->nf.Ws[k];
    std::memcpy(ctx->h_stage + off, ctx->C.data(), ctx->C.size() * sizeof(float));
    ctx->dC = reinterpret_cast<const float *>((unsigned char *)ctx->net_buf + off);
    off += c_bytes;
    CK(ctx, cudaMemcpyAsync(ctx->net_buf, ctx->h_stage, bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->h2d_pending += (int64_t)bytes;
    (void)rc;
    const std::vector<TileChoice> c32 = tile_candidates(ctx->nf);
    ctx->wide = ctx->opt.wide != 0 || c32.empty();
    if (ctx->wide) {
        if ((rc = build_wide(ctx, Lf))) return rc;
        ctx->T32 = ctx->NT32 = 0;
        // the FP64 re-check of the wide path's NEAR boxes runs the FP64 tile
        // kernel where the network fits it (none for the widest networks)
        choose_recheck_tile(ctx);
        ctx->tc_ok = false;
        ctx->H = 0;
        for (int k = 1; k < ctx->K; ++k) ctx->H += ctx->widths[k];
        // adjoint: one box per CTA, every hidden layer kept, state in global
        // memory (up to about 4 GB of CTA slots)
        slr::AdjArgs a{};
        a.net = ctx->nf;
        a.H = ctx->H;
        a.n_max = 0;
        for (int k = 1; k <= ctx->K; ++k) a.n_max = std::max(a.n_max, ctx->nf.n[k]);
        a.nck = ctx->K - 1;
        a.boxes_per_cta = 1;
        const size_t box = slr::adjoint_box_bytes(a);
        ctx->adj_nmax = a.n_max;
        ctx->adj_nck = a.nck;
        ctx->adj_boxes = 1;
        ctx->adj_smem = 0;
        ctx->adj_gmem = true;
        ctx->adj_grid = (int)std::max<size_t>(1, std::min<size_t>((size_t)2 * ctx->sm_count, ((size_t)4 << 30) / box));
        ctx->dev_dirty = false;
        return SLR_OK;
    }
    TileChoice best = c32[0];
    if (ctx->opt.tile_boxes > 0) {
        bool found = false;
        for (const TileChoice &c : c32)
            if (c.T == ctx->opt.tile_boxes && c.NT == ctx->opt.tile_threads) {
                best = c;
                found = true;
            }
        if (!found)
            return fail(ctx, SLR_EUNSUPPORTED, "tile %d x %d is not available for this network", ctx->opt.tile_boxes,
                        ctx->opt.tile_threads);
    } else if (c32.size() > 1) {
        if ((rc = autotune(ctx, c32, best))) return rc;
    }
    ctx->T32 = best.T;
    ctx->NT32 = best.NT;
    ctx->smem32 = best.smem;
    ctx->grid32 = best.blocks * ctx->sm_count;
    choose_recheck_tile(ctx);
    // adjoint: keep as many hidden layers' equations in shared memory as fit in
    // 96 KB, recompute the others
    {
        slr::AdjArgs a{};
        a.net = ctx->nf;
        a.H = 0;
        for (int k = 1; k < ctx->K; ++k) a.H += ctx->widths[k];
        a.n_max = 0;
        for (int k = 1; k <= ctx->K; ++k) a.n_max = std::max(a.n_max, ctx->nf.n[k]);
        // keep as many hidden layers' equations as fit 96 KB for one box, then
        // put as many boxes in a CTA as fit about 110 KB (at most 8)
        a.boxes_per_cta = 1;
        a.nck = 0;
        while (a.nck < ctx->K - 1) {
            a.nck += 1;
            if (slr::adjoint_smem_bytes(a) > 96 * 1024) {
                a.nck -= 1;
                break;
            }
        }
        const size_t one = slr::adjoint_smem_bytes(a);
        a.boxes_per_cta = (int)std::max<size_t>(1, std::min<size_t>(8, (size_t)(110 * 1024) / std::max<size_t>(1, one)));
        ctx->H = a.H;
        ctx->adj_nmax = a.n_max;
        ctx->adj_nck = a.nck;
        ctx->adj_boxes = a.boxes_per_cta;
        ctx->adj_gmem = false;
        ctx->adj_smem = slr::adjoint_smem_bytes(a);
        const int nb = ctx->adj_smem <= (size_t)kMaxSmem ? slr::adjoint_blocks_per_sm(ctx->adj_smem) : 0;
        ctx->adj_grid = nb * ctx->sm_count;
    }
    if (ctx->opt.precision == SLR_PREC_TC_TF32) {
        if ((rc = build_tc(ctx, Lf))) return rc;
    } else {
        ctx->tc_ok = false;
    }
    ctx->dev_dirty = false;
    return SLR_OK;
}

int ensure_scratch(slr_ctx *ctx, size_t bytes) {
    if (ctx->scratch_bytes >= bytes) return SLR_OK;
    if (ctx->scratch) cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    CK(ctx, cudaMalloc(&ctx->scratch, bytes));
    ctx->scratch_bytes = bytes;
    return SLR_OK;
}

void free_count_buffers(slr_ctx *ctx) {
    cudaFree(ctx->codes[0]);
    cudaFree(ctx->codes[1]);
    cudaFree(ctx->cls);
    cudaFree(ctx->near_list);
    cudaFree(ctx->near_list2);
    ctx->codes[0] = ctx->codes[1] = nullptr;
    ctx->cls = nullptr;
    ctx->near_list = nullptr;
    ctx->near_list2 = nullptr;
    ctx->cap = 0;
}

int ensure_count_buffers(slr_ctx *ctx) {
    const int64_t cap = ctx->opt.frontier_cap;
    if (ctx->cap != cap) {
        free_count_buffers(ctx);
        CK(ctx, cudaMalloc(&ctx->codes[0], (size_t)cap * sizeof(uint64_t)));
        CK(ctx, cudaMalloc(&ctx->codes[1], (size_t)cap * sizeof(uint64_t)));
        CK(ctx, cudaMalloc(&ctx->cls, (size_t)cap));
        ctx->near_cap = std::max<int64_t>(1024, cap / 4);
        CK(ctx, cudaMalloc(&ctx->near_list, (size_t)ctx->near_cap * sizeof(int64_t)));
        CK(ctx, cudaMalloc(&ctx->near_list2, (size_t)ctx->near_cap * sizeof(int64_t)));
        ctx->cap = cap;
    }
    if (!ctx->ctr) {
        CK(ctx, cudaMalloc(&ctx->ctr, sizeof(slr::LevelCounters)));
        CK(ctx, cudaMalloc(&ctx->status, sizeof(unsigned int)));
        CK(ctx, cudaMallocHost(&ctx->h_ctr, sizeof(slr::LevelCounters)));
        CK(ctx, cudaMallocHost(&ctx->h_status, sizeof(unsigned int)));
    }
    const int d = ctx->widths[0];
    if (ctx->root_d != d) {
        cudaFree(ctx->root);
        cudaFree(ctx->masks);
        ctx->root = nullptr;
        ctx->masks = nullptr;
        CK(ctx, cudaMalloc(&ctx->root, 2 * (size_t)d * sizeof(double)));
        CK(ctx, cudaMalloc(&ctx->masks, (size_t)d * sizeof(unsigned long long)));
        ctx->root_d = d;
    }
    if (ctx->opt.record_leaves && ctx->leaf_cap_alloc != ctx->opt.leaf_cap) {
        cudaFree(ctx->leaf_codes);
        cudaFree(ctx->leaf_depth);
        cudaFree(ctx->leaf_cls);
        ctx->leaf_codes = nullptr;
        ctx->leaf_depth = ctx->leaf_cls = nullptr;
        ctx->leaf_cap_alloc = 0;
        const size_t lc = (size_t)ctx->opt.leaf_cap;
        CK(ctx, cudaMalloc(&ctx->leaf_codes, lc * sizeof(uint64_t)));
        CK(ctx, cudaMalloc(&ctx->leaf_depth, lc));
        CK(ctx, cudaMalloc(&ctx->leaf_cls, lc));
        ctx->leaf_cap_alloc = ctx->opt.leaf_cap;
    }
    return SLR_OK;
}

int check_boxes(slr_ctx *ctx, int64_t n, int d, const float *box_lo, const float *box_hi) {
    for (int64_t k = 0; k < n * d; ++k) {
        if (!std::isfinite(box_lo[k]) || !std::isfinite(box_hi[k]) || box_lo[k] > box_hi[k])
            return fail(ctx, SLR_EINVAL, "box %lld: bad endpoints in dimension %d", (long long)(k / d), (int)(k % d));
    }
    return SLR_OK;
}

int check_ready(slr_ctx *ctx) {
    if (!ctx) return fail(nullptr, SLR_EINVAL, "null context");
    if (!ctx->has_net || !ctx->has_box || !ctx->has_prop)
        return fail(ctx, SLR_ESTATE, "network, box and property must be set before counting");
    if ((int)ctx->lo.size() != ctx->widths[0])
        return fail(ctx, SLR_EINVAL, "box has %zu dimensions but the network has %d inputs", ctx->lo.size(),
                    ctx->widths[0]);
    return SLR_OK;
}

}  // namespace

int slr_internal_noalloc_view(slr_ctx *ctx, slr_noalloc_view *v) {
    if (!ctx) return fail(nullptr, SLR_EINVAL, "null context");
    if (!ctx->has_net || !ctx->has_box || !ctx->has_prop)
        return fail(ctx, SLR_ESTATE, "network, box and property must be set before counting");
    if ((int)ctx->lo.size() != ctx->widths[0])
        return fail(ctx, SLR_EINVAL, "box has %zu dimensions but the network has %d inputs", ctx->lo.size(),
                    ctx->widths[0]);
    if (ctx->dev_dirty || !ctx->net_buf)
        return fail(ctx, SLR_ESTATE,
                    "slr_count_noalloc needs the network and property on the device: call slr_count (or "
                    "slr_bounds with n >= 1) once after setting them");
    if (ctx->wide) return fail(ctx, SLR_EUNSUPPORTED, "slr_count_noalloc does not run the wide path");
    if (ctx->opt.split_rule != SLR_SPLIT_WIDEST)
        return fail(ctx, SLR_EUNSUPPORTED, "slr_count_noalloc splits the widest side only");
    if (ctx->opt.shard_count > 1) return fail(ctx, SLR_EUNSUPPORTED, "slr_count_noalloc does not shard");
    // options whose count differs from the fixed-slope FP32 tile path it runs
    if (ctx->opt.alpha_steps > 0)
        return fail(ctx, SLR_EUNSUPPORTED, "slr_count_noalloc counts with fixed slopes only (alpha_steps > 0)");
    if (ctx->opt.precision != SLR_PREC_FP32)
        return fail(ctx, SLR_EUNSUPPORTED, "slr_count_noalloc runs the FP32 contraction only (precision != FP32)");
    if (ctx->opt.recheck_cluster != 0)
        return fail(ctx, SLR_EUNSUPPORTED, "slr_count_noalloc re-checks each tile on one CTA (recheck_cluster)");
    v->device = ctx->device;
    v->stream = ctx->stream;
    v->d = ctx->widths[0];
    v->T32 = ctx->T32;
    v->NT32 = ctx->NT32;
    v->grid32 = ctx->grid32;
    v->T64 = ctx->T64;
    v->NT64 = ctx->NT64;
    v->grid64 = ctx->grid64;
    v->sm_count = ctx->sm_count;
    v->smem32 = ctx->smem32;
    v->smem64 = ctx->smem64;
    v->nf = &ctx->nf;
    v->nd = &ctx->nd;
    v->lo = ctx->lo.data();
    v->hi = ctx->hi.data();
    v->fp64_recheck = ctx->opt.fp64_recheck;
    v->ev0 = ctx->ev0;
    v->ev1 = ctx->ev1;
    return SLR_OK;
}

int slr_internal_fail(slr_ctx *ctx, int code, const char *msg) { return fail(ctx, code, "%s", msg); }

int slr_internal_alpha_level(slr_ctx *ctx, const slr::BoxSource &frontier, int t, int64_t *launches);
int slr_internal_split_root(slr_ctx *ctx, const slr::BoxSource &root, int64_t *launches);
int slr_internal_split_level(slr_ctx *ctx, const slr::BoxSource &frontier, int t, bool slopes, int64_t *launches);
namespace {
int check_adjoint(slr_ctx *ctx);
}

extern "C" {

void slr_default_options(slr_options *opt) {
    if (!opt) return;
    opt->precision = SLR_PREC_FP32;
    opt->relax_mode = SLR_RELAX_NEURIFY;
    opt->fp64_recheck = 1;
    opt->record_leaves = 0;
    opt->profile = 0;
    opt->split_rule = SLR_SPLIT_WIDEST;
    opt->frontier_cap = (int64_t)1 << 24;
    opt->leaf_cap = (int64_t)1 << 22;
    opt->alpha_steps = 0;
    opt->alpha_lr = 0.1f;
    opt->alpha_cap = (int64_t)1 << 16;
    opt->alpha_margin = 0.2f;
    opt->recheck_pairs = 1;
    opt->tile_boxes = 0;
    opt->tile_threads = 0;
    opt->wide = 0;
    opt->shard_count = 1;
    opt->shard_index = 0;
    opt->shard_level = 0;
    opt->recheck_cluster = 0;
}

int slr_create(slr_ctx **out, int device, void *cuda_stream) {
    if (!out) return fail(nullptr, SLR_EINVAL, "out is NULL");
    *out = nullptr;
    int n_dev = 0;
    cudaError_t e = cudaGetDeviceCount(&n_dev);
    if (e != cudaSuccess) return fail(nullptr, SLR_ECUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
    if (device < 0 || device >= n_dev) return fail(nullptr, SLR_EINVAL, "device %d out of range (%d devices)", device, n_dev);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(nullptr, SLR_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    slr_ctx *ctx = new (std::nothrow) slr_ctx();
    if (!ctx) return fail(nullptr, SLR_ENOMEM, "host allocation failed");
    ctx->device = device;
    slr_default_options(&ctx->opt);
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete ctx;
            return fail(nullptr, SLR_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        }
        ctx->own_stream = true;
    }
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    cudaEventCreate(&ctx->ev0);
    cudaEventCreate(&ctx->ev1);
    *out = ctx;
    return SLR_OK;
}

int slr_destroy(slr_ctx *ctx) {
    if (!ctx) return SLR_OK;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_count_buffers(ctx);
    cudaFree(ctx->net_buf);
    cudaFree(ctx->tc_buf);
    cudaFree(ctx->ctr);
    cudaFree(ctx->status);
    cudaFree(ctx->root);
    cudaFree(ctx->masks);
    cudaFree(ctx->leaf_codes);
    cudaFree(ctx->leaf_depth);
    cudaFree(ctx->leaf_cls);
    cudaFree(ctx->scratch);
    cudaFree(ctx->alpha_buf);
    cudaFree(ctx->alpha_ctr);
    cudaFree(ctx->wide_img);
    cudaFree(ctx->wide_buf);
    cudaFree(ctx->adj_scratch);
    for (slr_ctx *h : ctx->wide_helpers) slr_destroy(h);
    cudaFree(ctx->split_buf);
    cudaFree(ctx->wadj_buf);
    cudaFree(ctx->approx_buf);
    if (ctx->count_graph) cudaGraphExecDestroy(ctx->count_graph);
    if (ctx->h_ctr) cudaFreeHost(ctx->h_ctr);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->gemm_ev) cudaEventDestroy(e);
    if (ctx->batch) {
        if (ctx->batch->graph) cudaGraphExecDestroy(ctx->batch->graph);
        cudaFree(ctx->batch->arena);
        if (ctx->batch->h_upload) cudaFreeHost(ctx->batch->h_upload);
        if (ctx->batch->h_ctrs) cudaFreeHost(ctx->batch->h_ctrs);
        delete ctx->batch;
    }
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return SLR_OK;
}

int slr_set_options(slr_ctx *ctx, const slr_options *opt) {
    if (!ctx || !opt) return fail(ctx, SLR_EINVAL, "null argument");
    if (opt->precision != SLR_PREC_FP32 && opt->precision != SLR_PREC_TC_TF32)
        return fail(ctx, SLR_EINVAL, "precision %d unknown", opt->precision);
    if (opt->relax_mode != SLR_RELAX_NEURIFY && opt->relax_mode != SLR_RELAX_PAPER_LITERAL &&
        opt->relax_mode != SLR_RELAX_INTERVAL)
        return fail(ctx, SLR_EINVAL, "relax_mode %d unknown", opt->relax_mode);
    if (opt->frontier_cap < 2 || opt->frontier_cap > ((int64_t)1 << 34))
        return fail(ctx, SLR_EINVAL, "frontier_cap %lld out of range", (long long)opt->frontier_cap);
    if (opt->split_rule != SLR_SPLIT_WIDEST && opt->split_rule != SLR_SPLIT_GRADIENT)
        return fail(ctx, SLR_EINVAL, "split_rule must be SLR_SPLIT_WIDEST or SLR_SPLIT_GRADIENT");
    if (opt->record_leaves && (opt->leaf_cap < 1 || opt->leaf_cap > ((int64_t)1 << 34)))
        return fail(ctx, SLR_EINVAL, "leaf_cap %lld out of range", (long long)opt->leaf_cap);
    if (opt->alpha_steps < 0 || opt->alpha_steps > 1000)
        return fail(ctx, SLR_EINVAL, "alpha_steps %d out of range [0, 1000]", opt->alpha_steps);
    if (opt->alpha_steps > 0) {
        if (!(opt->alpha_lr > 0.f) || !std::isfinite(opt->alpha_lr))
            return fail(ctx, SLR_EINVAL, "alpha_lr must be finite and positive");
        if (opt->alpha_cap < 1 || opt->alpha_cap > ((int64_t)1 << 24))
            return fail(ctx, SLR_EINVAL, "alpha_cap %lld out of range", (long long)opt->alpha_cap);
        if (!(opt->alpha_margin >= 0.f) || !std::isfinite(opt->alpha_margin))
            return fail(ctx, SLR_EINVAL, "alpha_margin must be finite and >= 0");
        if (opt->relax_mode != SLR_RELAX_NEURIFY)
            return fail(ctx, SLR_EUNSUPPORTED, "slope optimisation needs relax mode NEURIFY");
    }
    if (opt->recheck_cluster != 0 && opt->recheck_cluster != 1)
        return fail(ctx, SLR_EINVAL, "recheck_cluster must be 0 or 1");
    if (opt->recheck_pairs != 0 && opt->recheck_pairs != 1)
        return fail(ctx, SLR_EINVAL, "recheck_pairs must be 0 or 1");
    if (opt->shard_count < 1 || opt->shard_index < 0 || opt->shard_index >= opt->shard_count ||
        opt->shard_level < 0 || opt->shard_level > slr::kMaxDepth)
        return fail(ctx, SLR_EINVAL, "shard %d of %d at level %d is not valid", opt->shard_index, opt->shard_count,
                    opt->shard_level);
    if (opt->wide != 0 && opt->wide != 1) return fail(ctx, SLR_EINVAL, "wide must be 0 or 1");
    if ((opt->tile_boxes == 0) != (opt->tile_threads == 0))
        return fail(ctx, SLR_EINVAL, "tile_boxes and tile_threads are set together");
    if (opt->relax_mode != ctx->opt.relax_mode || opt->precision != ctx->opt.precision ||
        opt->tile_boxes != ctx->opt.tile_boxes || opt->tile_threads != ctx->opt.tile_threads ||
        opt->wide != ctx->opt.wide || opt->recheck_cluster != ctx->opt.recheck_cluster)
        ctx->dev_dirty = true;
    ctx->opt = *opt;
    return SLR_OK;
}

int slr_load_network(slr_ctx *ctx, int K, const int32_t *widths, const float *const *W, const float *const *b) {
    if (!ctx) return fail(nullptr, SLR_EINVAL, "null context");
    if (K < 1 || K > slr::kMaxLayers) return fail(ctx, SLR_EINVAL, "K=%d out of range [1, %d]", K, slr::kMaxLayers);
    if (!widths || !W || !b) return fail(ctx, SLR_EINVAL, "null widths/W/b");
    for (int k = 0; k <= K; ++k)
        if (widths[k] < 1 || widths[k] > slr::kMaxWidth)
            return fail(ctx, SLR_EINVAL, "widths[%d]=%d out of range [1, %d]", k, widths[k], slr::kMaxWidth);
    std::vector<std::vector<float>> Wv(K), bv(K);
    for (int k = 0; k < K; ++k) {
        if (!W[k] || !b[k]) return fail(ctx, SLR_EINVAL, "null W[%d] or b[%d]", k, k);
        const size_t nw = (size_t)widths[k + 1] * widths[k];
        if (!finite_all(W[k], nw) || !finite_all(b[k], widths[k + 1]))
            return fail(ctx, SLR_EINVAL, "non-finite value in layer %d", k);
        Wv[k].assign(W[k], W[k] + nw);
        bv[k].assign(b[k], b[k] + widths[k + 1]);
    }
    ctx->K = K;
    ctx->widths.assign(widths, widths + K + 1);
    ctx->W.swap(Wv);
    ctx->b.swap(bv);
    ctx->act.clear();
    ctx->has_net = true;
    ctx->dev_dirty = true;
    ctx->leaves_valid = false;
    return SLR_OK;
}

int slr_set_box(slr_ctx *ctx, int d, const float *lo, const float *hi) {
    if (!ctx) return fail(nullptr, SLR_EINVAL, "null context");
    if (d < 1 || d > slr::kMaxWidth || !lo || !hi) return fail(ctx, SLR_EINVAL, "bad box arguments (d=%d)", d);
    for (int i = 0; i < d; ++i) {
        if (!std::isfinite(lo[i]) || !std::isfinite(hi[i]))
            return fail(ctx, SLR_EINVAL, "non-finite box endpoint in dimension %d", i);
        if (lo[i] > hi[i]) return fail(ctx, SLR_EINVAL, "lo > hi in dimension %d", i);
    }
    ctx->lo.assign(lo, lo + d);
    ctx->hi.assign(hi, hi + d);
    ctx->has_box = true;
    ctx->leaves_valid = false;
    return SLR_OK;
}

int slr_set_activations(slr_ctx *ctx, int n, const int32_t *act) {
    if (!ctx) return fail(nullptr, SLR_EINVAL, "null context");
    if (!ctx->has_net) return fail(ctx, SLR_ESTATE, "load the network before its activations");
    if (n != ctx->K - 1 || (n > 0 && !act))
        return fail(ctx, SLR_EINVAL, "%d activations given for %d hidden layers", n, ctx->K - 1);
    for (int k = 0; k < n; ++k)
        if (act[k] != SLR_ACT_RELU && act[k] != SLR_ACT_TANH && act[k] != SLR_ACT_SIGMOID)
            return fail(ctx, SLR_EINVAL, "activation %d of hidden layer %d unknown", act[k], k);
    ctx->act.assign(act, act + n);
    ctx->dev_dirty = true;
    ctx->leaves_valid = false;
    return SLR_OK;
}

int slr_set_property(slr_ctx *ctx, int n_clauses, const int32_t *rows_per_clause, int n_out, const float *C,
                     const float *e, const uint8_t *strict) {
    if (!ctx) return fail(nullptr, SLR_EINVAL, "null context");
    if (n_clauses < 1 || !rows_per_clause || !C || !e || !strict || n_out < 1 || n_out > slr::kMaxWidth)
        return fail(ctx, SLR_EINVAL, "bad property arguments");
    int R = 0;
    for (int c = 0; c < n_clauses; ++c) {
        if (rows_per_clause[c] < 1) return fail(ctx, SLR_EINVAL, "clause %d has no rows", c);
        R += rows_per_clause[c];
        if (R > slr::kMaxRows) return fail(ctx, SLR_EINVAL, "more than %d property rows", slr::kMaxRows);
    }
    if (!finite_all(C, (size_t)R * n_out) || !finite_all(e, R))
        return fail(ctx, SLR_EINVAL, "non-finite value in the property");
    ctx->n_clauses = n_clauses;
    ctx->rpc.assign(rows_per_clause, rows_per_clause + n_clauses);
    ctx->C.assign(C, C + (size_t)R * n_out);
    ctx->e.assign(e, e + R);
    ctx->strict.assign(strict, strict + R);
    ctx->has_prop = true;
    ctx->dev_dirty = true;
    ctx->leaves_valid = false;
    return SLR_OK;
}

// A count's state at a level boundary (checkpoint): the counters of the
// levels already counted and the frontier of the first level still to run.
struct ResumeState {
    int t_first;
    const slr::LevelCounters *counters;   // host
    const uint64_t *codes;                // host, frontier of level t_first
    int64_t n;
};

// Levels t_first .. t_last of a count to depth D (t_first = 0 without a
// resume state, t_last = D for a whole count); the result covers every level
// counted so far.
namespace {
uint64_t fnv1a(uint64_t h, const void *p, size_t n);
}  // namespace

static int count_levels(slr_ctx *ctx, int D, slr_result *out, int t_last, const ResumeState *rs) {
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (!out) return fail(ctx, SLR_EINVAL, "out is NULL");
    if (D < 0 || D > slr::kMaxDepth) return fail(ctx, SLR_EINVAL, "D=%d out of range [0, %d]", D, slr::kMaxDepth);
    const bool grad_split = ctx->opt.split_rule == SLR_SPLIT_GRADIENT;
    if (grad_split && D > slr::kSplitMaxDepth)
        return fail(ctx, SLR_EINVAL, "the gradient split rule counts to depth %d at most (D=%d)", slr::kSplitMaxDepth, D);
    const bool sharded = ctx->opt.shard_count > 1;
    const int shard_g = ctx->opt.shard_level;
    if (sharded && shard_g > D)
        return fail(ctx, SLR_EINVAL, "shard level %d is below the depth cap D=%d", shard_g, D);
    CK(ctx, cudaSetDevice(ctx->device));
    if ((rc = prepare_device(ctx))) return rc;
    if ((rc = ensure_count_buffers(ctx))) return rc;
    const int d = ctx->widths[0];

    // split schedule: widest side first, ties to the lowest index (Sec. 2.2 bisection)
    std::vector<double> root(2 * (size_t)d);
    std::vector<unsigned long long> masks(d, 0ull);
    std::vector<int> cnt(d, 0);
    for (int i = 0; i < d; ++i) {
        root[i] = (double)ctx->lo[i];
        root[d + i] = (double)ctx->hi[i] - (double)ctx->lo[i];
    }
    ctx->sched.assign(D, 0);
    for (int t = 0; t < D; ++t) {
        int best = 0;
        double bw = -1.0;
        for (int i = 0; i < d; ++i) {
            const double w = std::ldexp(root[d + i], -cnt[i]);
            if (w > bw) {
                bw = w;
                best = i;
            }
        }
        ctx->sched[t] = best;
        cnt[best] += 1;
        masks[best] |= 1ull << (D - 1 - t);
    }
    const size_t root_bytes = root.size() * sizeof(double);
    const size_t mask_bytes = masks.size() * sizeof(unsigned long long);
    if ((rc = ensure_stage(ctx, root_bytes + mask_bytes))) return rc;
    std::memcpy(ctx->h_stage, root.data(), root_bytes);
    std::memcpy(ctx->h_stage + root_bytes, masks.data(), mask_bytes);
    CK(ctx, cudaMemcpyAsync(ctx->root, ctx->h_stage, root_bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaMemcpyAsync(ctx->masks, ctx->h_stage + root_bytes, mask_bytes, cudaMemcpyHostToDevice, ctx->stream));
    const int64_t h2d = ctx->h2d_pending + (int64_t)(root_bytes + mask_bytes);
    ctx->h2d_pending = 0;
    const int t_first = rs ? rs->t_first : 0;
    CK(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(unsigned int), ctx->stream));
    int64_t h2d_state = 0;
    if (!rs) {
        CK(ctx, cudaMemsetAsync(ctx->ctr, 0, sizeof(slr::LevelCounters), ctx->stream));
        CK(ctx, slr::launch_init_count(ctx->codes[0], ctx->ctr, ctx->stream));
    } else {
        if (rs->n > ctx->cap)
            return fail(ctx, SLR_EINVAL, "the checkpoint's frontier of %lld boxes exceeds frontier_cap=%lld",
                        (long long)rs->n, (long long)ctx->cap);
        CK(ctx, cudaMemcpyAsync(ctx->ctr, rs->counters, sizeof(slr::LevelCounters), cudaMemcpyHostToDevice,
                                ctx->stream));
        if (rs->n > 0)
            CK(ctx, cudaMemcpyAsync(ctx->codes[t_first & 1], rs->codes, (size_t)rs->n * sizeof(uint64_t),
                                    cudaMemcpyHostToDevice, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));   // the caller's host buffers are free after return
        h2d_state = (int64_t)sizeof(slr::LevelCounters) + rs->n * (int64_t)sizeof(uint64_t);
    }

    const bool leaves = ctx->opt.record_leaves != 0;
    const bool recheck = ctx->opt.fp64_recheck != 0 && ctx->T64 > 0;
    const bool slopes = ctx->opt.alpha_steps > 0;
    if (slopes || grad_split) {
        if ((rc = check_adjoint(ctx))) return rc;
        if (!ctx->alpha_ctr)
            CK(ctx, cudaMalloc(&ctx->alpha_ctr, 2 * (slr::kMaxDepth + 2) * sizeof(unsigned long long)));
        CK(ctx, cudaMemsetAsync(ctx->alpha_ctr, 0, 2 * (slr::kMaxDepth + 2) * sizeof(unsigned long long), ctx->stream));
    }
    const bool use_tc = ctx->opt.precision == SLR_PREC_TC_TF32 && ctx->tc_ok;
    const int compact_grid = std::max(1, ctx->sm_count * 4);
    const bool prof = ctx->opt.profile != 0;
    const size_t n_prof = prof ? (size_t)(D + 1) * 6 : 0;
    while (ctx->prof_ev.size() < n_prof) {
        cudaEvent_t e;
        CK(ctx, cudaEventCreate(&e));
        ctx->prof_ev.push_back(e);
    }
    // while the level loop is captured as a graph, the timing events become
    // event-record nodes of the graph (an ordinary record there is only an edge)
    bool capturing = false;
    auto mark = [&](int t, int slot) -> cudaError_t {
        if (!prof) return cudaSuccess;
        cudaEvent_t e = ctx->prof_ev[(size_t)t * 6 + slot];
        return capturing ? cudaEventRecordWithFlags(e, ctx->stream, cudaEventRecordExternal)
                         : cudaEventRecord(e, ctx->stream);
    };
    int64_t launches = rs ? 0 : 1;
    ctx->gemm_ev_used = 0;
    ctx->gemm_launches = 0;
    ctx->gemm_flop = 0;
    auto level_source = [&](int t) {
        slr::BoxSource src{};
        src.mode = 0;
        src.codes = ctx->codes[t & 1];
        src.count = &ctx->ctr->frontier_n[t];
        src.t = t;
        src.D = D;
        src.dim_mask = ctx->masks;
        src.root_lo = ctx->root;
        src.root_w = ctx->root + d;
        src.cap = ctx->cap;
        return src;
    };
    ctx->split_set.clear();
    if (grad_split) {
        // the split set from the box gradient at the root (before the timed region)
        if ((rc = slr_internal_split_root(ctx, level_source(0), &launches))) return rc;
        launches = 1;
    }
    const uint64_t path_mask = grad_split ? (1ull << slr::kSplitPathBits) - 1ull : ~0ull;
    auto run_levels = [&]() -> int {
    for (int t = t_first; t <= t_last; ++t) {
        if (sharded && t == shard_g) {
            // this shard's subtrees: every shard_count-th box of level g
            CK(ctx, slr::launch_shard_level(ctx->codes[t & 1], ctx->codes[(t + 1) & 1], ctx->ctr, t,
                                            ctx->opt.shard_count, ctx->opt.shard_index, ctx->cap, ctx->sm_count,
                                            ctx->stream));
            launches += 3;
        }
        slr::BoxSource src = level_source(t);
        if (grad_split) src.split_of = (const int8_t *)ctx->split_buf;
        slr::EvalOutputs o{};
        o.cls = ctx->cls;
        o.near_list = recheck ? ctx->near_list : nullptr;
        o.near_count = &ctx->ctr->near_n[t];
        o.near_cap = ctx->near_cap;
        o.tie_count = &ctx->ctr->ties;
        o.status = ctx->status;
        CK(ctx, mark(t, 0));
        if (ctx->wide) {
            // the chunk loop needs the level's size on the host
            CK(ctx, cudaMemcpyAsync(&ctx->h_ctr->frontier_n[t], &ctx->ctr->frontier_n[t], sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, ctx->stream));
            CK(ctx, cudaStreamSynchronize(ctx->stream));
            const int64_t nt = std::min<int64_t>((int64_t)ctx->h_ctr->frontier_n[t], ctx->cap);
            slr::EvalOutputs ow{};
            ow.cls = ctx->cls;
            ow.tie_count = &ctx->ctr->ties;
            ow.status = ctx->status;
            ow.near_list = recheck ? ctx->near_list : nullptr;
            ow.near_count = &ctx->ctr->near_n[t];
            ow.near_cap = ctx->near_cap;
            if ((rc = run_wide(ctx, src, nt, ow, &launches))) return rc;
            CK(ctx, mark(t, 1));
            if (recheck) {
                // boxes whose class depends on the wide path's widening, in FP64
                slr::BoxSource s2 = src;
                s2.index = ctx->near_list;
                s2.index_count = &ctx->ctr->near_n[t];
                s2.cap = ctx->near_cap;
                slr::EvalOutputs o2{};
                o2.cls = ctx->cls;
                o2.tie_count = &ctx->ctr->ties;
                o2.status = ctx->status;
                int64_t nl = 0;
                CK(ctx, launch_recheck(ctx, s2, o2, t, &nl));
                launches += nl;
            }
        } else if (use_tc) {
            // tier 1 on the tensor cores; boxes whose class depends on its
            // widening are re-bounded by the FP32 path (tier 2), and those whose
            // class still depends on the FP32 widening in FP64 (tier 3)
            o.near_list = ctx->near_list;
            CK(ctx, slr::launch_eval_tc(ctx->T_tc, ctx->grid_tc, ctx->smem_tc, ctx->stream, ctx->nf, ctx->tcp, src, o, 0));
            CK(ctx, mark(t, 1));
            ++launches;
            slr::BoxSource s1 = src;
            s1.index = ctx->near_list;
            s1.index_count = &ctx->ctr->near_n[t];
            s1.cap = ctx->near_cap;
            slr::EvalOutputs o1 = o;
            o1.near_list = recheck ? ctx->near_list2 : nullptr;
            o1.near_count = &ctx->ctr->near2_n[t];
            CK(ctx, slr::launch_eval_f32(ctx->T32, ctx->NT32, ctx->grid32, ctx->smem32, ctx->stream, ctx->nf, s1, o1, 0));
            ++launches;
            if (recheck) {
                slr::BoxSource s2 = src;
                s2.index = ctx->near_list2;
                s2.index_count = &ctx->ctr->near2_n[t];
                s2.cap = ctx->near_cap;
                slr::EvalOutputs o2{};
                o2.cls = ctx->cls;
                o2.tie_count = &ctx->ctr->ties;
                o2.status = ctx->status;
                int64_t nl = 0;
                CK(ctx, launch_recheck(ctx, s2, o2, t, &nl));
                launches += nl;
            }
        } else {
        CK(ctx, slr::launch_eval_f32(ctx->T32, ctx->NT32, ctx->grid32, ctx->smem32, ctx->stream, ctx->nf, src, o, 0));
        CK(ctx, mark(t, 1));
        ++launches;
        if (recheck) {
            slr::BoxSource s2 = src;
            s2.index = ctx->near_list;
            s2.index_count = &ctx->ctr->near_n[t];
            s2.cap = ctx->near_cap;
            slr::EvalOutputs o2{};
            o2.cls = ctx->cls;
            o2.tie_count = &ctx->ctr->ties;
            o2.status = ctx->status;
            int64_t nl = 0;
            CK(ctx, launch_recheck(ctx, s2, o2, t, &nl));
            launches += nl;
        }
        }
        CK(ctx, mark(t, 2));
        if (slopes && t < D) {
            // boxes at depth D are leaves either way; above it, optimised slopes
            // may decide boxes that would otherwise be split
            if ((rc = slr_internal_alpha_level(ctx, src, t, &launches))) return rc;
        }
        if (grad_split && t < D) {
            if ((rc = slr_internal_split_level(ctx, src, t, slopes, &launches))) return rc;
        }
        CK(ctx, mark(t, 3));
        CK(ctx, mark(t, 4));
        CK(ctx, slr::launch_compact(ctx->codes[t & 1], ctx->cls, ctx->codes[(t + 1) & 1], ctx->ctr, ctx->status,
                                    ctx->cap, t, D, leaves ? ctx->leaf_codes : nullptr, ctx->leaf_depth,
                                    ctx->leaf_cls, ctx->opt.leaf_cap, compact_grid, ctx->stream, path_mask,
                                    !sharded || ctx->opt.shard_index == 0 || t >= shard_g));
        CK(ctx, mark(t, 5));
        launches += 2;
    }
    return SLR_OK;
    };
    // The tile path reads no count on the host between levels: its level loop
    // is captured as a CUDA graph once per configuration and buffer set, and
    // replayed (fewer launch gaps between the small kernels of a level).  The
    // key holds everything the captured launches take by value (the network
    // parameters' bytes, hashed, so that a problem uploaded again into the
    // same buffers replays the graph), the buffers and the launch shapes;
    // the values in those buffers are read when the graph runs.
    const bool graphable = !ctx->wide && !slopes && !grad_split && !rs && t_last == D;
    if (graphable) {
        uint64_t hp = fnv1a(14695981039346656037ull, &ctx->nf, sizeof ctx->nf);
        hp = fnv1a(hp, &ctx->nd, sizeof ctx->nd);
        if (use_tc) hp = fnv1a(hp, &ctx->tcp, sizeof ctx->tcp);
        char key[640];
        std::snprintf(key, sizeof key,
                      "%d|%d|%d|%d|%d|%d|%d|%d|%llu|%p|%p|%p|%p|%p|%p|%p|%p|%p|%lld|%lld|%lld|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d",
                      D, leaves ? 1 : 0, recheck ? 1 : 0, use_tc ? 1 : 0, prof ? 1 : 0, ctx->opt.shard_count,
                      ctx->opt.shard_index, shard_g,
                      (unsigned long long)hp, (void *)ctx->codes[0], (void *)ctx->codes[1],
                      (void *)ctx->cls, (void *)ctx->ctr, (void *)ctx->near_list, (void *)ctx->near_list2,
                      (void *)ctx->leaf_codes, (void *)ctx->masks, (void *)ctx->root, (long long)ctx->cap,
                      (long long)ctx->near_cap, (long long)ctx->opt.leaf_cap, ctx->T32, ctx->NT32, ctx->T64,
                      ctx->NT64, ctx->grid32, ctx->grid64, ctx->grid64c, ctx->opt.recheck_pairs,
                      ctx->pairs_fit ? 1 : 0, use_tc ? ctx->T_tc : 0, use_tc ? ctx->grid_tc : 0);
        if (!ctx->count_graph || ctx->count_graph_key != key) {
            if (ctx->count_graph) cudaGraphExecDestroy(ctx->count_graph);
            ctx->count_graph = nullptr;
            ctx->count_graph_key.clear();
            CK(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            const int64_t l0 = launches;
            capturing = true;
            const int rcap = run_levels();
            capturing = false;
            cudaGraph_t g = nullptr;
            const cudaError_t ee = cudaStreamEndCapture(ctx->stream, &g);
            if (rcap) {
                if (ee == cudaSuccess && g) cudaGraphDestroy(g);
                return rcap;
            }
            if (ee != cudaSuccess) return cuda_fail(ctx, ee, "capturing the level loop");
            const cudaError_t ie = cudaGraphInstantiate(&ctx->count_graph, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) {
                ctx->count_graph = nullptr;
                return cuda_fail(ctx, ie, "cudaGraphInstantiate");
            }
            ctx->count_graph_key = key;
            ctx->count_graph_launches = launches - l0;
            launches = l0;
        }
        CK(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
        CK(ctx, cudaGraphLaunch(ctx->count_graph, ctx->stream));
        launches += ctx->count_graph_launches;
    } else {
        CK(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
        if ((rc = run_levels())) return rc;
    }
    CK(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
    CK(ctx, cudaMemcpyAsync(ctx->h_ctr, ctx->ctr, sizeof(slr::LevelCounters), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaMemcpyAsync(ctx->h_status, ctx->status, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
    unsigned long long h_alpha[2 * (slr::kMaxDepth + 2)] = {};
    if (slopes || grad_split)
        CK(ctx, cudaMemcpyAsync(h_alpha, ctx->alpha_ctr, sizeof h_alpha, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (grad_split) {
        const int64_t list_cap = std::min<int64_t>(ctx->opt.alpha_cap, ctx->cap);
        for (int t = 0; t < D; ++t)
            if ((int64_t)h_alpha[2 * t] > list_cap)
                return fail(ctx, SLR_EOVERFLOW,
                            "level %d left %llu boxes UNDECIDED, more than alpha_cap=%lld boxes whose split the "
                            "gradient rule can choose", t, h_alpha[2 * t], (long long)list_cap);
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);

    const slr::LevelCounters &c = *ctx->h_ctr;
    std::memset(out, 0, sizeof *out);
    out->unsafe_lo = c.unsafe_lo;
    out->unsafe_hi = c.unsafe_lo + c.undecided_at_D;
    out->boxes = c.boxes;
    out->tie_leaves = c.ties;
    out->depth = D;
    int levels = 0;
    unsigned long long rech = 0, rech2 = 0, rech3 = 0;
    for (int t = 0; t <= D; ++t) {
        rech2 += std::min<unsigned long long>(c.near2_n[t], (unsigned long long)ctx->near_cap);
        rech3 += std::min<unsigned long long>(c.near3_n[t], (unsigned long long)ctx->near_cap);
        out->level_boxes[t] = c.level_boxes[t];
        out->level_safe[t] = c.level_safe[t];
        out->level_unsafe[t] = c.level_unsafe[t];
        out->level_undecided[t] = c.level_undecided[t];
        rech += std::min<unsigned long long>(c.near_n[t], (unsigned long long)ctx->near_cap);
        if (c.level_boxes[t]) levels = t + 1;
    }
    out->rechecked = recheck ? (use_tc ? rech2 : rech) : 0;
    out->rechecked_fp32 = use_tc ? rech : 0;
    out->rechecked_fp64 = (ctx->opt.recheck_pairs && ctx->pairs_fit && ctx->grid64c == 0) ? rech3 : out->rechecked;
    out->levels = levels;
    out->device_ms = ms;
    out->launches = launches;
    out->h2d_bytes = h2d + h2d_state;
    out->tile_boxes = ctx->wide ? ctx->wide_Bc : ctx->T32;
    out->tile_threads = ctx->wide ? 0 : ctx->NT32;
    out->d2h_bytes = (int64_t)(sizeof(slr::LevelCounters) + sizeof(unsigned int) + (slopes ? sizeof h_alpha : 0));
    if (slopes) {
        const int64_t acap = std::min<int64_t>(ctx->opt.alpha_cap, ctx->cap);
        for (int t = 0; t <= D; ++t) {
            out->alpha_boxes += std::min<unsigned long long>(h_alpha[2 * t], (unsigned long long)acap);
            out->alpha_decided += h_alpha[2 * t + 1];
        }
    }
    if (prof) {
        for (int t = t_first; t <= t_last; ++t) {
            float a = 0.f, b = 0.f, c2 = 0.f;
            cudaEventElapsedTime(&a, ctx->prof_ev[(size_t)t * 6 + 0], ctx->prof_ev[(size_t)t * 6 + 1]);
            cudaEventElapsedTime(&b, ctx->prof_ev[(size_t)t * 6 + 1], ctx->prof_ev[(size_t)t * 6 + 2]);
            cudaEventElapsedTime(&c2, ctx->prof_ev[(size_t)t * 6 + 4], ctx->prof_ev[(size_t)t * 6 + 5]);
            float s3 = 0.f;
            cudaEventElapsedTime(&s3, ctx->prof_ev[(size_t)t * 6 + 2], ctx->prof_ev[(size_t)t * 6 + 3]);
            out->alpha_ms += s3;
            out->kernel_ms[0] += a;
            out->kernel_ms[1] += b;
            out->kernel_ms[2] += c2;
        }
        (void)cudaGetLastError();   // a timing read that failed must not surface at the next launch
    }
    out->gemm_launches = ctx->gemm_launches;
    out->gemm_flop = ctx->gemm_flop;
    for (size_t i = 0; i + 1 < ctx->gemm_ev_used; i += 2) {
        float g = 0.f;
        cudaEventElapsedTime(&g, ctx->gemm_ev[i], ctx->gemm_ev[i + 1]);
        out->gemm_ms += g;
    }
    ctx->n_leaves = leaves ? (int64_t)c.leaves : 0;
    ctx->leaves_valid = leaves;
    const unsigned st = *ctx->h_status;
    if (st & slr::kStatusOverflow)
        return fail(ctx, SLR_EOVERFLOW, "a level exceeded frontier_cap=%lld boxes", (long long)ctx->cap);
    if (st & slr::kStatusNearOverflow)
        return fail(ctx, SLR_EOVERFLOW, "FP64 re-check list exceeded %lld boxes", (long long)ctx->near_cap);
    if (st & slr::kStatusLeafOverflow)
        return fail(ctx, SLR_EOVERFLOW, "leaf recording exceeded leaf_cap=%lld", (long long)ctx->opt.leaf_cap);
    if (st & slr::kStatusTimeout)
        return fail(ctx, SLR_ETIMEOUT, "a bounded wait on the tensor core gave up; the result is incomplete");
    return SLR_OK;
}

int slr_count(slr_ctx *ctx, int D, slr_result *out) { return count_levels(ctx, D, out, D, nullptr); }

// ---- checkpoint / resume ----------------------------------------------------
namespace {
constexpr uint32_t kCkptMagic = 0x43524c53u;   // "SLRC"
constexpr uint32_t kCkptVersion = 3;

// The FP32 tile (boxes and threads per CTA) is part of the state: small tiles
// split a product's inputs over lanes, so the summation order, and with it
// which boxes land on the FP64 re-check list, depends on the tile.  A resume
// runs the checkpoint's tile whatever the autotuner of its context chose.
struct CkptHeader {
    uint32_t magic, version;
    int32_t D, t;
    uint64_t fingerprint;
    uint64_t n_codes;
    uint64_t counters_bytes;
    int32_t tile_boxes, tile_threads;
};

uint64_t fnv1a(uint64_t h, const void *p, size_t n) {
    const unsigned char *c = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= c[i];
        h *= 1099511628211ull;
    }
    return h;
}

// Network, box, property and the options that change a count's result.
uint64_t problem_fingerprint(const slr_ctx *ctx) {
    uint64_t h = 14695981039346656037ull;
    h = fnv1a(h, &ctx->K, sizeof ctx->K);
    h = fnv1a(h, ctx->widths.data(), ctx->widths.size() * sizeof(int));
    for (const auto &w : ctx->W) h = fnv1a(h, w.data(), w.size() * sizeof(float));
    for (const auto &v : ctx->b) h = fnv1a(h, v.data(), v.size() * sizeof(float));
    h = fnv1a(h, ctx->lo.data(), ctx->lo.size() * sizeof(float));
    h = fnv1a(h, ctx->hi.data(), ctx->hi.size() * sizeof(float));
    h = fnv1a(h, &ctx->n_clauses, sizeof ctx->n_clauses);
    h = fnv1a(h, ctx->rpc.data(), ctx->rpc.size() * sizeof(int));
    h = fnv1a(h, ctx->C.data(), ctx->C.size() * sizeof(float));
    h = fnv1a(h, ctx->e.data(), ctx->e.size() * sizeof(float));
    h = fnv1a(h, ctx->strict.data(), ctx->strict.size());
    h = fnv1a(h, ctx->act.data(), ctx->act.size() * sizeof(int));
    const int32_t o[6] = {ctx->opt.precision, ctx->opt.relax_mode, ctx->opt.fp64_recheck, ctx->wide ? 1 : 0,
                          ctx->opt.recheck_cluster, ctx->opt.recheck_pairs};
    return fnv1a(h, o, sizeof o);
}

int check_resumable(slr_ctx *ctx, const char *what) {
    if (ctx->opt.record_leaves) return fail(ctx, SLR_EUNSUPPORTED, "%s does not record leaves", what);
    if (ctx->opt.alpha_steps > 0) return fail(ctx, SLR_EUNSUPPORTED, "%s runs fixed slopes only", what);
    if (ctx->opt.split_rule != SLR_SPLIT_WIDEST)
        return fail(ctx, SLR_EUNSUPPORTED, "%s splits the widest side only", what);
    if (ctx->opt.shard_count > 1) return fail(ctx, SLR_EUNSUPPORTED, "%s does not shard", what);
    return SLR_OK;
}
}  // namespace

int slr_count_checkpoint(slr_ctx *ctx, int D, int t, void *buf, size_t cap, size_t *used) {
    if (!ctx) return fail(nullptr, SLR_EINVAL, "null context");
    if (!used) return fail(ctx, SLR_EINVAL, "used is NULL");
    *used = 0;
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (D < 1 || D > slr::kMaxDepth) return fail(ctx, SLR_EINVAL, "D=%d out of range [1, %d]", D, slr::kMaxDepth);
    if (t < 0 || t >= D) return fail(ctx, SLR_EINVAL, "checkpoint level t=%d out of range [0, %d)", t, D);
    if ((rc = check_resumable(ctx, "slr_count_checkpoint"))) return rc;
    slr_result part;
    if ((rc = count_levels(ctx, D, &part, t, nullptr))) return rc;
    // count_levels synchronised the stream and copied the counters to h_ctr
    const uint64_t n = ctx->h_ctr->frontier_n[t + 1];
    const size_t need = sizeof(CkptHeader) + sizeof(slr::LevelCounters) + (size_t)n * sizeof(uint64_t);
    *used = need;
    if (!buf || cap < need)
        return fail(ctx, SLR_EINVAL, "the checkpoint needs %zu bytes (buffer of %zu)", need, buf ? cap : (size_t)0);
    CkptHeader h{kCkptMagic, kCkptVersion, D, t, problem_fingerprint(ctx), n, sizeof(slr::LevelCounters),
                 ctx->T32, ctx->NT32};
    unsigned char *p = static_cast<unsigned char *>(buf);
    std::memcpy(p, &h, sizeof h);
    std::memcpy(p + sizeof h, ctx->h_ctr, sizeof(slr::LevelCounters));
    if (n > 0)
        CK(ctx, cudaMemcpyAsync(p + sizeof h + sizeof(slr::LevelCounters), ctx->codes[(t + 1) & 1],
                                (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return SLR_OK;
}

int slr_count_resume(slr_ctx *ctx, const void *buf, size_t bytes, slr_result *out) {
    if (!ctx) return fail(nullptr, SLR_EINVAL, "null context");
    if (!out) return fail(ctx, SLR_EINVAL, "out is NULL");
    int rc = check_ready(ctx);
    if (rc) return rc;
    if ((rc = check_resumable(ctx, "slr_count_resume"))) return rc;
    const size_t head = sizeof(CkptHeader) + sizeof(slr::LevelCounters);
    if (!buf || bytes < head) return fail(ctx, SLR_EINVAL, "not a checkpoint (%zu bytes)", bytes);
    const unsigned char *p = static_cast<const unsigned char *>(buf);
    CkptHeader h;
    std::memcpy(&h, p, sizeof h);
    if (h.magic != kCkptMagic || h.version != kCkptVersion || h.counters_bytes != sizeof(slr::LevelCounters))
        return fail(ctx, SLR_EINVAL, "not a checkpoint of this library version");
    if (h.D < 1 || h.D > slr::kMaxDepth || h.t < 0 || h.t >= h.D)
        return fail(ctx, SLR_EINVAL, "checkpoint with D=%d, t=%d is not valid", h.D, h.t);
    if (h.n_codes > (bytes - head) / sizeof(uint64_t) || bytes != head + h.n_codes * sizeof(uint64_t))
        return fail(ctx, SLR_EINVAL, "checkpoint of %zu bytes does not hold its %llu codes", bytes,
                    (unsigned long long)h.n_codes);
    CK(ctx, cudaSetDevice(ctx->device));
    if ((rc = prepare_device(ctx))) return rc;   // decides the path (tile or wide) the fingerprint includes
    if (h.fingerprint != problem_fingerprint(ctx))
        return fail(ctx, SLR_EINVAL, "the checkpoint is of another network, box, property or result options");
    std::vector<unsigned char> ctr(sizeof(slr::LevelCounters));
    std::memcpy(ctr.data(), p + sizeof h, ctr.size());
    const slr::LevelCounters *c = reinterpret_cast<const slr::LevelCounters *>(ctr.data());
    if (c->frontier_n[h.t + 1] != h.n_codes)
        return fail(ctx, SLR_EINVAL, "checkpoint counters and frontier disagree");
    std::vector<uint64_t> codes((size_t)h.n_codes);
    if (h.n_codes > 0) std::memcpy(codes.data(), p + head, (size_t)h.n_codes * sizeof(uint64_t));
    ResumeState rs{h.t + 1, c, codes.data(), (int64_t)h.n_codes};
    if (ctx->wide || (h.tile_boxes == ctx->T32 && h.tile_threads == ctx->NT32))
        return count_levels(ctx, h.D, out, h.D, &rs);
    // the checkpoint's FP32 tile for the resumed levels, the context's own afterwards
    TileChoice tile{};
    for (const TileChoice &cand : tile_candidates(ctx->nf))
        if (cand.T == h.tile_boxes && cand.NT == h.tile_threads) tile = cand;
    if (tile.T == 0)
        return fail(ctx, SLR_EINVAL, "the checkpoint's tile %d x %d is not available for this network", h.tile_boxes,
                    h.tile_threads);
    const int T0 = ctx->T32, NT0 = ctx->NT32, g0 = ctx->grid32;
    const size_t s0 = ctx->smem32;
    ctx->T32 = tile.T;
    ctx->NT32 = tile.NT;
    ctx->smem32 = tile.smem;
    ctx->grid32 = tile.blocks * ctx->sm_count;
    rc = count_levels(ctx, h.D, out, h.D, &rs);
    ctx->T32 = T0;
    ctx->NT32 = NT0;
    ctx->grid32 = g0;
    ctx->smem32 = s0;
    return rc;
}

// ---- approximate counter (CountingProVe_SLR, Sec. 2.3; Table 1) ------------
namespace {

// The exact count of the box [lo, hi] with the context's network, property and
// options; the context's own box is put back afterwards.
int count_sub_box(slr_ctx *ctx, const std::vector<float> &lo, const std::vector<float> &hi, int D, slr_result *out) {
    std::vector<float> lo0 = ctx->lo, hi0 = ctx->hi;
    ctx->lo = lo;
    ctx->hi = hi;
    const int rc = count_levels(ctx, D, out, D, nullptr);
    ctx->lo.swap(lo0);
    ctx->hi.swap(hi0);
    return rc;
}

}  // namespace

void slr_default_approx_options(slr_approx_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->trials = 8;
    o->splits = 10;
    o->samples = 4096;
    o->leaf_depth = 12;
    o->beta = 1.0;
    o->seed = 0;
}

int slr_count_approx(slr_ctx *ctx, const slr_approx_options *o, slr_approx_result *out, float *leaf_lo,
                     float *leaf_hi) {
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (!o || !out) return fail(ctx, SLR_EINVAL, "null options or result");
    if (o->trials < 1 || o->trials > SLR_APPROX_MAX_TRIALS)
        return fail(ctx, SLR_EINVAL, "trials=%d out of range [1, %d]", o->trials, SLR_APPROX_MAX_TRIALS);
    if (o->splits < 0 || o->splits > slr::kMaxDepth)
        return fail(ctx, SLR_EINVAL, "splits=%d out of range [0, %d]", o->splits, slr::kMaxDepth);
    if (o->samples < 1 || o->samples >= slr::kApproxCoinPoint)
        return fail(ctx, SLR_EINVAL, "samples=%d out of range [1, %d)", o->samples, slr::kApproxCoinPoint);
    if (o->leaf_depth < 0 || o->leaf_depth > slr::kMaxDepth)
        return fail(ctx, SLR_EINVAL, "leaf_depth=%d out of range [0, %d]", o->leaf_depth, slr::kMaxDepth);
    if (!(o->beta > 0.0) || !std::isfinite(o->beta)) return fail(ctx, SLR_EINVAL, "beta must be finite and > 0");
    if (ctx->opt.shard_count > 1) return fail(ctx, SLR_EUNSUPPORTED, "the approximate counter does not shard");
    CK(ctx, cudaSetDevice(ctx->device));
    if ((rc = prepare_device(ctx))) return rc;
    const int d = ctx->widths[0];
    const size_t need = align_up(2 * (size_t)d * sizeof(double)) + align_up((size_t)o->samples * sizeof(double)) +
                        align_up(sizeof(unsigned long long));
    if (ctx->approx_bytes < need) {
        cudaFree(ctx->approx_buf);
        ctx->approx_buf = nullptr;
        ctx->approx_bytes = 0;
        CK(ctx, cudaMalloc(&ctx->approx_buf, need));
        ctx->approx_bytes = need;
    }
    unsigned char *base = static_cast<unsigned char *>(ctx->approx_buf);
    double *d_box = reinterpret_cast<double *>(base);
    double *d_coord = reinterpret_cast<double *>(base + align_up(2 * (size_t)d * sizeof(double)));
    unsigned long long *d_cnt = reinterpret_cast<unsigned long long *>(
        base + align_up(2 * (size_t)d * sizeof(double)) + align_up((size_t)o->samples * sizeof(double)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(ctx, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(ctx, SLR_ECUDA, "cudaEventCreate");
    }
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } guard{e0, e1};

    std::memset(out, 0, sizeof *out);
    out->trials = o->trials;
    std::vector<double> box(2 * (size_t)d), coord;
    double est_min = 0.0, est_sum = 0.0;
    for (int t = 0; t < o->trials; ++t) {
        std::vector<float> lo = ctx->lo, hi = ctx->hi;
        int s = 0;
        for (int j = 0; j < o->splits; ++j) {
            // the widest side, ties to the lowest index
            int dim = 0;
            double wmax = -1.0;
            for (int i = 0; i < d; ++i) {
                const double w = (double)hi[i] - (double)lo[i];
                if (w > wmax) {
                    wmax = w;
                    dim = i;
                }
            }
            if (!(wmax > 0.0)) break;
            for (int i = 0; i < d; ++i) {
                box[i] = lo[i];
                box[d + i] = hi[i];
            }
            CK(ctx, cudaMemcpyAsync(d_box, box.data(), box.size() * sizeof(double), cudaMemcpyHostToDevice,
                                    ctx->stream));
            CK(ctx, cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), ctx->stream));
            CK(ctx, cudaEventRecord(e0, ctx->stream));
            CK(ctx, slr::launch_approx_sample(ctx->nd, d_box, d_box + d, dim, o->seed, t, j, o->samples, d_coord,
                                              d_cnt, ctx->sm_count, ctx->stream));
            CK(ctx, cudaEventRecord(e1, ctx->stream));
            unsigned long long n_uns = 0;
            CK(ctx, cudaMemcpyAsync(&n_uns, d_cnt, sizeof n_uns, cudaMemcpyDeviceToHost, ctx->stream));
            CK(ctx, cudaStreamSynchronize(ctx->stream));
            n_uns = std::min<unsigned long long>(n_uns, (unsigned long long)o->samples);
            coord.resize((size_t)n_uns);
            if (n_uns > 0) {
                CK(ctx, cudaMemcpyAsync(coord.data(), d_coord, (size_t)n_uns * sizeof(double),
                                        cudaMemcpyDeviceToHost, ctx->stream));
                CK(ctx, cudaStreamSynchronize(ctx->stream));
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            out->device_ms += ms;
            out->samples_unsafe += n_uns;
            // split point: the lower median of the sampled violations on this
            // side (the midpoint without any), to the nearest float32, strictly inside
            double m64;
            if (n_uns > 0) {
                const size_t k = (size_t)(n_uns - 1) / 2;
                std::nth_element(coord.begin(), coord.begin() + k, coord.end());
                m64 = coord[k];
            } else {
                m64 = 0.5 * ((double)lo[dim] + (double)hi[dim]);
            }
            float m = (float)m64;
            if (!(lo[dim] < m && m < hi[dim])) {
                m = (float)(0.5 * ((double)lo[dim] + (double)hi[dim]));
                if (!(lo[dim] < m && m < hi[dim])) break;
            }
            // a fair coin keeps one half
            const unsigned long long c = slr::splitmix64(o->seed, slr::approx_draw_index(t, j, slr::kApproxCoinPoint, 0));
            if ((c >> 63) == 0ull) hi[dim] = m;
            else lo[dim] = m;
            ++s;
        }
        slr_result r;
        if ((rc = count_sub_box(ctx, lo, hi, o->leaf_depth, &r))) return rc;
        double vol = 1.0;
        for (int i = 0; i < d; ++i) {
            const double wr = (double)ctx->hi[i] - (double)ctx->lo[i];
            if (wr > 0.0) vol = vol * (((double)hi[i] - (double)lo[i]) / wr);
        }
        const double est = std::ldexp((double)r.unsafe_lo * vol, s - o->leaf_depth);
        out->splits_done[t] = s;
        out->leaf_unsafe_lo[t] = r.unsafe_lo;
        out->leaf_unsafe_hi[t] = r.unsafe_hi;
        out->leaf_volume[t] = vol;
        out->estimate[t] = est;
        out->estimate_hi[t] = std::ldexp((double)r.unsafe_hi * vol, s - o->leaf_depth);
        out->boxes += r.boxes;
        out->device_ms += r.device_ms;
        est_min = t == 0 ? est : std::min(est_min, est);
        est_sum += est;
        if (leaf_lo) std::memcpy(leaf_lo + (size_t)t * d, lo.data(), (size_t)d * sizeof(float));
        if (leaf_hi) std::memcpy(leaf_hi + (size_t)t * d, hi.data(), (size_t)d * sizeof(float));
    }
    out->vr_lower = est_min * std::pow(2.0, -o->beta);
    out->confidence = 1.0 - std::pow(2.0, -o->beta * o->trials);
    out->vr_mean = est_sum / o->trials;
    return SLR_OK;
}

int slr_bounds(slr_ctx *ctx, int64_t n, const float *box_lo, const float *box_hi, const float *alpha,
               float *row_lo, float *row_hi, float *row_err, uint8_t *cls, int on_device) {
    if (!ctx) return fail(nullptr, SLR_EINVAL, "null context");
    if (!ctx->has_net || !ctx->has_prop) return fail(ctx, SLR_ESTATE, "network and property must be set");
    if (n < 0 || (n > 0 && (!box_lo || !box_hi))) return fail(ctx, SLR_EINVAL, "bad box arguments");
    if ((row_lo == nullptr) != (row_hi == nullptr)) return fail(ctx, SLR_EINVAL, "row_lo and row_hi go together");
    if (alpha && ctx->opt.relax_mode != SLR_RELAX_NEURIFY)
        return fail(ctx, SLR_EUNSUPPORTED, "supplied slopes need relax mode NEURIFY");
    if (alpha)
        for (int a : ctx->act)
            if (a != SLR_ACT_RELU) return fail(ctx, SLR_EUNSUPPORTED, "supplied slopes need a ReLU network");
    if (n == 0) return SLR_OK;
    CK(ctx, cudaSetDevice(ctx->device));
    int rc = prepare_device(ctx);
    if (rc) return rc;
    const int d = ctx->widths[0];
    const int R = (int)ctx->e.size();
    const int64_t H = ctx->H;
    const float *dlo = box_lo, *dhi = box_hi, *dal = alpha;
    float *drl = row_lo, *drh = row_hi, *dre = row_err;
    uint8_t *dcls = cls;
    if (!on_device) {
        if ((rc = check_boxes(ctx, n, d, box_lo, box_hi))) return rc;
        const size_t na = alpha ? (size_t)n * H : 0;
        const size_t need = align_up(2 * (size_t)n * d * sizeof(float)) + align_up(3 * (size_t)n * R * sizeof(float)) +
                            align_up((size_t)n) + align_up(na * sizeof(float));
        if ((rc = ensure_scratch(ctx, need))) return rc;
        unsigned char *p = (unsigned char *)ctx->scratch;
        float *slo = (float *)p;
        float *shi = slo + (size_t)n * d;
        p += align_up(2 * (size_t)n * d * sizeof(float));
        drl = row_lo ? (float *)p : nullptr;
        drh = row_lo ? (float *)p + (size_t)n * R : nullptr;
        dre = row_err ? (float *)p + 2 * (size_t)n * R : nullptr;
        p += align_up(3 * (size_t)n * R * sizeof(float));
        dcls = cls ? (uint8_t *)p : nullptr;
        p += align_up((size_t)n);
        CK(ctx, cudaMemcpyAsync(slo, box_lo, (size_t)n * d * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
        CK(ctx, cudaMemcpyAsync(shi, box_hi, (size_t)n * d * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
        if (alpha) {
            CK(ctx, cudaMemcpyAsync(p, alpha, na * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
            dal = (const float *)p;
        }
        dlo = slo;
        dhi = shi;
    }
    slr::BoxSource src{};
    src.mode = 1;
    src.n_explicit = n;
    src.lo = dlo;
    src.hi = dhi;
    src.cap = n;
    src.alpha = dal;
    src.alpha_ld = H;
    slr::EvalOutputs o{};
    o.cls = dcls;
    o.row_lo = drl;
    o.row_hi = drh;
    o.row_err = dre;
    if (!ctx->status) {
        CK(ctx, cudaMalloc(&ctx->status, sizeof(unsigned int)));
        CK(ctx, cudaMallocHost(&ctx->h_status, sizeof(unsigned int)));
    }
    o.status = ctx->status;
    CK(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(unsigned int), ctx->stream));
    if (ctx->wide) {
        int64_t launches = 0;
        if ((rc = run_wide(ctx, src, n, o, &launches))) return rc;
    } else if (ctx->opt.precision == SLR_PREC_TC_TF32 && ctx->tc_ok && alpha == nullptr) {
        const int64_t tiles = (n + ctx->T_tc - 1) / ctx->T_tc;
        const int grid = (int)std::min<int64_t>(tiles, ctx->grid_tc);
        CK(ctx, slr::launch_eval_tc(ctx->T_tc, grid, ctx->smem_tc, ctx->stream, ctx->nf, ctx->tcp, src, o, 0));
    } else {
        const int64_t tiles = (n + ctx->T32 - 1) / ctx->T32;
        const int grid = (int)std::min<int64_t>(tiles, ctx->grid32);
        CK(ctx, slr::launch_eval_f32(ctx->T32, ctx->NT32, grid, ctx->smem32, ctx->stream, ctx->nf, src, o, 0));
    }
    if (!on_device) {
        if (row_lo) {
            CK(ctx, cudaMemcpyAsync(row_lo, drl, (size_t)n * R * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
            CK(ctx, cudaMemcpyAsync(row_hi, drh, (size_t)n * R * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        }
        if (row_err)
            CK(ctx, cudaMemcpyAsync(row_err, dre, (size_t)n * R * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        if (cls) CK(ctx, cudaMemcpyAsync(cls, dcls, (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(ctx, cudaMemcpyAsync(ctx->h_status, ctx->status, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (*ctx->h_status & slr::kStatusTimeout)
        return fail(ctx, SLR_ETIMEOUT, "a bounded wait on the tensor core gave up; the bounds are incomplete");
    return SLR_OK;
}

int slr_leaves(slr_ctx *ctx, int64_t cap, uint64_t *codes, uint8_t *depth, uint8_t *cls, int64_t *n) {
    if (!ctx || !n) return fail(ctx, SLR_EINVAL, "null argument");
    if (!ctx->leaves_valid) return fail(ctx, SLR_ESTATE, "no leaves recorded (set record_leaves and count)");
    *n = ctx->n_leaves;
    const int64_t m = std::min(std::min(cap, ctx->n_leaves), ctx->leaf_cap_alloc);
    CK(ctx, cudaSetDevice(ctx->device));
    if (m > 0) {
        if (codes) CK(ctx, cudaMemcpy(codes, ctx->leaf_codes, (size_t)m * sizeof(uint64_t), cudaMemcpyDeviceToHost));
        if (depth) CK(ctx, cudaMemcpy(depth, ctx->leaf_depth, (size_t)m, cudaMemcpyDeviceToHost));
        if (cls) CK(ctx, cudaMemcpy(cls, ctx->leaf_cls, (size_t)m, cudaMemcpyDeviceToHost));
    }
    if (ctx->n_leaves > ctx->leaf_cap_alloc)
        return fail(ctx, SLR_EOVERFLOW, "%lld leaves exceeded leaf_cap=%lld", (long long)ctx->n_leaves,
                    (long long)ctx->leaf_cap_alloc);
    return SLR_OK;
}

int slr_schedule(slr_ctx *ctx, int D, int32_t *dims) {
    if (!ctx || !dims) return fail(ctx, SLR_EINVAL, "null argument");
    if (!ctx->split_set.empty())
        return fail(ctx, SLR_ESTATE, "the last count chose split dimensions per box (gradient split rule)");
    if (D < 0 || D > (int)ctx->sched.size())
        return fail(ctx, SLR_EINVAL, "D=%d exceeds the last count's depth %zu", D, ctx->sched.size());
    for (int t = 0; t < D; ++t) dims[t] = ctx->sched[t];
    return SLR_OK;
}

int slr_wait_selfcheck(slr_ctx *ctx, int32_t limit) {
    if (!ctx) return fail(nullptr, SLR_EINVAL, "null context");
    if (limit < 1 || limit > (1 << 20)) return fail(ctx, SLR_EINVAL, "limit %d out of range [1, 2^20]", limit);
    CK(ctx, cudaSetDevice(ctx->device));
    unsigned int *d_status = nullptr;
    CK(ctx, cudaMalloc(&d_status, sizeof(unsigned int)));
    unsigned int st = 0;
    cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof st, ctx->stream);
    if (e == cudaSuccess) e = slr::launch_wait_selfcheck(d_status, limit, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, d_status, sizeof st, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d_status);
    if (e != cudaSuccess) return fail(ctx, SLR_ECUDA, "%s", cudaGetErrorString(e));
    if (st & slr::kStatusTimeout)
        return fail(ctx, SLR_ETIMEOUT, "a bounded device wait gave up after %d polls", limit);
    return SLR_OK;
}

int slr_split_set(slr_ctx *ctx, int32_t *dims, int32_t *n) {
    if (!ctx || !dims || !n) return fail(ctx, SLR_EINVAL, "null argument");
    if (ctx->split_set.empty()) return fail(ctx, SLR_ESTATE, "the last count did not use the gradient split rule");
    for (size_t j = 0; j < ctx->split_set.size(); ++j) dims[j] = ctx->split_set[j];
    *n = (int32_t)ctx->split_set.size();
    return SLR_OK;
}

const char *slr_last_error(const slr_ctx *ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->err.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched count: many (network, box, property, depth) problems, one persistent
// kernel launch per level step for all of them, the whole step loop captured
// in one CUDA graph and replayed while the batch keeps its shape.
// ---------------------------------------------------------------------------
namespace {

struct ProblemHost {
    struct {
        int relax_mode;
    } opt;
    int K = 0;
    std::vector<int> widths;
    std::vector<std::vector<float>> W, b;
    std::vector<float> lo, hi;
    int n_clauses = 0;
    std::vector<int> rpc;
    std::vector<float> C, e;
    std::vector<uint8_t> strict;
    std::vector<int> act;                 // empty: ReLU after every hidden layer
    int depth = 0;
};

int read_problem(slr_ctx *ctx, int idx, const slr_problem &q, int relax_mode, ProblemHost &h) {
    if (q.K < 1 || q.K > slr::kMaxLayers || !q.widths || !q.W || !q.b)
        return fail(ctx, SLR_EINVAL, "problem %d: bad network", idx);
    for (int k = 0; k <= q.K; ++k)
        if (q.widths[k] < 1 || q.widths[k] > slr::kMaxWidth)
            return fail(ctx, SLR_EINVAL, "problem %d: widths[%d]=%d out of range", idx, k, q.widths[k]);
    h.opt.relax_mode = relax_mode;
    h.K = q.K;
    h.widths.assign(q.widths, q.widths + q.K + 1);
    h.W.resize(q.K);
    h.b.resize(q.K);
    for (int k = 0; k < q.K; ++k) {
        const size_t nw = (size_t)q.widths[k + 1] * q.widths[k];
        if (!q.W[k] || !q.b[k] || !finite_all(q.W[k], nw) || !finite_all(q.b[k], q.widths[k + 1]))
            return fail(ctx, SLR_EINVAL, "problem %d: bad or non-finite layer %d", idx, k);
        h.W[k].assign(q.W[k], q.W[k] + nw);
        h.b[k].assign(q.b[k], q.b[k] + q.widths[k + 1]);
    }
    const int d = q.widths[0];
    if (!q.lo || !q.hi) return fail(ctx, SLR_EINVAL, "problem %d: no box", idx);
    for (int i = 0; i < d; ++i)
        if (!std::isfinite(q.lo[i]) || !std::isfinite(q.hi[i]) || q.lo[i] > q.hi[i])
            return fail(ctx, SLR_EINVAL, "problem %d: bad box in dimension %d", idx, i);
    h.lo.assign(q.lo, q.lo + d);
    h.hi.assign(q.hi, q.hi + d);
    if (q.n_clauses < 1 || !q.rows_per_clause || !q.C || !q.e || !q.strict)
        return fail(ctx, SLR_EINVAL, "problem %d: bad property", idx);
    int R = 0;
    for (int c = 0; c < q.n_clauses; ++c) {
        if (q.rows_per_clause[c] < 1) return fail(ctx, SLR_EINVAL, "problem %d: empty clause", idx);
        R += q.rows_per_clause[c];
    }
    if (R > slr::kMaxRows) return fail(ctx, SLR_EINVAL, "problem %d: more than %d rows", idx, slr::kMaxRows);
    const int n_out = q.widths[q.K];
    if (!finite_all(q.C, (size_t)R * n_out) || !finite_all(q.e, R))
        return fail(ctx, SLR_EINVAL, "problem %d: non-finite property", idx);
    h.n_clauses = q.n_clauses;
    h.rpc.assign(q.rows_per_clause, q.rows_per_clause + q.n_clauses);
    h.C.assign(q.C, q.C + (size_t)R * n_out);
    h.e.assign(q.e, q.e + R);
    h.strict.assign(q.strict, q.strict + R);
    if (q.depth < 0 || q.depth > slr::kMaxDepth) return fail(ctx, SLR_EINVAL, "problem %d: depth out of range", idx);
    h.depth = q.depth;
    return SLR_OK;
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

namespace {

// The batched count of problems whose per-box state fits a shared-memory tile.
// Problem shape as the fused kernel sees it: inputs, rows, widest layer
// (padded to 8, the property rows counted) and widest layer input.
struct TileShape {
    int d, R, nmp, n_in;
};

TileShape problem_shape(const ProblemHost &h) {
    TileShape s{h.widths[0], (int)h.e.size(), 0, 0};
    int m = s.R;
    for (int k = 1; k < h.K; ++k) m = std::max(m, h.widths[k]);
    s.nmp = (m + 7) & ~7;
    for (int k = 0; k < h.K; ++k) s.n_in = std::max(s.n_in, h.widths[k]);
    return s;
}

// Boxes per tile of the batched kernel that fit one problem: the largest of
// 32, 16, 8, 4 whose product tiles fit two per thread and whose shared memory
// fits next to a problem's shared copies.
constexpr int kBatchTiles[] = {32, 16, 8, 4};
constexpr size_t kBatchStatic = 4096;
int batch_tile_for(const TileShape &s) {
    for (int t : kBatchTiles)
        if (slr::eval_gemm_items(t, s.d, s.nmp) <= 2 * 256 &&
            slr::eval_smem_bytes<float>(t, s.d, s.R, s.nmp, s.n_in) + kBatchStatic <= (size_t)kMaxSmem)
            return t;
    return 0;
}

int count_batch_sorted(slr_ctx *ctx, int n, const slr_problem *problems, slr_result *results);

// Problems grouped by the tile size that fits them (one persistent launch per
// group and level step): sorted by group, counted, results put back in order.
int count_batch_tile(slr_ctx *ctx, int n, const slr_problem *problems, slr_result *results) {
    std::vector<int> tile(n);
    for (int i = 0; i < n; ++i) {
        ProblemHost h;
        int rc = read_problem(ctx, i, problems[i], ctx->opt.relax_mode, h);
        if (rc) return rc;
        tile[i] = batch_tile_for(problem_shape(h));
        if (!tile[i]) return fail(ctx, SLR_EUNSUPPORTED, "problem %d is too large for the fused kernel", i);
    }
    std::vector<int> ord(n);
    for (int i = 0; i < n; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return tile[a] > tile[b]; });
    std::vector<slr_problem> sorted(n);
    std::vector<slr_result> res(n);
    for (int j = 0; j < n; ++j) sorted[j] = problems[ord[j]];
    const int rc = count_batch_sorted(ctx, n, sorted.data(), res.data());
    for (int j = 0; j < n; ++j) results[ord[j]] = res[j];
    return rc;
}

// The batch with problems sorted by tile size (runs of equal size are the groups).
int count_batch_sorted(slr_ctx *ctx, int n, const slr_problem *problems, slr_result *results) {
    CK(ctx, cudaSetDevice(ctx->device));
    const int P = n;
    std::vector<ProblemHost> ph(P);
    int rc;
    for (int i = 0; i < P; ++i)
        if ((rc = read_problem(ctx, i, problems[i], ctx->opt.relax_mode, ph[i]))) return rc;

    // host images of every problem's layers (property folded into the last)
    std::vector<HostLayers<float>> Lf(P);
    std::vector<HostLayers<double>> Ld(P);
    size_t wbytes = 0;
    for (int i = 0; i < P; ++i) {
        build_layers(&ph[i], Lf[i]);
        build_layers(&ph[i], Ld[i]);
        wbytes += layers_bytes(Lf[i]) + layers_bytes(Ld[i]);
    }
    int Dmax = 0;
    std::string key = "B" + std::to_string(ctx->opt.relax_mode) + ":" + std::to_string(ctx->opt.fp64_recheck);
    for (const ProblemHost &h : ph) {
        Dmax = std::max(Dmax, h.depth);
        key += "|" + std::to_string(h.depth) + "," + std::to_string(h.e.size()) + "," + std::to_string(h.n_clauses);
        for (int w : h.widths) key += "," + std::to_string(w);
        for (int r : h.rpc) key += "c" + std::to_string(r);
    }
    const bool recheck = ctx->opt.fp64_recheck != 0;
    BatchState *bs = ctx->batch;
    if (!bs || bs->key != key) {
        if (bs) {
            if (bs->graph) cudaGraphExecDestroy(bs->graph);
            cudaFree(bs->arena);
            if (bs->h_upload) cudaFreeHost(bs->h_upload);
            if (bs->h_ctrs) cudaFreeHost(bs->h_ctrs);
            delete bs;
            ctx->batch = nullptr;
        }
        bs = new BatchState();
        ctx->batch = bs;
        bs->key = key;
        bs->P = P;
        bs->Dmax = Dmax;
        // ---- arena layout: [upload: weights | nets32 | nets64 | roots+masks] [per problem] [step tables]
        size_t off = 0;
        const size_t o_w = off;
        off += al(wbytes);
        const size_t o_n32 = off;
        off += al((size_t)P * sizeof(slr::NetParams<float>));
        const size_t o_n64 = off;
        off += al((size_t)P * sizeof(slr::NetParams<double>));
        std::vector<size_t> o_root(P), o_masks(P), o_c0(P), o_c1(P), o_cls(P), o_near(P);
        std::vector<int64_t> cap(P);
        bs->near_cap.assign(P, 0);
        for (int i = 0; i < P; ++i) {
            const int d = ph[i].widths[0];
            o_root[i] = off;
            off += al(2 * (size_t)d * sizeof(double));
            o_masks[i] = off;
            off += al((size_t)d * sizeof(unsigned long long));
        }
        bs->upload_bytes = off;
        const size_t o_ctr = off;
        off += al((size_t)P * sizeof(slr::LevelCounters));
        const size_t o_status = off;
        off += al(sizeof(unsigned int) + sizeof(unsigned long long));
        for (int i = 0; i < P; ++i) {
            cap[i] = std::min<int64_t>((int64_t)1 << std::max(1, ph[i].depth), ctx->opt.frontier_cap);
            bs->near_cap[i] = std::max<int64_t>(1024, cap[i] / 4);
            o_c0[i] = off;
            off += al((size_t)cap[i] * 8);
            o_c1[i] = off;
            off += al((size_t)cap[i] * 8);
            o_cls[i] = off;
            off += al((size_t)cap[i]);
            o_near[i] = off;
            off += al((size_t)bs->near_cap[i] * 8);
        }
        const size_t nsteps = (size_t)Dmax + 1;
        const size_t o_sm = off;
        off += al(nsteps * P * sizeof(slr::BoxSource));
        const size_t o_sr = off;
        off += al(nsteps * P * sizeof(slr::BoxSource));
        const size_t o_om = off;
        off += al(nsteps * P * sizeof(slr::EvalOutputs));
        const size_t o_or = off;
        off += al(nsteps * P * sizeof(slr::EvalOutputs));
        const size_t o_ca = off;
        off += al(2 * (size_t)P * sizeof(slr::CompactArgs));
        const size_t o_pm = off;
        off += al(((size_t)P + 4) * sizeof(long long));   // one prefix per group (at most 4 groups)
        const size_t o_pr = off;
        off += al(((size_t)P + 1) * sizeof(long long));
        CK(ctx, cudaMalloc(&bs->arena, off));
        CK(ctx, cudaMallocHost(&bs->h_upload, bs->upload_bytes));
        CK(ctx, cudaMallocHost(&bs->h_ctrs, (size_t)P * sizeof(slr::LevelCounters)));
        unsigned char *A = (unsigned char *)bs->arena;
        bs->ctrs = (slr::LevelCounters *)(A + o_ctr);
        bs->status = (unsigned int *)(A + o_status);
        const unsigned long long *zero = (const unsigned long long *)(A + o_status + 8);

        // ---- network params (device pointers into the weights region) ------
        std::memset(bs->h_upload, 0, bs->upload_bytes);
        size_t woff = o_w;
        std::vector<slr::NetParams<float>> n32(P);
        std::vector<slr::NetParams<double>> n64(P);
        slr::BatchShape sh32{0, 0, 0, 0}, sh64{0, 0, 0, 0};
        for (int i = 0; i < P; ++i) {
            layout_params(&ph[i], Lf[i], A, bs->h_upload, woff, n32[i]);
            layout_params(&ph[i], Ld[i], A, bs->h_upload, woff, n64[i]);
            for (int k = 1; k + 1 < n64[i].K; ++k) n64[i].Wsf[k] = n32[i].Ws[k];
            for (slr::BatchShape *sh : {&sh32, &sh64}) {
                sh->nmp = std::max(sh->nmp, n32[i].n_max_pad);
                sh->d = std::max(sh->d, n32[i].d);
                sh->n_in_max = std::max(sh->n_in_max, n32[i].n_in_max);
                sh->R = std::max(sh->R, n32[i].R);
            }
        }
        std::memcpy(bs->h_upload + o_n32, n32.data(), (size_t)P * sizeof(slr::NetParams<float>));
        std::memcpy(bs->h_upload + o_n64, n64.data(), (size_t)P * sizeof(slr::NetParams<double>));

        // ---- tiles: the most boxes in flight that the largest problem allows ----
        const size_t kStatic = 4096;   // shared copies of one problem's params, source and outputs
        auto pick = [&](bool f64, int &T, size_t &smem, int &grid) {
            T = 0;
            long best = 0;
            for (int t : slr::kTileSizes) {
                const size_t sm = f64 ? slr::eval_smem_bytes<double>(t, sh64.d, sh64.R, sh64.nmp, sh64.n_in_max)
                                      : slr::eval_smem_bytes<float>(t, sh32.d, sh32.R, sh32.nmp, sh32.n_in_max);
                if (sm + kStatic > (size_t)kMaxSmem) continue;
                bool fits = true;   // each problem's contraction tiles must fit two per thread
                for (int i = 0; i < P && fits; ++i)
                    fits = slr::eval_gemm_items(t, n32[i].d, n32[i].n_max_pad) <= 2 * 256;
                if (!fits) continue;
                const int nb = f64 ? slr::eval_batch_blocks_per_sm_f64(t, sm) : slr::eval_batch_blocks_per_sm_f32(t, sm);
                if (nb <= 0) continue;
                const long score = f64 ? (long)(1000 - t) : (long)nb * t;   // FP64: short lists, small tiles
                if (score > best) {
                    best = score;
                    T = t;
                    smem = sm;
                    grid = nb * ctx->sm_count;
                }
            }
        };
        int T64 = 0, g64 = 0;
        size_t sm64 = 0;
        pick(true, T64, sm64, g64);
        // FP32 groups: runs of problems with the same tile size, each launched
        // with the shared memory and occupancy of its own largest shape
        struct Group {
            int p0, p1, T, grid;
            size_t smem;
            slr::BatchShape sh;
        };
        std::vector<Group> groups;
        bs->tile_of.assign(P, 0);
        for (int i = 0; i < P;) {
            const int t = batch_tile_for(problem_shape(ph[i]));
            int j = i;
            slr::BatchShape sh{0, 0, 0, 0};
            while (j < P && batch_tile_for(problem_shape(ph[j])) == t) {
                sh.nmp = std::max(sh.nmp, n32[j].n_max_pad);
                sh.d = std::max(sh.d, n32[j].d);
                sh.n_in_max = std::max(sh.n_in_max, n32[j].n_in_max);
                sh.R = std::max(sh.R, n32[j].R);
                ++j;
            }
            Group gr{i, j, 0, 0, 0, sh};
            // the group's combined shape may need a smaller tile than each member alone
            for (int tt : kBatchTiles) {
                if (tt > t) continue;
                const size_t sm = slr::eval_smem_bytes<float>(tt, sh.d, sh.R, sh.nmp, sh.n_in_max);
                if (sm + kStatic > (size_t)kMaxSmem) continue;
                const int nb = slr::eval_batch_blocks_per_sm_f32(tt, sm);
                if (nb <= 0) continue;
                gr.T = tt;
                gr.smem = sm;
                gr.grid = nb * ctx->sm_count;
                break;
            }
            if (!gr.T) return fail(ctx, SLR_EUNSUPPORTED, "a problem of the batch is too large for the fused kernel");
            for (int k = i; k < j; ++k) bs->tile_of[k] = gr.T;
            groups.push_back(gr);
            i = j;
        }
        if (groups.size() > 4) return fail(ctx, SLR_EUNSUPPORTED, "more than four tile groups");
        bs->T32 = groups[0].T;
        bs->T64 = T64;
        const bool rch = recheck && T64 > 0;

        // ---- per-step sources, outputs and compaction arguments ------------
        std::vector<slr::BoxSource> sm(nsteps * P), sr(nsteps * P);
        std::vector<slr::EvalOutputs> om(nsteps * P), orr(nsteps * P);
        std::vector<slr::CompactArgs> ca(2 * (size_t)P);
        for (int i = 0; i < P; ++i) {
            slr::LevelCounters *ctr = bs->ctrs + i;
            const int d = ph[i].widths[0];
            for (int par = 0; par < 2; ++par) {
                slr::CompactArgs &c = ca[(size_t)par * P + i];
                c.codes_in = (uint64_t *)(A + (par ? o_c1[i] : o_c0[i]));
                c.codes_out = (uint64_t *)(A + (par ? o_c0[i] : o_c1[i]));
                c.cls = A + o_cls[i];
                c.ctr = ctr;
                c.cap = cap[i];
                c.D = ph[i].depth;
            }
            for (size_t t = 0; t < nsteps; ++t) {
                slr::BoxSource &b = sm[t * P + i];
                b = slr::BoxSource{};
                b.mode = 0;
                b.codes = (uint64_t *)(A + ((t & 1) ? o_c1[i] : o_c0[i]));
                b.count = (int)t <= ph[i].depth ? &ctr->frontier_n[t] : zero;
                b.t = (int)t;
                b.D = std::max(ph[i].depth, (int)t);
                b.dim_mask = (unsigned long long *)(A + o_masks[i]);
                b.root_lo = (double *)(A + o_root[i]);
                b.root_w = (double *)(A + o_root[i]) + d;
                b.cap = cap[i];
                slr::BoxSource &b2 = sr[t * P + i];
                b2 = b;
                b2.index = (int64_t *)(A + o_near[i]);
                b2.index_count = (int)t <= ph[i].depth ? &ctr->near_n[t] : zero;
                b2.cap = bs->near_cap[i];
                slr::EvalOutputs &o = om[t * P + i];
                o = slr::EvalOutputs{};
                o.cls = A + o_cls[i];
                o.near_list = rch ? (int64_t *)(A + o_near[i]) : nullptr;
                o.near_count = &ctr->near_n[t];
                o.near_cap = bs->near_cap[i];
                o.tie_count = &ctr->ties;
                o.status = bs->status;
                slr::EvalOutputs &o2 = orr[t * P + i];
                o2 = slr::EvalOutputs{};
                o2.cls = A + o_cls[i];
                o2.tie_count = &ctr->ties;
                o2.status = bs->status;
            }
        }
        CK(ctx, cudaMemcpy(A + o_sm, sm.data(), sm.size() * sizeof(slr::BoxSource), cudaMemcpyHostToDevice));
        CK(ctx, cudaMemcpy(A + o_sr, sr.data(), sr.size() * sizeof(slr::BoxSource), cudaMemcpyHostToDevice));
        CK(ctx, cudaMemcpy(A + o_om, om.data(), om.size() * sizeof(slr::EvalOutputs), cudaMemcpyHostToDevice));
        CK(ctx, cudaMemcpy(A + o_or, orr.data(), orr.size() * sizeof(slr::EvalOutputs), cudaMemcpyHostToDevice));
        CK(ctx, cudaMemcpy(A + o_ca, ca.data(), ca.size() * sizeof(slr::CompactArgs), cudaMemcpyHostToDevice));

        // ---- capture the step loop ----------------------------------------
        int64_t maxcap = 1;
        for (int i = 0; i < P; ++i) maxcap = std::max(maxcap, cap[i]);
        const int bpp = (int)std::max<int64_t>(1, std::min<int64_t>(128, maxcap / 32768));
        const slr::NetParams<float> *dn32 = (const slr::NetParams<float> *)(A + o_n32);
        const slr::NetParams<double> *dn64 = (const slr::NetParams<double> *)(A + o_n64);
        long long *pm = (long long *)(A + o_pm);
        long long *pr = (long long *)(A + o_pr);
        cudaGraph_t g;
        CK(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        int64_t L = 0;
        cudaError_t ce = cudaMemsetAsync(bs->ctrs, 0, (size_t)P * sizeof(slr::LevelCounters), ctx->stream);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(bs->status, 0, 16, ctx->stream);
        if (ce == cudaSuccess) ce = slr::launch_init_batch((const slr::CompactArgs *)(A + o_ca), P, ctx->stream), ++L;
        while (ce == cudaSuccess && bs->step_ev.size() < nsteps) {
            cudaEvent_t e;
            ce = cudaEventCreate(&e);
            if (ce == cudaSuccess) bs->step_ev.push_back(e);
        }
        for (size_t t = 0; t < nsteps && ce == cudaSuccess; ++t) {
            const slr::BoxSource *s_m = (const slr::BoxSource *)(A + o_sm) + t * P;
            const slr::BoxSource *s_r = (const slr::BoxSource *)(A + o_sr) + t * P;
            const slr::EvalOutputs *o_m = (const slr::EvalOutputs *)(A + o_om) + t * P;
            const slr::EvalOutputs *o_r = (const slr::EvalOutputs *)(A + o_or) + t * P;
            for (size_t gi = 0; gi < groups.size() && ce == cudaSuccess; ++gi) {
                const Group &gr = groups[gi];
                long long *pg = pm + gr.p0 + gi;
                ce = slr::launch_tile_prefix(s_m + gr.p0, gr.p1 - gr.p0, gr.T, pg, ctx->stream);
                if (ce == cudaSuccess)
                    ce = slr::launch_eval_batch_f32(gr.T, gr.grid, gr.smem, ctx->stream, dn32 + gr.p0, s_m + gr.p0,
                                                    o_m + gr.p0, gr.p1 - gr.p0, pg, gr.sh, 0);
                L += 2;
            }
            if (rch && ce == cudaSuccess) {
                ce = slr::launch_tile_prefix(s_r, P, T64, pr, ctx->stream);
                if (ce == cudaSuccess)
                    ce = slr::launch_eval_batch_f64(T64, g64, sm64, ctx->stream, dn64, s_r, o_r, P, pr, sh64, 1);
                L += 2;
            }
            if (ce == cudaSuccess)
                ce = slr::launch_compact_batch((const slr::CompactArgs *)(A + o_ca) + (t & 1) * P, P, (int)t, bs->status,
                                               bpp, ctx->stream);
            ++L;
            // an event-record node: the end of level step t (per-problem completion times)
            if (ce == cudaSuccess) ce = cudaEventRecordWithFlags(bs->step_ev[t], ctx->stream, cudaEventRecordExternal);
        }
        const cudaError_t ee = cudaStreamEndCapture(ctx->stream, &g);
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "capturing the batched count");
        if (ee != cudaSuccess) return cuda_fail(ctx, ee, "cudaStreamEndCapture");
        ce = cudaGraphInstantiate(&bs->graph, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaGraphInstantiate");
        bs->launches = L;
    }

    // ---- data of this call: weights, params, roots and split masks ----------
    unsigned char *A = (unsigned char *)bs->arena;
    {
        size_t woff = 0;
        std::vector<slr::NetParams<float>> n32(P);
        std::vector<slr::NetParams<double>> n64(P);
        for (int i = 0; i < P; ++i) {
            layout_params(&ph[i], Lf[i], A, bs->h_upload, woff, n32[i]);
            layout_params(&ph[i], Ld[i], A, bs->h_upload, woff, n64[i]);
            for (int k = 1; k + 1 < n64[i].K; ++k) n64[i].Wsf[k] = n32[i].Ws[k];
        }
        const size_t o_n32 = al(wbytes);
        const size_t o_n64 = o_n32 + al((size_t)P * sizeof(slr::NetParams<float>));
        std::memcpy(bs->h_upload + o_n32, n32.data(), (size_t)P * sizeof(slr::NetParams<float>));
        std::memcpy(bs->h_upload + o_n64, n64.data(), (size_t)P * sizeof(slr::NetParams<double>));
        size_t off = o_n64 + al((size_t)P * sizeof(slr::NetParams<double>));
        for (int i = 0; i < P; ++i) {
            const int d = ph[i].widths[0];
            const int D = ph[i].depth;
            double *root = (double *)(bs->h_upload + off);
            unsigned long long *masks = (unsigned long long *)(bs->h_upload + off + al(2 * (size_t)d * sizeof(double)));
            std::vector<int> cnt(d, 0);
            for (int k = 0; k < d; ++k) {
                root[k] = (double)ph[i].lo[k];
                root[d + k] = (double)ph[i].hi[k] - (double)ph[i].lo[k];
                masks[k] = 0ull;
            }
            for (int t = 0; t < D; ++t) {   // widest side first, ties to the lowest index
                int best = 0;
                double bw = -1.0;
                for (int k = 0; k < d; ++k) {
                    const double w = std::ldexp(root[d + k], -cnt[k]);
                    if (w > bw) {
                        bw = w;
                        best = k;
                    }
                }
                cnt[best] += 1;
                masks[best] |= 1ull << (D - 1 - t);
            }
            off += al(2 * (size_t)d * sizeof(double)) + al((size_t)d * sizeof(unsigned long long));
        }
    }
    CK(ctx, cudaMemcpyAsync(A, bs->h_upload, bs->upload_bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
    CK(ctx, cudaGraphLaunch(bs->graph, ctx->stream));
    CK(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
    unsigned int st = 0;
    CK(ctx, cudaMemcpyAsync(bs->h_ctrs, bs->ctrs, (size_t)P * sizeof(slr::LevelCounters), cudaMemcpyDeviceToHost,
                            ctx->stream));
    CK(ctx, cudaMemcpyAsync(&st, bs->status, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    std::vector<float> step_ms(bs->step_ev.size(), 0.f);
    for (size_t t = 0; t < step_ms.size() && t < (size_t)bs->Dmax + 1; ++t)
        cudaEventElapsedTime(&step_ms[t], ctx->ev0, bs->step_ev[t]);
    (void)cudaGetLastError();
    for (int i = 0; i < P; ++i) {
        const slr::LevelCounters &c = bs->h_ctrs[i];
        slr_result &out = results[i];
        std::memset(&out, 0, sizeof out);
        const int D = ph[i].depth;
        out.unsafe_lo = c.unsafe_lo;
        out.unsafe_hi = c.unsafe_lo + c.undecided_at_D;
        out.boxes = c.boxes;
        out.tie_leaves = c.ties;
        out.depth = D;
        unsigned long long rech = 0;
        for (int t = 0; t <= D; ++t) {
            out.level_boxes[t] = c.level_boxes[t];
            out.level_safe[t] = c.level_safe[t];
            out.level_unsafe[t] = c.level_unsafe[t];
            out.level_undecided[t] = c.level_undecided[t];
            rech += std::min<unsigned long long>(c.near_n[t], (unsigned long long)bs->near_cap[i]);
            if (c.level_boxes[t]) out.levels = t + 1;
        }
        out.rechecked = recheck ? rech : 0;
        out.rechecked_fp64 = out.rechecked;
        out.device_ms = ms;              // the whole batch
        out.launches = bs->launches;
        out.h2d_bytes = (int64_t)bs->upload_bytes;
        out.d2h_bytes = (int64_t)((size_t)P * sizeof(slr::LevelCounters) + sizeof st);
        out.tile_boxes = bs->tile_of[i];
        out.tile_threads = 256;
        // done at the end of the step of its last level (its depth cap, or
        // earlier when its frontier empties)
        const int last = std::max(0, out.levels - 1);
        out.completion_ms = (size_t)last < step_ms.size() ? step_ms[last] : ms;
    }
    if (st & slr::kStatusOverflow) return fail(ctx, SLR_EOVERFLOW, "a problem's level exceeded its frontier capacity");
    if (st & slr::kStatusNearOverflow) return fail(ctx, SLR_EOVERFLOW, "an FP64 re-check list overflowed");
    return SLR_OK;
}

}  // namespace

// Whether a problem's per-box state fits the batched tile kernel (its
// smallest tile, two product tiles per thread).
static bool batch_tile_fits(const slr_problem &q) {
    if (q.K < 1 || q.K > slr::kMaxLayers || !q.widths || !q.rows_per_clause) return true;   // validated later
    int R = 0;
    for (int c = 0; c < q.n_clauses; ++c) R += q.rows_per_clause[c];
    const int d = q.widths[0];
    int nmax = R, nin = d;
    for (int k = 1; k < q.K; ++k) {
        nmax = std::max(nmax, q.widths[k]);
        nin = std::max(nin, q.widths[k]);
    }
    const int nmp = (nmax + 7) & ~7;
    return slr::eval_gemm_items(4, d, nmp) <= 2 * 256 &&
           slr::eval_smem_bytes<float>(4, d, R, nmp, nin) + kBatchStatic <= (size_t)kMaxSmem;
}

extern "C" int slr_count_batch(slr_ctx *ctx, int n, const slr_problem *problems, slr_result *results) {
    if (!ctx) return fail(nullptr, SLR_EINVAL, "null context");
    if (n < 1 || n > 65535 || !problems || !results) return fail(ctx, SLR_EINVAL, "bad batch arguments");
    if (ctx->opt.split_rule != SLR_SPLIT_WIDEST)
        return fail(ctx, SLR_EUNSUPPORTED, "batched counts split the widest side; the gradient rule runs in slr_count");
    if (ctx->opt.shard_count > 1) return fail(ctx, SLR_EUNSUPPORTED, "batched counts are not sharded");
    std::vector<int> tile, wide;
    for (int i = 0; i < n; ++i) (batch_tile_fits(problems[i]) ? tile : wide).push_back(i);
    if (wide.empty()) return count_batch_tile(ctx, n, problems, results);
    int rc;
    // problems that fit a tile: one persistent launch per level step together
    if (!tile.empty()) {
        std::vector<slr_problem> sub(tile.size());
        std::vector<slr_result> res(tile.size());
        for (size_t j = 0; j < tile.size(); ++j) sub[j] = problems[tile[j]];
        if ((rc = count_batch_tile(ctx, (int)sub.size(), sub.data(), res.data()))) return rc;
        for (size_t j = 0; j < tile.size(); ++j) results[tile[j]] = res[j];
    }
    // wider problems: one wide-path count each, kWideWorkers at a time, each
    // worker a host thread with a helper context and stream of its own (a
    // wide count reads its level sizes on the host, so one problem alone
    // leaves the GPU idle between its launches)
    constexpr int kWideWorkers = 4;
    const int K = std::min<int>(kWideWorkers, (int)wide.size());
    while ((int)ctx->wide_helpers.size() < K) {
        slr_ctx *h = nullptr;
        if ((rc = slr_create(&h, ctx->device, nullptr)))
            return fail(ctx, rc, "wide helper context: %s", slr_last_error(nullptr));
        ctx->wide_helpers.push_back(h);
    }
    const double tile_ms = tile.empty() ? 0.0 : results[tile[0]].device_ms;
    slr_options o = ctx->opt;
    o.wide = 1;
    o.alpha_steps = 0;
    o.record_leaves = 0;
    o.tile_boxes = o.tile_threads = 0;
    for (int w = 0; w < K; ++w)
        if ((rc = slr_set_options(ctx->wide_helpers[w], &o)))
            return fail(ctx, rc, "problem batch: %s", slr_last_error(ctx->wide_helpers[w]));
    // the wide phase starts when the context stream's work is done
    cudaEvent_t ev_start = nullptr;
    std::vector<cudaEvent_t> ev_end(wide.size(), nullptr);
    cudaError_t ce = cudaEventCreate(&ev_start);
    for (size_t j = 0; j < wide.size() && ce == cudaSuccess; ++j) ce = cudaEventCreate(&ev_end[j]);
    if (ce == cudaSuccess) ce = cudaEventRecord(ev_start, ctx->stream);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(ev_start);
    std::atomic<int> next{0};
    std::vector<int> wrc(K, SLR_OK);
    std::vector<std::string> wmsg(K);
    auto worker = [&](int w) {
        slr_ctx *h = ctx->wide_helpers[w];
        cudaSetDevice(ctx->device);
        for (int j = next.fetch_add(1); j < (int)wide.size(); j = next.fetch_add(1)) {
            const int i = wide[j];
            const slr_problem &q = problems[i];
            int r = SLR_OK;
            if ((r = slr_load_network(h, q.K, q.widths, q.W, q.b)) || (r = slr_set_box(h, q.widths[0], q.lo, q.hi)) ||
                (r = slr_set_property(h, q.n_clauses, q.rows_per_clause, q.widths[q.K], q.C, q.e, q.strict)) ||
                (r = slr_count(h, q.depth, &results[i]))) {
                wrc[w] = r;
                wmsg[w] = "problem " + std::to_string(i) + ": " + slr_last_error(h);
                next.store((int)wide.size());   // the others stop at their next problem
                return;
            }
            if (cudaEventRecord(ev_end[j], h->stream) != cudaSuccess || cudaEventSynchronize(ev_end[j]) != cudaSuccess) {
                wrc[w] = SLR_ECUDA;
                wmsg[w] = "problem " + std::to_string(i) + ": completion event";
                next.store((int)wide.size());
                return;
            }
        }
    };
    if (ce == cudaSuccess) {
        std::vector<std::thread> th;
        for (int w = 0; w < K; ++w) th.emplace_back(worker, w);
        for (std::thread &t : th) t.join();
    }
    double wide_ms = 0.0;
    for (int w = 0; w < K && rc == SLR_OK && ce == cudaSuccess; ++w)
        if (wrc[w] != SLR_OK) rc = fail(ctx, wrc[w], "%s", wmsg[w].c_str());
    for (size_t j = 0; j < wide.size() && rc == SLR_OK && ce == cudaSuccess; ++j) {
        float ms = 0.f;
        ce = cudaEventElapsedTime(&ms, ev_start, ev_end[j]);
        results[wide[j]].completion_ms = tile_ms + ms;
        wide_ms = std::max(wide_ms, (double)ms);
    }
    for (cudaEvent_t e : ev_end)
        if (e) cudaEventDestroy(e);
    if (ev_start) cudaEventDestroy(ev_start);
    if (rc != SLR_OK) return rc;
    if (ce != cudaSuccess) return fail(ctx, SLR_ECUDA, "batch of wide problems: %s", cudaGetErrorString(ce));
    // every result reports the whole batch's device time
    for (int i = 0; i < n; ++i) results[i].device_ms = tile_ms + wide_ms;
    return SLR_OK;
}

// ---------------------------------------------------------------------------
// Lower-slope optimisation: the adjoint of the SLR pass and projected Adam.
// ---------------------------------------------------------------------------
namespace {

constexpr float kBeta1 = 0.9f, kBeta2 = 0.999f, kAdamEps = 1e-8f;

slr::AdjArgs adj_base(const slr_ctx *ctx) {
    slr::AdjArgs a{};
    a.net = ctx->nf;
    a.H = ctx->H;
    a.n_max = ctx->adj_nmax;
    a.nck = ctx->adj_nck;
    a.boxes_per_cta = ctx->adj_boxes;
    a.gscratch = ctx->adj_gmem ? (float *)ctx->adj_scratch : nullptr;
    a.Cprop = ctx->dC;
    a.n_out = ctx->widths[ctx->K];
    a.lr = 0.f;
    a.beta1 = kBeta1;
    a.beta2 = kBeta2;
    a.eps = kAdamEps;
    return a;
}

void adam_step(slr::AdjArgs &a, int t, float lr) {
    a.adam_t = t;
    a.lr = lr;
    a.beta1_t = (float)std::pow((double)kBeta1, t);
    a.beta2_t = (float)std::pow((double)kBeta2, t);
}

int check_adjoint(slr_ctx *ctx) {
    if (ctx->opt.relax_mode != SLR_RELAX_NEURIFY)
        return fail(ctx, SLR_EUNSUPPORTED, "the adjoint needs relax mode NEURIFY");
    for (int a : ctx->act)
        if (a != SLR_ACT_RELU)
            return fail(ctx, SLR_EUNSUPPORTED, "slopes, the adjoint and the gradient split rule need ReLU networks");
    if (ctx->adj_grid <= 0)
        return fail(ctx, SLR_EUNSUPPORTED, "network too large for the adjoint kernel (%zu bytes of shared memory)",
                    ctx->adj_smem);
    if (ctx->adj_gmem) {
        slr::AdjArgs a = adj_base(ctx);
        const size_t need = slr::adjoint_box_bytes(a) * (size_t)ctx->adj_grid;
        if (ctx->adj_scratch_bytes < need) {
            cudaFree(ctx->adj_scratch);
            ctx->adj_scratch = nullptr;
            ctx->adj_scratch_bytes = 0;
            CK(ctx, cudaMalloc(&ctx->adj_scratch, need));
            ctx->adj_scratch_bytes = need;
        }
    }
    return SLR_OK;
}

// Device regions of a slope optimisation over `cap` boxes.
struct AlphaBuffers {
    float *alpha, *m, *v, *lo_new, *hi_new, *lo_best, *hi_best;
    int8_t *dir;
    int64_t *list, *list2;
    unsigned long long *n_all;    // boxes gathered before the margin filter
};

size_t alpha_bytes(int64_t cap, int64_t H, int R) {
    return align_up((size_t)cap * H * sizeof(float)) * 3 + align_up((size_t)cap * R * sizeof(float)) * 4 +
           align_up((size_t)cap) + 2 * align_up((size_t)cap * sizeof(int64_t)) + align_up(sizeof(unsigned long long));
}

AlphaBuffers carve_alpha(void *base, int64_t cap, int64_t H, int R) {
    unsigned char *p = (unsigned char *)base;
    AlphaBuffers b;
    auto take = [&](size_t bytes) {
        unsigned char *q = p;
        p += align_up(bytes);
        return q;
    };
    b.alpha = (float *)take((size_t)cap * H * sizeof(float));
    b.m = (float *)take((size_t)cap * H * sizeof(float));
    b.v = (float *)take((size_t)cap * H * sizeof(float));
    b.lo_new = (float *)take((size_t)cap * R * sizeof(float));
    b.hi_new = (float *)take((size_t)cap * R * sizeof(float));
    b.lo_best = (float *)take((size_t)cap * R * sizeof(float));
    b.hi_best = (float *)take((size_t)cap * R * sizeof(float));
    b.dir = (int8_t *)take((size_t)cap);
    b.list = (int64_t *)take((size_t)cap * sizeof(int64_t));
    b.list2 = (int64_t *)take((size_t)cap * sizeof(int64_t));
    b.n_all = (unsigned long long *)take(sizeof(unsigned long long));
    return b;
}

// Sound bounds at the slopes in `alpha` (NULL: u/(u-l)) for positions of `src`,
// written by position.
int eval_by_position(slr_ctx *ctx, slr::BoxSource src, const float *alpha, float *lo, float *hi, int64_t n_hint) {
    src.alpha = alpha;
    src.alpha_ld = ctx->H;
    slr::EvalOutputs o{};
    o.row_lo = lo;
    o.row_hi = hi;
    o.by_position = 1;
    o.status = ctx->status;
    if (ctx->wide) {
        // the chunk loop needs the number of positions on the host
        int64_t n = src.n_explicit;
        if (src.index != nullptr || src.mode == 0) {
            unsigned long long c = 0;
            CK(ctx, cudaMemcpyAsync(&c, src.index != nullptr ? src.index_count : src.count, sizeof c,
                                    cudaMemcpyDeviceToHost, ctx->stream));
            CK(ctx, cudaStreamSynchronize(ctx->stream));
            n = (int64_t)c;
        }
        n = std::min<int64_t>(n, src.cap);
        int64_t launches = 0;
        return n > 0 ? run_wide(ctx, src, n, o, &launches) : SLR_OK;
    }
    const int64_t tiles = (n_hint + ctx->T32 - 1) / ctx->T32;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, ctx->grid32));
    CK(ctx, slr::launch_eval_f32(ctx->T32, ctx->NT32, grid, ctx->smem32, ctx->stream, ctx->nf, src, o, 0));
    return SLR_OK;
}

// `steps` projected-Adam steps on the slopes of the boxes of `src` (positions
// 0..cap-1, count on the device when `count` is set), keeping in (lo_best,
// hi_best) the intersection of the sound bounds of every step, starting with
// the slopes u/(u-l); class bytes go to cls_pos (by position) and/or
// cls_idx (through src.index).  Returns the number of kernel launches in *launches.
int optimise_slopes(slr_ctx *ctx, const slr::BoxSource &src, int64_t cap, const unsigned long long *count,
                    const AlphaBuffers &b, int steps, float lr, uint8_t *cls_pos, uint8_t *cls_idx,
                    unsigned long long *decided, bool want_alpha, int64_t *launches) {
    int rc;
    if ((rc = eval_by_position(ctx, src, nullptr, b.lo_new, b.hi_new, cap))) return rc;
    CK(ctx, slr::launch_merge_bounds(ctx->nf, cap, count, b.lo_new, b.hi_new, b.lo_best, b.hi_best,
                                     steps == 0 ? cls_pos : nullptr, steps == 0 ? cls_idx : nullptr, src.index, 1,
                                     steps == 0 ? decided : nullptr, ctx->stream));
    *launches += 2;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((cap + ctx->adj_boxes - 1) / ctx->adj_boxes,
                                                                 ctx->adj_grid));
    slr::AdjArgs a = adj_base(ctx);
    a.src = src;
    a.n = cap;
    a.count = count;
    a.alpha = b.alpha;
    a.dir = b.dir;
    a.adam_m = b.m;
    a.adam_v = b.v;
    if (steps == 0 && want_alpha) {
        a.alpha_mode = slr::kAlphaInit;
        if ((rc = run_adjoint(ctx, a, grid, launches))) return rc;
    }
    for (int t = 1; t <= steps; ++t) {
        a.alpha_mode = t == 1 ? slr::kAlphaInit : slr::kAlphaFree;
        adam_step(a, t, lr);
        if ((rc = run_adjoint(ctx, a, grid, launches))) return rc;
        if ((rc = eval_by_position(ctx, src, b.alpha, b.lo_new, b.hi_new, cap))) return rc;
        const bool last = t == steps;
        CK(ctx, slr::launch_merge_bounds(ctx->nf, cap, count, b.lo_new, b.hi_new, b.lo_best, b.hi_best,
                                         last ? cls_pos : nullptr, last ? cls_idx : nullptr, src.index, 0,
                                         last ? decided : nullptr, ctx->stream));
        *launches += 3;
    }
    return SLR_OK;
}

int ensure_alpha_buf(slr_ctx *ctx, size_t bytes) {
    if (ctx->alpha_buf_bytes >= bytes) return SLR_OK;
    cudaFree(ctx->alpha_buf);
    ctx->alpha_buf = nullptr;
    ctx->alpha_buf_bytes = 0;
    CK(ctx, cudaMalloc(&ctx->alpha_buf, bytes));
    ctx->alpha_buf_bytes = bytes;
    return SLR_OK;
}

}  // namespace

// Slope optimisation of the boxes a level of a count leaves UNDECIDED.
int slr_internal_alpha_level(slr_ctx *ctx, const slr::BoxSource &frontier, int t, int64_t *launches) {
    const int64_t cap = std::min<int64_t>(ctx->opt.alpha_cap, ctx->cap);
    const int R = (int)ctx->e.size();
    int rc = ensure_alpha_buf(ctx, alpha_bytes(cap, ctx->H, R));
    if (rc) return rc;
    if (!ctx->alpha_ctr) CK(ctx, cudaMalloc(&ctx->alpha_ctr, 2 * (slr::kMaxDepth + 2) * sizeof(unsigned long long)));
    const AlphaBuffers b = carve_alpha(ctx->alpha_buf, cap, ctx->H, R);
    unsigned long long *list_n = ctx->alpha_ctr + 2 * t;
    slr::BoxSource src = frontier;
    src.cap = cap;
    // (the gradient split rule takes every UNDECIDED box's split from its
    // optimised slopes, so there every box is optimised)
    if (ctx->opt.alpha_margin > 0.f && ctx->opt.split_rule != SLR_SPLIT_GRADIENT) {
        // only boxes whose decision gap at the fixed slopes is within
        // alpha_margin of their widest row bound: the rest are far from any
        // decision that tighter slopes could reach
        CK(ctx, cudaMemsetAsync(b.n_all, 0, sizeof(unsigned long long), ctx->stream));
        CK(ctx, slr::launch_gather_undecided(ctx->cls, frontier.count, ctx->cap, b.list2, b.n_all, cap,
                                             std::max(1, ctx->sm_count * 4), ctx->stream));
        src.index = b.list2;
        src.index_count = b.n_all;
        if ((rc = eval_by_position(ctx, src, nullptr, b.lo_new, b.hi_new, cap))) return rc;
        CK(ctx, slr::launch_margin_filter(ctx->nf, b.lo_new, b.hi_new, b.n_all, cap, b.list2, b.list, list_n,
                                          ctx->opt.alpha_margin, std::max(1, ctx->sm_count * 4), ctx->stream));
        *launches += 3;
    } else {
        CK(ctx, slr::launch_gather_undecided(ctx->cls, frontier.count, ctx->cap, b.list, list_n, cap,
                                             std::max(1, ctx->sm_count * 4), ctx->stream));
        *launches += 1;
    }
    src.index = b.list;
    src.index_count = list_n;
    return optimise_slopes(ctx, src, cap, list_n, b, ctx->opt.alpha_steps, ctx->opt.alpha_lr, nullptr, ctx->cls,
                           list_n + 1, false, launches);
}

// Gradient split rule, the split set: the (at most kSplitSetMax) input
// dimensions with the largest |dM/dr_i| w_i at the root box, M the decision
// loss at the fixed slopes u/(u-l), r the box radius and w the root widths;
// ties go to the lowest index.  Kept in ascending order: a code's nibble is a
// position in it.
int slr_internal_split_root(slr_ctx *ctx, const slr::BoxSource &root, int64_t *launches) {
    const int d = ctx->widths[0];
    const size_t grad_off = align_up((size_t)d) + align_up(slr::kSplitSetMax * sizeof(int));
    if (!ctx->split_buf) CK(ctx, cudaMalloc(&ctx->split_buf, grad_off + (size_t)d * sizeof(float)));
    int8_t *split_of = (int8_t *)ctx->split_buf;
    int *dims_dev = (int *)((unsigned char *)ctx->split_buf + align_up((size_t)d));
    float *grad = (float *)((unsigned char *)ctx->split_buf + grad_off);
    slr::AdjArgs a = adj_base(ctx);
    a.src = root;
    a.n = 1;
    a.count = nullptr;
    a.alpha_mode = slr::kAlphaDefault;
    a.d_r = grad;
    int rc = run_adjoint(ctx, a, 1, launches);
    if (rc) return rc;
    std::vector<float> g(d);
    CK(ctx, cudaMemcpyAsync(g.data(), grad, (size_t)d * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<int> order(d);
    std::vector<double> score(d);
    for (int i = 0; i < d; ++i) {
        order[i] = i;
        const double s = std::fabs((double)g[i]) * ((double)ctx->hi[i] - (double)ctx->lo[i]);
        score[i] = std::isfinite(s) ? s : -1.0;
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return score[x] > score[y]; });
    const int ns = std::min(d, slr::kSplitSetMax);
    std::vector<int> set(order.begin(), order.begin() + ns);
    std::sort(set.begin(), set.end());
    std::vector<int8_t> of(d, (int8_t)-1);
    for (int j = 0; j < ns; ++j) of[set[j]] = (int8_t)j;
    CK(ctx, cudaMemcpy(split_of, of.data(), (size_t)d, cudaMemcpyHostToDevice));
    CK(ctx, cudaMemcpy(dims_dev, set.data(), (size_t)ns * sizeof(int), cudaMemcpyHostToDevice));
    ctx->split_set = set;
    return SLR_OK;
}

// Gradient split rule, one level: each box the level leaves UNDECIDED (after
// any slope steps) takes the dimension of the split set with the largest
// |dM/dr_i| r_i, the gradient taken at its final slopes; the choice goes into
// the nibble of its code for this level.
int slr_internal_split_level(slr_ctx *ctx, const slr::BoxSource &frontier, int t, bool slopes, int64_t *launches) {
    const int64_t cap = std::min<int64_t>(ctx->opt.alpha_cap, ctx->cap);
    const int R = (int)ctx->e.size();
    unsigned long long *list_n = ctx->alpha_ctr + 2 * t;
    slr::AdjArgs a = adj_base(ctx);
    int64_t *list;
    if (slopes) {
        // the boxes of the level's slope optimisation, their slopes and directions
        const AlphaBuffers b = carve_alpha(ctx->alpha_buf, cap, ctx->H, R);
        list = b.list;
        a.alpha_mode = slr::kAlphaFree;
        a.alpha = b.alpha;
        a.dir = b.dir;
    } else {
        int rc = ensure_alpha_buf(ctx, align_up((size_t)cap * sizeof(int64_t)));
        if (rc) return rc;
        list = (int64_t *)ctx->alpha_buf;
        CK(ctx, slr::launch_gather_undecided(ctx->cls, frontier.count, ctx->cap, list, list_n, cap,
                                             std::max(1, ctx->sm_count * 4), ctx->stream));
        *launches += 1;
        a.alpha_mode = slr::kAlphaDefault;
    }
    slr::BoxSource src = frontier;
    src.index = list;
    src.index_count = list_n;
    src.cap = cap;
    a.src = src;
    a.n = cap;
    a.count = list_n;
    a.split_codes = ctx->codes[t & 1];
    a.split_cls = ctx->cls;
    a.split_dims = (const int *)((unsigned char *)ctx->split_buf + align_up((size_t)ctx->widths[0]));
    a.n_split = (int)ctx->split_set.size();
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((cap + ctx->adj_boxes - 1) / ctx->adj_boxes,
                                                                 ctx->adj_grid));
    return run_adjoint(ctx, a, grid, launches);
}

extern "C" {

int slr_alpha_width(slr_ctx *ctx, int64_t *H) {
    if (!ctx || !H) return fail(ctx, SLR_EINVAL, "null argument");
    if (!ctx->has_net) return fail(ctx, SLR_ESTATE, "network must be set");
    int64_t h = 0;
    for (int k = 1; k < ctx->K; ++k) h += ctx->widths[k];
    *H = h;
    return SLR_OK;
}

int slr_margin_backward(slr_ctx *ctx, int64_t n, const float *box_lo, const float *box_hi, const float *alpha,
                        const float *g_lo, const float *g_hi, float *row_lo, float *row_hi, float *d_alpha,
                        float *d_box_lo, float *d_box_hi, float *const *d_W, float *const *d_b, int on_device) {
    if (!ctx) return fail(nullptr, SLR_EINVAL, "null context");
    if (!ctx->has_net || !ctx->has_prop) return fail(ctx, SLR_ESTATE, "network and property must be set");
    if (n < 0 || (n > 0 && (!box_lo || !box_hi || !g_lo || !g_hi))) return fail(ctx, SLR_EINVAL, "bad arguments");
    if ((row_lo == nullptr) != (row_hi == nullptr)) return fail(ctx, SLR_EINVAL, "row_lo and row_hi go together");
    if ((d_box_lo == nullptr) != (d_box_hi == nullptr))
        return fail(ctx, SLR_EINVAL, "d_box_lo and d_box_hi go together");
    const int K = ctx->K;
    bool want_w = d_W != nullptr || d_b != nullptr;
    if (want_w) {
        if (!d_W || !d_b) return fail(ctx, SLR_EINVAL, "d_W and d_b go together");
        for (int k = 0; k < K; ++k)
            if (!d_W[k] || !d_b[k]) return fail(ctx, SLR_EINVAL, "d_W[%d] or d_b[%d] is NULL", k, k);
    }
    CK(ctx, cudaSetDevice(ctx->device));
    int rc = prepare_device(ctx);
    if (rc) return rc;
    if ((rc = check_adjoint(ctx))) return rc;
    const int d = ctx->widths[0];
    const int R = (int)ctx->e.size();
    const int64_t H = ctx->H;
    size_t wsz = 0;
    std::vector<size_t> woff(K), boff(K);
    for (int k = 0; k < K; ++k) {
        woff[k] = wsz;
        wsz += align_up((size_t)ctx->widths[k + 1] * ctx->widths[k] * sizeof(float));
        boff[k] = wsz;
        wsz += align_up((size_t)ctx->widths[k + 1] * sizeof(float));
    }
    // device views: inputs, outputs and the weight-gradient accumulators
    const size_t s_box = align_up((size_t)n * d * sizeof(float)), s_al = align_up((size_t)n * H * sizeof(float));
    const size_t s_row = align_up((size_t)n * R * sizeof(float));
    const size_t need = on_device ? 0 : 4 * s_box + 2 * s_al + 4 * s_row + (want_w ? wsz : 0);
    if (!on_device && n > 0 && (rc = check_boxes(ctx, n, d, box_lo, box_hi))) return rc;
    if (need && (rc = ensure_scratch(ctx, need))) return rc;
    unsigned char *p = (unsigned char *)ctx->scratch;
    auto take = [&](size_t bytes) {
        unsigned char *q = p;
        p += bytes;
        return q;
    };
    const float *dlo = box_lo, *dhi = box_hi, *dal = alpha, *dgl = g_lo, *dgh = g_hi;
    float *drl = row_lo, *drh = row_hi, *dda = d_alpha, *ddl = d_box_lo, *ddh = d_box_hi;
    float *dW[slr::kMaxLayers] = {}, *db[slr::kMaxLayers] = {};
    if (!on_device) {
        float *t0 = (float *)take(s_box), *t1 = (float *)take(s_box);
        float *t2 = (float *)take(s_al), *t3 = (float *)take(s_row), *t4 = (float *)take(s_row);
        drl = row_lo ? (float *)take(s_row) : nullptr;
        drh = row_lo ? (float *)take(s_row) : nullptr;
        dda = d_alpha ? (float *)take(s_al) : nullptr;
        ddl = d_box_lo ? (float *)take(s_box) : nullptr;
        ddh = d_box_lo ? (float *)take(s_box) : nullptr;
        if (n > 0) {
            CK(ctx, cudaMemcpyAsync(t0, box_lo, (size_t)n * d * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
            CK(ctx, cudaMemcpyAsync(t1, box_hi, (size_t)n * d * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
            if (alpha)
                CK(ctx, cudaMemcpyAsync(t2, alpha, (size_t)n * H * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
            CK(ctx, cudaMemcpyAsync(t3, g_lo, (size_t)n * R * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
            CK(ctx, cudaMemcpyAsync(t4, g_hi, (size_t)n * R * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
        }
        dlo = t0;
        dhi = t1;
        dal = alpha ? t2 : nullptr;
        dgl = t3;
        dgh = t4;
        if (want_w) {
            unsigned char *wbase = take(wsz);
            for (int k = 0; k < K; ++k) {
                dW[k] = (float *)(wbase + woff[k]);
                db[k] = (float *)(wbase + boff[k]);
            }
            CK(ctx, cudaMemsetAsync(wbase, 0, wsz, ctx->stream));
        }
    } else if (want_w) {
        for (int k = 0; k < K; ++k) {
            dW[k] = d_W[k];
            db[k] = d_b[k];
            CK(ctx, cudaMemsetAsync(dW[k], 0, (size_t)ctx->widths[k + 1] * ctx->widths[k] * sizeof(float), ctx->stream));
            CK(ctx, cudaMemsetAsync(db[k], 0, (size_t)ctx->widths[k + 1] * sizeof(float), ctx->stream));
        }
    }
    if (n > 0) {
        slr::AdjArgs a = adj_base(ctx);
        a.src.mode = 1;
        a.src.n_explicit = n;
        a.src.lo = dlo;
        a.src.hi = dhi;
        a.src.cap = n;
        a.n = n;
        a.alpha_mode = alpha ? slr::kAlphaFree : slr::kAlphaDefault;
        a.alpha = const_cast<float *>(dal);
        a.g_lo = dgl;
        a.g_hi = dgh;
        a.row_lo = drl;
        a.row_hi = drh;
        a.d_alpha = dda;
        a.d_lo = ddl;
        a.d_hi = ddh;
        for (int k = 0; k < K; ++k) {
            a.dW[k] = dW[k];
            a.db[k] = db[k];
        }
        const int grid = (int)std::min<int64_t>((n + ctx->adj_boxes - 1) / ctx->adj_boxes, ctx->adj_grid);
        int64_t nl = 0;
        int rc2 = run_adjoint(ctx, a, grid, &nl);
        if (rc2) return rc2;
    }
    if (!on_device) {
        auto back = [&](float *host, const float *dev, size_t count) -> int {
            if (host && count) CK(ctx, cudaMemcpyAsync(host, dev, count * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
            return SLR_OK;
        };
        if ((rc = back(row_lo, drl, (size_t)n * R)) || (rc = back(row_hi, drh, (size_t)n * R)) ||
            (rc = back(d_alpha, dda, (size_t)n * H)) || (rc = back(d_box_lo, ddl, (size_t)n * d)) ||
            (rc = back(d_box_hi, ddh, (size_t)n * d)))
            return rc;
        if (want_w) {
            for (int k = 0; k < K; ++k) {
                if ((rc = back(d_W[k], dW[k], (size_t)ctx->widths[k + 1] * ctx->widths[k])) ||
                    (rc = back(d_b[k], db[k], (size_t)ctx->widths[k + 1])))
                    return rc;
            }
        }
    }
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return SLR_OK;
}

int slr_optimize_alpha(slr_ctx *ctx, int64_t n, const float *box_lo, const float *box_hi, int steps, float lr,
                       float *alpha, float *row_lo, float *row_hi, uint8_t *cls, int on_device) {
    if (!ctx) return fail(nullptr, SLR_EINVAL, "null context");
    if (!ctx->has_net || !ctx->has_prop) return fail(ctx, SLR_ESTATE, "network and property must be set");
    if (n < 0 || (n > 0 && (!box_lo || !box_hi))) return fail(ctx, SLR_EINVAL, "bad box arguments");
    if ((row_lo == nullptr) != (row_hi == nullptr)) return fail(ctx, SLR_EINVAL, "row_lo and row_hi go together");
    if (steps < 0 || steps > 1000) return fail(ctx, SLR_EINVAL, "steps %d out of range [0, 1000]", steps);
    if (!(lr > 0.f) || !std::isfinite(lr)) return fail(ctx, SLR_EINVAL, "lr must be finite and positive");
    if (n == 0) return SLR_OK;
    CK(ctx, cudaSetDevice(ctx->device));
    int rc = prepare_device(ctx);
    if (rc) return rc;
    if ((rc = check_adjoint(ctx))) return rc;
    const int d = ctx->widths[0];
    const int R = (int)ctx->e.size();
    const int64_t H = ctx->H;
    const size_t s_box = align_up((size_t)n * d * sizeof(float));
    const size_t need = alpha_bytes(n, H, R) + align_up((size_t)n) + (on_device ? 0 : 2 * s_box);
    if (!on_device && (rc = check_boxes(ctx, n, d, box_lo, box_hi))) return rc;
    if ((rc = ensure_scratch(ctx, need))) return rc;
    if (!ctx->status) {
        CK(ctx, cudaMalloc(&ctx->status, sizeof(unsigned int)));
        CK(ctx, cudaMallocHost(&ctx->h_status, sizeof(unsigned int)));
    }
    CK(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(unsigned int), ctx->stream));
    unsigned char *p = (unsigned char *)ctx->scratch;
    const AlphaBuffers b = carve_alpha(p, n, H, R);
    p += alpha_bytes(n, H, R);
    uint8_t *dcls = (uint8_t *)p;
    p += align_up((size_t)n);
    const float *dlo = box_lo, *dhi = box_hi;
    if (!on_device) {
        float *t0 = (float *)p, *t1 = (float *)(p + s_box);
        CK(ctx, cudaMemcpyAsync(t0, box_lo, (size_t)n * d * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
        CK(ctx, cudaMemcpyAsync(t1, box_hi, (size_t)n * d * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
        dlo = t0;
        dhi = t1;
    }
    slr::BoxSource src{};
    src.mode = 1;
    src.n_explicit = n;
    src.lo = dlo;
    src.hi = dhi;
    src.cap = n;
    int64_t launches = 0;
    if ((rc = optimise_slopes(ctx, src, n, nullptr, b, steps, lr, dcls, nullptr, nullptr, alpha != nullptr,
                              &launches)))
        return rc;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (row_lo) {
        CK(ctx, cudaMemcpyAsync(row_lo, b.lo_best, (size_t)n * R * sizeof(float), kind, ctx->stream));
        CK(ctx, cudaMemcpyAsync(row_hi, b.hi_best, (size_t)n * R * sizeof(float), kind, ctx->stream));
    }
    if (cls) CK(ctx, cudaMemcpyAsync(cls, dcls, (size_t)n, kind, ctx->stream));
    if (alpha) CK(ctx, cudaMemcpyAsync(alpha, b.alpha, (size_t)n * H * sizeof(float), kind, ctx->stream));
    CK(ctx, cudaMemcpyAsync(ctx->h_status, ctx->status, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return SLR_OK;
}

}  // extern "C"
