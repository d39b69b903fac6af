// slr_count_noalloc: the count of slr_count for callers that must not
// allocate GPU memory.
//
// Who needs it: a caller that sets the library up once and then counts from a
// loop in which allocation is not allowed or not possible, for example while
// a framework's caching allocator already holds the device memory, or inside
// a real-time control loop that must not stall on cudaMalloc/cudaFree (they
// can synchronise the device).
//
// How: every buffer the count needs besides the network (two frontiers of
// path codes, the class bytes, the re-check list, the level counters and the
// root box with its split masks) is carved out of one file-scope device array
// of fixed size.  The array exists once per GPU that loads the library and
// lives until the process exits.  Its device address is looked up once per
// device with cudaGetSymbolAddress (the host-side symbol is only a stand-in,
// never a device pointer) and handed to the same kernels slr_count launches.
#include <cmath>
#include <cstring>
#include <mutex>

#include "slrcount.h"
#include "slr_kernels.h"
#include "slr_noalloc.h"

namespace {

constexpr int64_t kFrontierCap = (int64_t)1 << 18;   // boxes per level
constexpr int64_t kNearCap = (int64_t)1 << 16;       // FP64 re-check list
constexpr int kMaxD = slr::kMaxWidth;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffCodes0 = 0;
constexpr size_t kOffCodes1 = kOffCodes0 + align256(kFrontierCap * sizeof(uint64_t));
constexpr size_t kOffNear = kOffCodes1 + align256(kFrontierCap * sizeof(uint64_t));
constexpr size_t kOffCtr = kOffNear + align256(kNearCap * sizeof(int64_t));
constexpr size_t kOffStatus = kOffCtr + align256(sizeof(slr::LevelCounters));
constexpr size_t kOffRoot = kOffStatus + align256(sizeof(unsigned int));
constexpr size_t kOffMasks = kOffRoot + align256(2 * (size_t)kMaxD * sizeof(double));
constexpr size_t kOffCls = kOffMasks + align256((size_t)kMaxD * sizeof(unsigned long long));
constexpr size_t kScratchBytes = kOffCls + align256(kFrontierCap);   // about 4.8 MB

__device__ __align__(256) unsigned char g_count_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).
cudaError_t scratch_address(int device, unsigned char **out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_count_scratch);
        if (e != cudaSuccess) return e;
        g_addr[device] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" int slr_count_noalloc(slr_ctx *ctx, int D, slr_result *out) {
    slr_noalloc_view v;
    int rc = slr_internal_noalloc_view(ctx, &v);
    if (rc) return rc;
    if (!out) return slr_internal_fail(ctx, SLR_EINVAL, "out is NULL");
    if (D < 0 || D > slr::kMaxDepth) return slr_internal_fail(ctx, SLR_EINVAL, "D out of range [0, 62]");
    cudaError_t e = cudaSetDevice(v.device);
    unsigned char *base = nullptr;
    if (e == cudaSuccess) e = scratch_address(v.device, &base);
    if (e != cudaSuccess) return slr_internal_fail(ctx, SLR_ECUDA, cudaGetErrorString(e));

    uint64_t *codes[2] = {reinterpret_cast<uint64_t *>(base + kOffCodes0), reinterpret_cast<uint64_t *>(base + kOffCodes1)};
    int64_t *near_list = reinterpret_cast<int64_t *>(base + kOffNear);
    slr::LevelCounters *ctr = reinterpret_cast<slr::LevelCounters *>(base + kOffCtr);
    unsigned int *status = reinterpret_cast<unsigned int *>(base + kOffStatus);
    double *root = reinterpret_cast<double *>(base + kOffRoot);
    unsigned long long *masks = reinterpret_cast<unsigned long long *>(base + kOffMasks);
    uint8_t *cls = base + kOffCls;

    // split schedule (widest side, ties to the lowest index) in fixed host arrays
    const int d = v.d;
    double h_root[2 * kMaxD];
    unsigned long long h_masks[kMaxD];
    int cnt[kMaxD];
    for (int i = 0; i < d; ++i) {
        h_root[i] = (double)v.lo[i];
        h_root[kMaxD + i] = (double)v.hi[i] - (double)v.lo[i];
        h_masks[i] = 0ull;
        cnt[i] = 0;
    }
    for (int t = 0; t < D; ++t) {
        int best = 0;
        double bw = -1.0;
        for (int i = 0; i < d; ++i) {
            const double w = std::ldexp(h_root[kMaxD + i], -cnt[i]);
            if (w > bw) {
                bw = w;
                best = i;
            }
        }
        cnt[best] += 1;
        h_masks[best] |= 1ull << (D - 1 - t);
    }
    cudaStream_t s = v.stream;
#define NA_CK(call)                                                                     \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) return slr_internal_fail(ctx, SLR_ECUDA, cudaGetErrorString(e_)); \
    } while (0)
    NA_CK(cudaMemcpyAsync(root, h_root, d * sizeof(double), cudaMemcpyHostToDevice, s));
    NA_CK(cudaMemcpyAsync(root + d, h_root + kMaxD, d * sizeof(double), cudaMemcpyHostToDevice, s));
    NA_CK(cudaMemcpyAsync(masks, h_masks, d * sizeof(unsigned long long), cudaMemcpyHostToDevice, s));
    // the array keeps the previous call's contents: clear the counters and status
    NA_CK(cudaMemsetAsync(ctr, 0, sizeof(slr::LevelCounters), s));
    NA_CK(cudaMemsetAsync(status, 0, sizeof(unsigned int), s));
    NA_CK(slr::launch_init_count(codes[0], ctr, s));

    const bool recheck = v.fp64_recheck != 0 && v.T64 > 0;
    int64_t launches = 1;
    NA_CK(cudaEventRecord(v.ev0, s));
    for (int t = 0; t <= D; ++t) {
        slr::BoxSource src{};
        src.mode = 0;
        src.codes = codes[t & 1];
        src.count = &ctr->frontier_n[t];
        src.t = t;
        src.D = D;
        src.dim_mask = masks;
        src.root_lo = root;
        src.root_w = root + d;
        src.cap = kFrontierCap;
        slr::EvalOutputs o{};
        o.cls = cls;
        o.near_list = recheck ? near_list : nullptr;
        o.near_count = &ctr->near_n[t];
        o.near_cap = kNearCap;
        o.tie_count = &ctr->ties;
        o.status = status;
        NA_CK(slr::launch_eval_f32(v.T32, v.NT32, v.grid32, v.smem32, s, *v.nf, src, o, 0));
        ++launches;
        if (recheck) {
            slr::BoxSource s2 = src;
            s2.index = near_list;
            s2.index_count = &ctr->near_n[t];
            s2.cap = kNearCap;
            slr::EvalOutputs o2{};
            o2.cls = cls;
            o2.tie_count = &ctr->ties;
            o2.status = status;
            NA_CK(slr::launch_eval_f64(v.T64, v.NT64, v.grid64, v.smem64, s, *v.nd, s2, o2, 1));
            ++launches;
        }
        NA_CK(slr::launch_compact(codes[t & 1], cls, codes[(t + 1) & 1], ctr, status, kFrontierCap, t, D, nullptr,
                                  nullptr, nullptr, 0, v.sm_count * 4, s));
        launches += 2;
    }
    NA_CK(cudaEventRecord(v.ev1, s));
    slr::LevelCounters c;
    unsigned int st = 0;
    NA_CK(cudaMemcpyAsync(&c, ctr, sizeof c, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaMemcpyAsync(&st, status, sizeof st, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
#undef NA_CK
    float ms = 0.f;
    cudaEventElapsedTime(&ms, v.ev0, v.ev1);
    std::memset(out, 0, sizeof *out);
    out->unsafe_lo = c.unsafe_lo;
    out->unsafe_hi = c.unsafe_lo + c.undecided_at_D;
    out->boxes = c.boxes;
    out->tie_leaves = c.ties;
    out->depth = D;
    unsigned long long rech = 0;
    for (int t = 0; t <= D; ++t) {
        out->level_boxes[t] = c.level_boxes[t];
        out->level_safe[t] = c.level_safe[t];
        out->level_unsafe[t] = c.level_unsafe[t];
        out->level_undecided[t] = c.level_undecided[t];
        rech += c.near_n[t] < (unsigned long long)kNearCap ? c.near_n[t] : (unsigned long long)kNearCap;
        if (c.level_boxes[t]) out->levels = t + 1;
    }
    out->rechecked = recheck ? rech : 0;
    out->rechecked_fp64 = out->rechecked;
    out->device_ms = ms;
    out->launches = launches;
    out->h2d_bytes = (int64_t)(2 * d * sizeof(double) + d * sizeof(unsigned long long));
    out->d2h_bytes = (int64_t)(sizeof c + sizeof st);
    out->tile_boxes = v.T32;
    out->tile_threads = v.NT32;
    if (st & slr::kStatusOverflow)
        return slr_internal_fail(ctx, SLR_EOVERFLOW,
                                 "slr_count_noalloc: a level exceeded the 262144-box frontier of its fixed scratch");
    if (st & slr::kStatusNearOverflow)
        return slr_internal_fail(ctx, SLR_EOVERFLOW,
                                 "slr_count_noalloc: the FP64 re-check list exceeded its 65536 entries");
    return SLR_OK;
}
