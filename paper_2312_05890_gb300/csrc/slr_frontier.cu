// Frontier kernels of the level-by-level count (Alg. 1, Sec. 3).
//
// compact_kernel is the split/volume step of one level: it reads the path
// codes and classes of the level's boxes and
//   UNSAFE     adds 2^(D-t) to the unsafe volume (one unit = 2^-D of the root),
//   SAFE       drops the box,
//   UNDECIDED  writes the two children codes 2c, 2c+1 to the next level when
//              t < D, or adds one unit to the undecided volume when t = D.
// The single-problem count keeps the frontier's order (two passes, below);
// the batched count appends with one atomic per warp (ballot + popc).
// Integer sums make the volumes independent of order either way.
#include <algorithm>

#include "slr_eval.cuh"
#include "slr_kernels.h"

namespace slr {

__global__ void init_count_kernel(uint64_t *codes0, LevelCounters *ctr) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        codes0[0] = 0ull;
        ctr->frontier_n[0] = 1ull;
    }
}

__device__ __forceinline__ void compact_body(const uint64_t *__restrict__ codes_in, const uint8_t *__restrict__ cls,
                                             uint64_t *__restrict__ codes_out, LevelCounters *ctr,
                                             unsigned int *status, int64_t cap, int t, int D, uint64_t *leaf_codes,
                                             uint8_t *leaf_depth, uint8_t *leaf_cls, int64_t leaf_cap, int block,
                                             int nblocks) {
    const unsigned long long n_raw = ctr->frontier_n[t];
    const int64_t n = (int64_t)n_raw < cap ? (int64_t)n_raw : cap;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t warp_global = ((int64_t)block * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)nblocks * blockDim.x) >> 5;
    if (block == 0 && threadIdx.x == 0) {
        ctr->level_boxes[t] = (unsigned long long)n;
        atomicAdd(&ctr->boxes, (unsigned long long)n);
    }
    unsigned long long n_unsafe = 0, n_safe = 0, n_und = 0;
    for (int64_t base = warp_global * 32; base < n; base += n_warps * 32) {
        const int64_t i = base + lane;
        const bool valid = i < n;
        const uint8_t c = valid ? cls[i] : (uint8_t)255;
        const uint64_t code = valid ? codes_in[i] : 0ull;
        const bool und = c == kUndecided;
        const unsigned m_und = __ballot_sync(0xffffffffu, und);
        const unsigned m_uns = __ballot_sync(0xffffffffu, c == kUnsafe);
        const unsigned m_safe = __ballot_sync(0xffffffffu, c == kSafe);
        n_unsafe += __popc(m_uns);
        n_safe += __popc(m_safe);
        n_und += __popc(m_und);
        if (t < D) {
            unsigned long long slot = 0;
            if (lane == 0 && m_und != 0u)
                slot = atomicAdd(&ctr->frontier_n[t + 1], 2ull * (unsigned long long)__popc(m_und));
            slot = __shfl_sync(0xffffffffu, slot, 0);
            if (und) {
                const int64_t pos = (int64_t)slot + 2 * __popc(m_und & lt_mask);
                if (pos + 1 < cap) {
                    codes_out[pos] = code << 1;
                    codes_out[pos + 1] = (code << 1) | 1ull;
                } else {
                    atomicOr(status, kStatusOverflow);
                }
            }
        }
        if (leaf_codes != nullptr) {
            const bool leaf = (c == kUnsafe) || (c == kSafe) || (und && t == D);
            const unsigned m_leaf = __ballot_sync(0xffffffffu, leaf);
            unsigned long long slot = 0;
            if (lane == 0 && m_leaf != 0u) slot = atomicAdd(&ctr->leaves, (unsigned long long)__popc(m_leaf));
            slot = __shfl_sync(0xffffffffu, slot, 0);
            if (leaf) {
                const int64_t pos = (int64_t)slot + __popc(m_leaf & lt_mask);
                if (pos < leaf_cap) {
                    leaf_codes[pos] = code;
                    leaf_depth[pos] = (uint8_t)t;
                    leaf_cls[pos] = c;
                } else {
                    atomicOr(status, kStatusLeafOverflow);
                }
            }
        }
    }
    // one atomic per warp for the level statistics and the volumes
    if (lane == 0) {
        if (n_unsafe) {
            atomicAdd(&ctr->level_unsafe[t], n_unsafe);
            atomicAdd(&ctr->unsafe_lo, n_unsafe << (D - t));
        }
        if (n_safe) atomicAdd(&ctr->level_safe[t], n_safe);
        if (n_und) {
            atomicAdd(&ctr->level_undecided[t], n_und);
            if (t == D) atomicAdd(&ctr->undecided_at_D, n_und);
        }
    }
}

// ---- order-preserving compaction (single problem) ---------------------------
// Block b of kCompactBlocks takes the contiguous range [b CH, (b+1) CH) of the
// level; the first pass counts its UNDECIDED boxes, the second writes their
// children at the block's exclusive prefix plus the in-block rank.  The next
// frontier keeps the order of the current one, so it stays sorted by path
// code: consecutive boxes are neighbours in the bisection tree, and the whole
// count is independent of scheduling.
__device__ __forceinline__ void compact_range(int64_t n, int64_t &lo, int64_t &hi) {
    int64_t ch = (n + kCompactBlocks - 1) / kCompactBlocks;
    ch = (ch + 255) & ~(int64_t)255;
    lo = (int64_t)blockIdx.x * ch;
    hi = lo + ch < n ? lo + ch : n;
}

__device__ __forceinline__ unsigned block_sum(unsigned v, unsigned *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
    __syncthreads();
    return tot;
}

__global__ void __launch_bounds__(256)
compact_count_kernel(const uint8_t *__restrict__ cls, LevelCounters *ctr, int64_t cap, int t) {
    __shared__ unsigned sh[8];
    const unsigned long long n_raw = ctr->frontier_n[t];
    const int64_t n = (int64_t)n_raw < cap ? (int64_t)n_raw : cap;
    int64_t lo, hi;
    compact_range(n, lo, hi);
    unsigned c = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) c += cls[i] == kUndecided ? 1u : 0u;
    c = block_sum(c, sh);
    if (threadIdx.x == 0) ctr->block_count[blockIdx.x] = c;
}

__global__ void __launch_bounds__(256)
compact_kernel(const uint64_t *__restrict__ codes_in, const uint8_t *__restrict__ cls,
               uint64_t *__restrict__ codes_out, LevelCounters *ctr, unsigned int *status,
               int64_t cap, int t, int D, uint64_t *leaf_codes, uint8_t *leaf_depth,
               uint8_t *leaf_cls, int64_t leaf_cap, uint64_t path_mask, int add_volume) {
    __shared__ unsigned sh[8];
    __shared__ unsigned long long s_off;
    const unsigned long long n_raw = ctr->frontier_n[t];
    const int64_t n = (int64_t)n_raw < cap ? (int64_t)n_raw : cap;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    // exclusive prefix of the blocks before this one (and, in block 0, the total)
    unsigned long long before = 0, total = 0;
    for (int b = threadIdx.x; b < kCompactBlocks; b += blockDim.x) {
        const unsigned long long v = ctr->block_count[b];
        total += v;
        if (b < (int)blockIdx.x) before += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        before += __shfl_xor_sync(0xffffffffu, before, o);
        total += __shfl_xor_sync(0xffffffffu, total, o);
    }
    __shared__ unsigned long long sb[8], st8[8];
    if (lane == 0) {
        sb[warp] = before;
        st8[warp] = total;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, z = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += sb[w];
            z += st8[w];
        }
        s_off = a;
        if (blockIdx.x == 0) {
            ctr->level_boxes[t] = (unsigned long long)n;
            atomicAdd(&ctr->boxes, (unsigned long long)n);
            if (t < D) {
                ctr->frontier_n[t + 1] = 2ull * z;
                if ((int64_t)(2ull * z) > cap) atomicOr(status, kStatusOverflow);
            }
        }
    }
    __syncthreads();
    unsigned long long off = s_off;
    int64_t lo, hi;
    compact_range(n, lo, hi);
    unsigned long long n_unsafe = 0, n_safe = 0, n_und = 0;
    for (int64_t base = lo; base < hi; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < hi;
        const uint8_t c = valid ? cls[i] : (uint8_t)255;
        const uint64_t code = valid ? codes_in[i] : 0ull;
        const bool und = c == kUndecided;
        const unsigned m_und = __ballot_sync(0xffffffffu, und);
        n_unsafe += __popc(__ballot_sync(0xffffffffu, c == kUnsafe));
        n_safe += __popc(__ballot_sync(0xffffffffu, c == kSafe));
        n_und += __popc(m_und);
        // in-block rank: warps in order
        if (lane == 0) sh[warp] = __popc(m_und);
        __syncthreads();
        unsigned wbefore = 0, ctot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            if (w < warp) wbefore += sh[w];
            ctot += sh[w];
        }
        __syncthreads();
        if (t < D && und) {
            const int64_t pos = 2 * (int64_t)(off + wbefore + __popc(m_und & lt_mask));
            if (pos + 1 < cap) {
                // children: the path bits (those under path_mask) shifted up by one
                const uint64_t child = code + (code & path_mask);
                codes_out[pos] = child;
                codes_out[pos + 1] = child | 1ull;
            }
        }
        off += ctot;
        if (leaf_codes != nullptr) {
            const bool leaf = (c == kUnsafe) || (c == kSafe) || (und && t == D);
            const unsigned m_leaf = __ballot_sync(0xffffffffu, leaf);
            unsigned long long slot = 0;
            if (lane == 0 && m_leaf != 0u) slot = atomicAdd(&ctr->leaves, (unsigned long long)__popc(m_leaf));
            slot = __shfl_sync(0xffffffffu, slot, 0);
            if (leaf) {
                const int64_t pos = (int64_t)slot + __popc(m_leaf & lt_mask);
                if (pos < leaf_cap) {
                    leaf_codes[pos] = code;
                    leaf_depth[pos] = (uint8_t)t;
                    leaf_cls[pos] = c;
                } else {
                    atomicOr(status, kStatusLeafOverflow);
                }
            }
        }
    }
    if (lane == 0) {
        if (n_unsafe) {
            atomicAdd(&ctr->level_unsafe[t], n_unsafe);
            if (add_volume) atomicAdd(&ctr->unsafe_lo, n_unsafe << (D - t));
        }
        if (n_safe) atomicAdd(&ctr->level_safe[t], n_safe);
        if (n_und) {
            atomicAdd(&ctr->level_undecided[t], n_und);
            if (t == D) atomicAdd(&ctr->undecided_at_D, n_und);
        }
    }
}

// ---- batched counting: many problems advance one level per step ------------

// Exclusive prefix of the tiles of each problem's source at this step
// (tile_prefix[P] = total).  One block; problems in chunks of its width.
__global__ void __launch_bounds__(1024) tile_prefix_kernel(const BoxSource *srcs, int P, int T, long long *prefix) {
    __shared__ long long buf[1024];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < P; c0 += 1024) {
        const int p = c0 + threadIdx.x;
        long long v = 0;
        if (p < P) {
            const int64_t n = source_count(srcs[p]);
            v = (n + T - 1) / T;
        }
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {   // inclusive Hillis-Steele scan
            const long long add = threadIdx.x >= off ? buf[threadIdx.x - off] : 0;
            __syncthreads();
            buf[threadIdx.x] += add;
            __syncthreads();
        }
        if (p < P) prefix[p] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += buf[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) prefix[P] = carry;
}

// Compaction of every active problem: block (x, p) works on problem p.
__global__ void __launch_bounds__(256) compact_batch_kernel(const CompactArgs *args, int t, unsigned int *status) {
    const CompactArgs a = args[blockIdx.y];
    if (t > a.D) return;
    compact_body(a.codes_in, a.cls, a.codes_out, a.ctr, status, a.cap, t, a.D, nullptr, nullptr, nullptr, 0,
                 blockIdx.x, gridDim.x);
}

// Start of a batched count: every problem's level 0 is its root box.
__global__ void init_batch_kernel(const CompactArgs *args, int P) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) {
        const_cast<uint64_t *>(args[p].codes_in)[0] = 0ull;
        args[p].ctr->frontier_n[0] = 1ull;
    }
}

cudaError_t launch_tile_prefix(const BoxSource *srcs, int P, int T, long long *prefix, cudaStream_t s) {
    tile_prefix_kernel<<<1, 1024, 0, s>>>(srcs, P, T, prefix);
    return cudaGetLastError();
}

cudaError_t launch_compact_batch(const CompactArgs *args, int P, int t, unsigned int *status, int blocks_per_problem,
                                 cudaStream_t s) {
    compact_batch_kernel<<<dim3(blocks_per_problem, P), 256, 0, s>>>(args, t, status);
    return cudaGetLastError();
}

cudaError_t launch_init_batch(const CompactArgs *args, int P, cudaStream_t s) {
    init_batch_kernel<<<(P + 127) / 128, 128, 0, s>>>(args, P);
    return cudaGetLastError();
}

cudaError_t launch_init_count(uint64_t *codes0, LevelCounters *ctr, cudaStream_t s) {
    init_count_kernel<<<1, 32, 0, s>>>(codes0, ctr);
    return cudaGetLastError();
}

cudaError_t launch_compact(const uint64_t *codes_in, const uint8_t *cls, uint64_t *codes_out,
                           LevelCounters *ctr, unsigned int *status, int64_t cap, int t, int D,
                           uint64_t *leaf_codes, uint8_t *leaf_depth, uint8_t *leaf_cls,
                           int64_t leaf_cap, int grid, cudaStream_t s, uint64_t path_mask, bool add_volume) {
    (void)grid;
    compact_count_kernel<<<kCompactBlocks, 256, 0, s>>>(cls, ctr, cap, t);
    compact_kernel<<<kCompactBlocks, 256, 0, s>>>(codes_in, cls, codes_out, ctr, status, cap, t, D, leaf_codes,
                                                  leaf_depth, leaf_cls, leaf_cap, path_mask, add_volume ? 1 : 0);
    return cudaGetLastError();
}

// One shard of a count: of level t keep the boxes at frontier positions
// index, index + count, index + 2 count, ... (each the root of a subtree), in
// order.  Copied out, copied back, then the level's size set.
__device__ __forceinline__ int64_t shard_size(const LevelCounters *ctr, int t, int count, int index, int64_t cap) {
    int64_t n = (int64_t)ctr->frontier_n[t];
    n = n < cap ? n : cap;
    return n > index ? (n - index + count - 1) / count : 0;
}

__global__ void shard_gather_kernel(const uint64_t *__restrict__ codes, uint64_t *__restrict__ scratch,
                                    const LevelCounters *ctr, int t, int count, int index, int64_t cap) {
    const int64_t m = shard_size(ctr, t, count, index, cap);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        scratch[j] = codes[index + j * count];
}

__global__ void shard_back_kernel(const uint64_t *__restrict__ scratch, uint64_t *__restrict__ codes,
                                  const LevelCounters *ctr, int t, int count, int index, int64_t cap) {
    const int64_t m = shard_size(ctr, t, count, index, cap);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        codes[j] = scratch[j];
}

__global__ void shard_size_kernel(LevelCounters *ctr, int t, int count, int index, int64_t cap) {
    if (threadIdx.x == 0 && blockIdx.x == 0) ctr->frontier_n[t] = (unsigned long long)shard_size(ctr, t, count, index, cap);
}

cudaError_t launch_shard_level(uint64_t *codes, uint64_t *scratch, LevelCounters *ctr, int t, int count, int index,
                               int64_t cap, int sms, cudaStream_t s) {
    const int grid = std::max(1, sms * 4);
    shard_gather_kernel<<<grid, 256, 0, s>>>(codes, scratch, ctr, t, count, index, cap);
    shard_back_kernel<<<grid, 256, 0, s>>>(scratch, codes, ctr, t, count, index, cap);
    shard_size_kernel<<<1, 32, 0, s>>>(ctr, t, count, index, cap);
    return cudaGetLastError();
}

}  // namespace slr
