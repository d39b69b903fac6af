// Sampling step of the approximate counter (CountingProVe_SLR, Sec. 2.3):
// draw points uniformly in the current box with SplitMix64, evaluate the
// network in float64 at each one, and list the coordinate on the split side
// of every point that lies in the unsafe set.  The host takes the lower
// median of that list as the split point, so that the sampled violations are
// shared evenly between the two halves.
#include "slr_approx.h"
#include "slr_kernels.h"

namespace slr {

namespace {

constexpr int kSampleThreads = 256;
constexpr int kSampleWarps = kSampleThreads / 32;

// One warp per point.  Shared memory: two activation rows of `width` doubles
// per warp; lanes own neurons j = lane, lane + 32, ...
__global__ void __launch_bounds__(kSampleThreads) approx_sample_kernel(const NetParams<double> net, const double *lo,
                                                                       const double *hi, int dim,
                                                                       unsigned long long seed, int trial, int split,
                                                                       int n, int width, double *coord,
                                                                       unsigned long long *count) {
    extern __shared__ __align__(16) double smem_d[];
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    double *h0 = smem_d + (size_t)warp * 2 * width;
    double *h1 = h0 + width;
    const int d = net.d;
    const int K = net.K;
    const int gw = blockIdx.x * kSampleWarps + warp;
    const int nw = gridDim.x * kSampleWarps;
    for (int k = gw; k < n; k += nw) {
        // the point: x_i = lo_i + (hi_i - lo_i) u, one rounding per operation
        for (int i = lane; i < d; i += 32) {
            const double u = splitmix_uniform(seed, approx_draw_index(trial, split, k, i));
            h0[i] = __dadd_rn(lo[i], __dmul_rn(__dsub_rn(hi[i], lo[i]), u));
        }
        __syncwarp();
        const double xd = h0[dim];
        // layers: 0 row-major (n[1] x d), k >= 1 transposed (n[k] x n[k+1]); the
        // last one carries the property rows folded in; the network's
        // activation after the others
        double *src = h0, *dst = h1;
        for (int layer = 0; layer < K; ++layer) {
            const int n_in = net.n[layer], n_out = net.n[layer + 1];
            const double *bias = net.b[layer];
            for (int j = lane; j < n_out; j += 32) {
                double acc = bias[j];
                if (layer == 0) {
                    const double *w = net.W0 + (size_t)j * n_in;
                    for (int i = 0; i < n_in; ++i) acc = __fma_rn(w[i], src[i], acc);
                } else {
                    const double *w = net.Wt[layer] + j;
                    for (int i = 0; i < n_in; ++i) acc = __fma_rn(w[(size_t)i * n_out], src[i], acc);
                }
                if (layer + 1 < K) {
                    const int a = net.act[layer];
                    acc = a == kActTanh ? tanh(acc) : (a == kActSigmoid ? 1.0 / (1.0 + exp(-acc)) : (acc < 0.0 ? 0.0 : acc));
                }
                dst[j] = acc;
            }
            __syncwarp();
            double *t = src;
            src = dst;
            dst = t;
        }
        // the unsafe set: some clause with every row >= 0 (> 0 where strict)
        if (lane == 0) {
            bool unsafe = false;
            int r0 = 0;
            for (int c = 0; c < net.n_clauses && !unsafe; ++c) {
                const int r1 = net.clause_end[c];
                bool all = true;
                for (int r = r0; r < r1; ++r) all = all && (net.strict[r] ? src[r] > 0.0 : src[r] >= 0.0);
                unsafe = all;
                r0 = r1;
            }
            if (unsafe) {
                const unsigned long long pos = atomicAdd(count, 1ull);
                if (pos < (unsigned long long)n) coord[pos] = xd;
            }
        }
        __syncwarp();
    }
}

}  // namespace

size_t approx_sample_smem(const NetParams<double> &net) {
    return (size_t)kSampleWarps * 2 * approx_width(net) * sizeof(double);
}

int approx_width(const NetParams<double> &net) {
    int w = net.d;
    for (int k = 1; k <= net.K; ++k) w = net.n[k] > w ? net.n[k] : w;
    return w;
}

cudaError_t launch_approx_sample(const NetParams<double> &net, const double *lo, const double *hi, int dim,
                                 unsigned long long seed, int trial, int split, int n, double *coord,
                                 unsigned long long *count, int sms, cudaStream_t s) {
    const size_t smem = approx_sample_smem(net);
    cudaError_t e = cudaFuncSetAttribute(approx_sample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int need = (n + kSampleWarps - 1) / kSampleWarps;
    const int grid = need < 4 * sms ? need : 4 * sms;
    approx_sample_kernel<<<grid > 0 ? grid : 1, kSampleThreads, smem, s>>>(net, lo, hi, dim, seed, trial, split, n,
                                                                          approx_width(net), coord, count);
    return cudaGetLastError();
}

}  // namespace slr
