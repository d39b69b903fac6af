// What slr_count_noalloc reads from a context (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include "slrcount.h"
#include "slr_device.cuh"

struct slr_noalloc_view {
    int device;
    cudaStream_t stream;
    int d;
    int T32, NT32, grid32, T64, NT64, grid64, sm_count;
    size_t smem32, smem64;
    const slr::NetParams<float> *nf;
    const slr::NetParams<double> *nd;
    const float *lo, *hi;
    int fp64_recheck;
    cudaEvent_t ev0, ev1;
};

// Fills *v when the network and property are resident on the device
// (SLR_ESTATE otherwise); allocates nothing.
int slr_internal_noalloc_view(slr_ctx *ctx, slr_noalloc_view *v);
// Records `msg` as the context's last error and returns `code`.
int slr_internal_fail(slr_ctx *ctx, int code, const char *msg);
