// The library context, shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "ssg.h"

// A library context: the device, the stream every call is ordered on, and
// settings shared by the systems and band operators created on it.
struct ssg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int driver = SSG_DRIVER_GRAPH;
    int num_sms = 0;
    int live_systems = 0;      // systems and band operators created on this context and not yet destroyed
    double inner_rtol = 1e-4;  // SSG_MIXED: inner FP32 CG tolerance
    int32_t max_outer = 30;    // SSG_MIXED: refinement steps cap
    int32_t rhs_block = 16;    // right-hand sides solved together (1, 2, 4, 8 or 16)
    int32_t unroll = 4;        // CG iterations per pass of a single-vector loop graph's body (measured: 4 beats 1)
    int32_t slice_sort = 0;    // interior slice sorting window: 0 auto (row lengths), 1 none, > 1 rows, -1 subdomain
    // one-cluster solve (cluster.cuh): the most CTAs per cluster this device
    // places (0: none), the count asked for (0: automatic), and the largest
    // system (local entries) solved that way
    int32_t cluster_ctas = 0;
    int32_t cluster_ctas_set = 0;
    int64_t cluster_max_n = 12288;
};

namespace ssg {
void set_error(const std::string &msg);
}

// Return SSG_E_OOM / SSG_E_CUDA (with the call and CUDA's message as the last
// error) from the enclosing function when a CUDA runtime call fails.
#define SSG_CUDA_TRY(call)                                                                      \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                      \
            return e_ == cudaErrorMemoryAllocation ? SSG_E_OOM : SSG_E_CUDA;                    \
        }                                                                                       \
    } while (0)
