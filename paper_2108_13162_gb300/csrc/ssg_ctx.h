// The library context, shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "ssg.h"

// A library context: the device, the stream every call is ordered on, and
// settings shared by the systems and band operators created on it.
struct ssg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int driver = SSG_DRIVER_GRAPH;
    int num_sms = 0;
    int live_systems = 0;      // systems and band operators created on this context and not yet destroyed
    int pdl = 0;               // programmatic dependent launch inside the loop bodies (measured: off is faster)
    double inner_rtol = 1e-4;  // SSG_MIXED: inner FP32 CG tolerance
    int32_t max_outer = 30;    // SSG_MIXED: refinement steps cap
    int32_t rhs_block = 16;    // right-hand sides solved together (1, 2, 4, 8 or 16)
};
