// Interface-weighted dot product that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: programs whose device
// memory is owned by their own caching allocator under a fixed budget (a
// library allocation outside it can fail or push the program out of memory),
// and latency-critical loops that must not take the implicit device
// synchronisation cudaMalloc/cudaFree can cause.  ssg_wdot_noalloc serves
// them: its only scratch (the per-block partial sums and the last-block
// ticket) lives in one file-scope __device__ array that every GPU loading
// this library holds until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "ssg_internal.h"

namespace ssg {
namespace {

constexpr int kBlock = 256;
constexpr int kNoAllocChunk = kBlock * 16;     // entries handled by one block
constexpr int kNoAllocMaxBlocks = 8192;        // partial sums the scratch holds
constexpr int64_t kNoAllocMaxN = static_cast<int64_t>(kNoAllocChunk) * kNoAllocMaxBlocks;  // 33,554,432
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
    double partials[kNoAllocMaxBlocks];
    unsigned int ticket;
};

// The scratch (about 64 KB).  Host code only sees a host-side stand-in under
// this name; kernels get the device address taken with cudaGetSymbolAddress.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_mu;
NoAllocScratch *g_scratch_ptr[kMaxDevices] = {};

// Fixed-order reductions, the same scheme as the system path's kernels.
__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double na_block_sum(double v) {
    __shared__ double ws[kBlock / 32];
    v = na_warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < kBlock / 32 ? ws[lane] : 0.0;
        t = na_warp_sum(t);
    }
    return t;
}

// Same arithmetic as the weighted dot of the system path (w = 1/m, one FMA per
// entry, fixed-order block and last-block sums), one chunk per block.  A
// multiplicity of 0 (no node has it) gets weight 0, as in the system path's
// weight table, so such an entry adds nothing instead of a non-finite value.
__global__ void __launch_bounds__(kBlock) k_wdot_noalloc(int64_t n, const double *__restrict__ u,
                                                         const double *__restrict__ v,
                                                         const uint8_t *__restrict__ mult, NoAllocScratch *sc,
                                                         double *out) {
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kNoAllocChunk;
    double acc = 0.0;
    for (int j = threadIdx.x; j < kNoAllocChunk; j += kBlock) {
        const int64_t i = base + j;
        if (i < n) {
            const unsigned int m = mult[i];
            const double w = (m == 1u) ? 1.0 : (m == 0u ? 0.0 : 1.0 / static_cast<double>(m));
            acc = fma(w * u[i], v[i], acc);
        }
    }
    const double bs = na_block_sum(acc);
    __shared__ int last;
    if (threadIdx.x == 0) {
        sc->partials[blockIdx.x] = bs;
        __threadfence();
        last = (atomicAdd(&sc->ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double t = 0.0;
        for (int i = threadIdx.x; i < static_cast<int>(gridDim.x); i += kBlock) t += __ldcg(sc->partials + i);
        const double tot = na_block_sum(t);
        if (threadIdx.x == 0) {
            sc->ticket = 0;
            *out = tot;
        }
    }
}

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.
int scratch_on_current_device(NoAllocScratch **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return SSG_E_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device id " + std::to_string(dev) + " beyond the " + std::to_string(kMaxDevices) +
                  " devices ssg_wdot_noalloc supports");
        return SSG_E_INVALID;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
            return SSG_E_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<NoAllocScratch *>(p);
    }
    *out = g_scratch_ptr[dev];
    return SSG_OK;
}

}  // namespace
}  // namespace ssg

using namespace ssg;

extern "C" int ssg_wdot_noalloc(const double *u_loc, const double *v_loc, const uint8_t *mult_loc, int64_t nloc,
                                double *result_dev, void *stream) {
    if (nloc < 0 || nloc > kNoAllocMaxN) {
        set_error("ssg_wdot_noalloc: nloc = " + std::to_string(nloc) + " outside [0, " +
                  std::to_string(kNoAllocMaxN) + "], the size its static scratch can reduce");
        return SSG_E_INVALID;
    }
    if (!result_dev || (nloc > 0 && (!u_loc || !v_loc || !mult_loc))) {
        set_error("ssg_wdot_noalloc: null pointer");
        return SSG_E_INVALID;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (nloc == 0) {
        cudaError_t e = cudaMemsetAsync(result_dev, 0, sizeof(double), s);
        if (e != cudaSuccess) {
            set_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
            return SSG_E_CUDA;
        }
        return SSG_OK;
    }
    NoAllocScratch *sc = nullptr;
    int rc = scratch_on_current_device(&sc);
    if (rc != SSG_OK) return rc;
    // the ticket must start at zero; the partials are all overwritten
    cudaError_t e = cudaMemsetAsync(&sc->ticket, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMemsetAsync(ticket): ") + cudaGetErrorString(e));
        return SSG_E_CUDA;
    }
    const int blocks = static_cast<int>((nloc + kNoAllocChunk - 1) / kNoAllocChunk);
    k_wdot_noalloc<<<blocks, kBlock, 0, s>>>(nloc, u_loc, v_loc, mult_loc, sc, result_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("k_wdot_noalloc launch: ") + cudaGetErrorString(e));
        return SSG_E_CUDA;
    }
    return SSG_OK;
}
