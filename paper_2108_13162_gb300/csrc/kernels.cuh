// Device kernels of the sub-structured CG (sm_103a).
//
// Vectors are concatenated local vectors (Section 3.4.1): entry k belongs to
// one subdomain's V_s; interface nodes have one entry per subdomain holding
// them.  Inside each subdomain the interior rows come first and the
// interface rows last (Eq. 2.4:eqn0), so the interior rows of all subdomains
// form contiguous ranges that the SpMV tiles stream through.
//
// Reductions are deterministic: every block reduces its values with a fixed
// warp-shuffle tree, writes one partial, and the last block to arrive (an
// atomic ticket, no waiting) sums the partials in a fixed order and applies
// the scalar step of Algorithm 3 (alpha, beta, the stopping test).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ssg.h"

namespace ssg {

constexpr int kBlock = 256;      // threads per block, every kernel
constexpr int kTileRows = 256;   // max rows of one interior SpMV tile
constexpr int kTileNnz = 3072;   // max nonzeros staged in shared memory per tile
constexpr int kHostChunk = 32;   // iterations per host-loop chunk (SSG_DRIVER_HOST)

// Scalar state of one CG solve, resident on the device.
struct Scal {
    double rho;      // (r_k, r_k)_w
    double alpha;    // alpha_k
    double beta;     // beta_k
    double pq;       // (S p_k, p_k)_w
    double bnorm;    // sqrt((b, b)_w)
    double rtol;
    double relres;   // sqrt(rho) / bnorm after the last completed iteration
    double aux;      // scratch result (true residual, dot results)
    int32_t iter;    // completed iterations
    int32_t max_iter;
    int32_t status;  // SSG_OK, SSG_E_BREAKDOWN, SSG_E_NOT_CONVERGED
    int32_t done;    // loop must stop before the next kernel does any work
    int32_t stop_after_xp;  // set by the residual update, applied after the x/p update
    int32_t guess;   // x holds an initial guess
    unsigned int ticket[4];
};

enum { kTicketSpmv = 0, kTicketR = 1, kTicketXP = 2, kTicketMisc = 3 };

// Matrix-side arrays on the device (one arena, see api.cu).
struct DevOp {
    const int32_t *rowptr;  // [nloc+1] concatenated local CSR row pointers
    const int32_t *col;     // [nnz] concatenated column index (subdomain offset + local column)
    const double *val;      // [nnz]
    const int2 *tiles;      // [ntiles] interior row ranges [x, y)
    int32_t ntiles;
    const int32_t *iptr;    // [ngamma+1]
    const int32_t *icopy;   // [ncopies]
    int32_t ngamma;
    int32_t niface_blocks;  // ceil(ngamma / kBlock)
    const uint8_t *mult;    // [nloc] multiplicity of each local entry's node
    const double *wtab;     // [256] wtab[m] = 1/m
};

enum { kEpiStore = 0, kEpiAlpha = 1 };

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order block sum; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[kBlock / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < kBlock / 32 ? ws[lane] : 0.0;
        t = warp_sum(t);
    }
    return t;
}

// Thread 0 of each block publishes its partial, then takes a ticket; returns
// true in every thread of the last block to arrive.
__device__ __forceinline__ bool publish_and_check_last(double *partials, double v0, unsigned int *ticket) {
    __shared__ int last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = v0;
        __threadfence();
        const unsigned int t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    return last != 0;
}

__device__ __forceinline__ double sum_partials(const double *partials, int G) {
    __threadfence();
    double v = 0.0;
    for (int i = threadIdx.x; i < G; i += kBlock) v += __ldcg(partials + i);
    return block_sum(v);
}

__device__ __forceinline__ void stop_loop(Scal *s, cudaGraphConditionalHandle h, int use_cond) {
    s->done = 1;
    if (use_cond) cudaGraphSetConditional(h, 0);
}

// ---------------------------------------------------------------------------
// Sub-structured SpMV (Section 3.4.1) with the interface assembly of
// Algorithms 4 and 5 fused in: blocks [0, niface_blocks) take one interface
// node per thread, compute the local row product of each of its copies, sum
// them in ascending subdomain order and write the sum to every copy; the
// remaining blocks stream interior tiles (values and columns staged in shared
// memory with coalesced loads, one thread per row).  Interior rows have
// m = 1, so no assembly touches them.  Every block also accumulates its share
// of (x, y)_w for the alpha step.
// ---------------------------------------------------------------------------
template <int EPI>
__global__ void __launch_bounds__(kBlock) k_spmv_asm(DevOp A, const double *__restrict__ x, double *__restrict__ y,
                                                     double *partials, Scal *s, double *out,
                                                     cudaGraphConditionalHandle h, int use_cond) {
    if (EPI == kEpiAlpha && s->done) return;
    __shared__ double sval[kTileNnz];
    __shared__ int32_t scol[kTileNnz];
    double dot = 0.0;
    if ((int)blockIdx.x < A.niface_blocks) {
        const int g = blockIdx.x * kBlock + threadIdx.x;
        if (g < A.ngamma) {
            const int c0 = A.iptr[g], c1 = A.iptr[g + 1];
            double S = 0.0;
            for (int c = c0; c < c1; ++c) {
                const int row = A.icopy[c];
                double acc = 0.0;
                const int k1 = A.rowptr[row + 1];
                for (int k = A.rowptr[row]; k < k1; ++k) acc = fma(A.val[k], __ldg(x + A.col[k]), acc);
                S += acc;
            }
            const double w = A.wtab[c1 - c0];
            for (int c = c0; c < c1; ++c) {
                const int row = A.icopy[c];
                y[row] = S;
                dot = fma(w * __ldg(x + row), S, dot);
            }
        }
    } else {
        const int2 tl = A.tiles[blockIdx.x - A.niface_blocks];
        const int r0 = tl.x, r1 = tl.y;
        const int e0 = A.rowptr[r0], e1 = A.rowptr[r1];
        const int ne = e1 - e0;
        if (ne <= kTileNnz) {
            for (int e = threadIdx.x; e < ne; e += kBlock) {
                sval[e] = __ldcs(A.val + e0 + e);
                scol[e] = __ldcs(A.col + e0 + e);
            }
            __syncthreads();
            for (int r = r0 + threadIdx.x; r < r1; r += kBlock) {
                const int a = A.rowptr[r] - e0, b = A.rowptr[r + 1] - e0;
                double acc = 0.0;
                for (int k = a; k < b; ++k) acc = fma(sval[k], __ldg(x + scol[k]), acc);
                y[r] = acc;
                dot = fma(__ldg(x + r), acc, dot);
            }
        } else {
            // a single row longer than a tile: block-strided partial sums, fixed tree
            double acc = 0.0;
            for (int k = e0 + threadIdx.x; k < e1; k += kBlock) acc = fma(A.val[k], __ldg(x + A.col[k]), acc);
            acc = block_sum(acc);
            if (threadIdx.x == 0) {
                y[r0] = acc;
                dot = __ldg(x + r0) * acc;
            }
        }
    }
    const double bs = block_sum(dot);
    if (publish_and_check_last(partials, bs, &s->ticket[kTicketSpmv])) {
        const double tot = sum_partials(partials, gridDim.x);
        if (threadIdx.x == 0) {
            s->ticket[kTicketSpmv] = 0;
            if (EPI == kEpiStore) {
                if (out) *out = tot;
            } else {
                s->pq = tot;
                if (!(tot > 0.0) || !isfinite(tot)) {
                    s->status = SSG_E_BREAKDOWN;
                    stop_loop(s, h, use_cond);
                } else {
                    s->alpha = s->rho / tot;
                }
            }
        }
    }
}

// r <- r - alpha q and (r, r)_w; the last block forms beta (Algorithm 3 lines
// 5 and 7, M = I) and the stopping decision, applied after the x/p update.
__global__ void __launch_bounds__(kBlock) k_update_r(int64_t N, double *__restrict__ r, const double *__restrict__ q,
                                                     const uint8_t *__restrict__ mult, const double *__restrict__ wtab,
                                                     double *partials, Scal *s) {
    if (s->done) return;
    const double alpha = s->alpha;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < N; i += stride) {
        const double ri = fma(-alpha, __ldcs(q + i), r[i]);
        r[i] = ri;
        acc = fma(__ldg(wtab + mult[i]) * ri, ri, acc);
    }
    const double bs = block_sum(acc);
    if (publish_and_check_last(partials, bs, &s->ticket[kTicketR])) {
        const double tot = sum_partials(partials, gridDim.x);
        if (threadIdx.x == 0) {
            s->ticket[kTicketR] = 0;
            s->beta = tot / s->rho;
            s->rho = tot;
            s->iter += 1;
            s->relres = s->bnorm > 0.0 ? sqrt(tot) / s->bnorm : 0.0;
            if (sqrt(tot) <= s->rtol * s->bnorm) {
                s->status = SSG_OK;
                s->stop_after_xp = 1;
            } else if (s->iter >= s->max_iter) {
                s->status = SSG_E_NOT_CONVERGED;
                s->stop_after_xp = 1;
            }
        }
    }
}

// x <- x + alpha p; p <- r + beta p (Algorithm 3 lines 4 and 8).
__global__ void __launch_bounds__(kBlock) k_update_xp(int64_t N, double *__restrict__ x, double *__restrict__ p,
                                                      const double *__restrict__ r, double *partials, Scal *s,
                                                      cudaGraphConditionalHandle h, int use_cond) {
    if (s->done) return;
    const double alpha = s->alpha, beta = s->beta;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < N; i += stride) {
        const double pi = p[i];
        x[i] = fma(alpha, pi, x[i]);
        p[i] = fma(beta, pi, __ldcs(r + i));
    }
    if (publish_and_check_last(partials, 0.0, &s->ticket[kTicketXP])) {
        if (threadIdx.x == 0) {
            s->ticket[kTicketXP] = 0;
            if (s->stop_after_xp) stop_loop(s, h, use_cond);
        }
    }
}

// Setup of Algorithm 3 line 1 with M = I: r = b - q (q = S x_1 when a guess
// is given, else r = b), p = r, rho = (r, r)_w, bnorm = sqrt((b, b)_w), and
// the stopping test before the first iteration.
__global__ void __launch_bounds__(kBlock) k_cg_init(int64_t N, const double *__restrict__ b,
                                                    const double *__restrict__ q, double *__restrict__ r,
                                                    double *__restrict__ p, const uint8_t *__restrict__ mult,
                                                    const double *__restrict__ wtab, double *partials, Scal *s,
                                                    cudaGraphConditionalHandle h, int use_cond) {
    const int guess = s->guess;
    double arr = 0.0, abb = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < N; i += stride) {
        const double bi = b[i];
        const double ri = guess ? bi - q[i] : bi;
        r[i] = ri;
        p[i] = ri;
        const double w = __ldg(wtab + mult[i]);
        arr = fma(w * ri, ri, arr);
        abb = fma(w * bi, bi, abb);
    }
    const double srr = block_sum(arr);
    const double sbb = block_sum(abb);
    if (threadIdx.x == 0) partials[gridDim.x + blockIdx.x] = sbb;
    if (publish_and_check_last(partials, srr, &s->ticket[kTicketMisc])) {
        const double rr = sum_partials(partials, gridDim.x);
        const double bb = sum_partials(partials + gridDim.x, gridDim.x);
        if (threadIdx.x == 0) {
            s->ticket[kTicketMisc] = 0;
            s->rho = rr;
            s->bnorm = sqrt(bb);
            s->iter = 0;
            s->done = 0;
            s->stop_after_xp = 0;
            s->alpha = 0.0;
            s->beta = 0.0;
            s->relres = s->bnorm > 0.0 ? sqrt(rr) / s->bnorm : 0.0;
            s->status = SSG_E_NOT_CONVERGED;
            int stop = 0;
            if (sqrt(rr) <= s->rtol * s->bnorm) {
                s->status = SSG_OK;
                stop = 1;
            } else if (s->max_iter <= 0) {
                stop = 1;
            }
            s->done = stop;
            if (use_cond) cudaGraphSetConditional(h, stop ? 0u : 1u);
        }
    }
}

__global__ void k_set_params(Scal *s, double rtol, int32_t max_iter, int32_t guess) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        s->rtol = rtol;
        s->max_iter = max_iter;
        s->guess = guess;
        s->done = 0;
    }
}

// sum_k w_k u_k v_k (DIFF = false) or sum_k w_k (u_k - v_k)^2 (DIFF = true),
// written to *out by the last block (Section 3.4.2 weighted dot).
template <bool DIFF>
__global__ void __launch_bounds__(kBlock) k_wdot(int64_t N, const double *__restrict__ u, const double *__restrict__ v,
                                                 const uint8_t *__restrict__ mult, const double *__restrict__ wtab,
                                                 double *partials, Scal *s, double *out) {
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < N; i += stride) {
        const double w = __ldg(wtab + mult[i]);
        if (DIFF) {
            const double d = u[i] - v[i];
            acc = fma(w * d, d, acc);
        } else {
            acc = fma(w * u[i], v[i], acc);
        }
    }
    const double bs = block_sum(acc);
    if (publish_and_check_last(partials, bs, &s->ticket[kTicketMisc])) {
        const double tot = sum_partials(partials, gridDim.x);
        if (threadIdx.x == 0) {
            s->ticket[kTicketMisc] = 0;
            *out = tot;
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_scatter(int64_t N, const int32_t *__restrict__ l2g,
                                                    const double *__restrict__ xg, double *__restrict__ xl) {
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < N; i += stride) xl[i] = __ldg(xg + l2g[i]);
}

__global__ void __launch_bounds__(kBlock) k_gather(int64_t n, const int32_t *__restrict__ own,
                                                   const double *__restrict__ xl, double *__restrict__ xg) {
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += stride) xg[i] = __ldg(xl + own[i]);
}

}  // namespace ssg
