// Kernels of the differentiable solve: new matrix values for an existing
// sub-structure, the gradient of a loss with respect to the stored entries
// (the adjoint rule dL/dA_ij = -sum_rhs lambda_i x_j with lambda = A^-1 dL/dx),
// and the 7-point finite-volume operator of the synthetic diffusion workloads
// with its adjoint, which carries dL/dA to the per-cell log conductivities.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace ssg {

// dst[i] = src[map[i]] (0 where map[i] < 0: sliced-ELL padding), and its FP32
// rounding: refreshes one device copy of the matrix values.
__global__ void __launch_bounds__(kBlock) k_gather_vals(int64_t n, const int32_t *__restrict__ map,
                                                        const double *__restrict__ src, double *__restrict__ dst,
                                                        float *__restrict__ dst32) {
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += stride) {
        const int32_t m = map[i];
        const double v = m >= 0 ? src[m] : 0.0;
        dst[i] = v;
        if (dst32) dst32[i] = float(v);
    }
}

// g[e] = -sum_j lam[j*n + row(e)] * x[j*n + col(e)] for every stored entry e
// of the input CSR.  One thread per local row; each stored entry lives in
// exactly one local matrix (entry ownership), so every g[e] is written once.
__global__ void __launch_bounds__(kBlock) k_pattern_grad(int64_t nloc, int64_t n, int k,
                                                         const int32_t *__restrict__ rowptr,
                                                         const int32_t *__restrict__ col,
                                                         const int32_t *__restrict__ l2g,
                                                         const int32_t *__restrict__ vmap,
                                                         const double *__restrict__ lam,
                                                         const double *__restrict__ x, double *__restrict__ g) {
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t r = (int64_t)blockIdx.x * kBlock + threadIdx.x; r < nloc; r += stride) {
        const int64_t gr = l2g[r];
        for (int32_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
            const int64_t gc = l2g[col[e]];
            double acc = 0.0;
            for (int j = 0; j < k; ++j) acc = fma(lam[j * n + gr], x[j * n + gc], acc);
            g[vmap[e]] = -acc;
        }
    }
}

// --- 7-point finite volumes on an nx x ny x nz cell grid ------------------
// Cell (ix, iy, iz) has id ix + nx (iy + ny iz) and conductivity
// kappa = exp(logk).  An interior face between cells a and b carries the
// harmonic mean t = 2 k_a k_b / (k_a + k_b), a boundary face (u = 0 outside)
// t = 2 k.  Row i of the CSR matrix lists, in ascending column order, the
// existing neighbours z-, y-, x-, the diagonal, x+, y+, z+: A_ij = -t of the
// shared face, A_ii = the sum of the six face coefficients (z-, y-, x-, x+,
// y+, z+ order).

struct Fv7Grid {
    int nx, ny, nz;
};

__device__ __forceinline__ double fv7_harm(double a, double b) { return 2.0 * a * b / (a + b); }

// Neighbours of cell i in the order z-, y-, x-, x+, y+, z+ (-1 at the boundary).
__device__ __forceinline__ void fv7_nb(const Fv7Grid &G, int64_t i, int64_t (&nb)[6]) {
    const int64_t sxy = (int64_t)G.nx * G.ny;
    const int ix = (int)(i % G.nx), iy = (int)((i / G.nx) % G.ny), iz = (int)(i / sxy);
    nb[0] = iz > 0 ? i - sxy : -1;
    nb[1] = iy > 0 ? i - G.nx : -1;
    nb[2] = ix > 0 ? i - 1 : -1;
    nb[3] = ix < G.nx - 1 ? i + 1 : -1;
    nb[4] = iy < G.ny - 1 ? i + G.nx : -1;
    nb[5] = iz < G.nz - 1 ? i + sxy : -1;
}

// Face coefficients of cell i in the same order.
__device__ __forceinline__ void fv7_faces(const Fv7Grid &G, const double *__restrict__ logk, int64_t i, double ki,
                                          double (&t)[6], int64_t (&nb)[6]) {
    fv7_nb(G, i, nb);
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        if (nb[d] < 0) {
            t[d] = 2.0 * ki;
        } else {
            const double kj = exp(logk[nb[d]]);
            // the same operand order from both sides of the face
            t[d] = d < 3 ? fv7_harm(kj, ki) : fv7_harm(ki, kj);
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_fv7_values(Fv7Grid G, const double *__restrict__ logk,
                                                       const int32_t *__restrict__ rowptr, double *__restrict__ val) {
    const int64_t n = (int64_t)G.nx * G.ny * G.nz;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += stride) {
        const double ki = exp(logk[i]);
        double t[6];
        int64_t nb[6];
        fv7_faces(G, logk, i, ki, t, nb);
        double diag = t[0] + t[1];
        diag = diag + t[2];
        diag = diag + t[3];
        diag = diag + t[4];
        diag = diag + t[5];
        int32_t e = rowptr[i];
        for (int d = 0; d < 3; ++d)
            if (nb[d] >= 0) val[e++] = -t[d];
        val[e++] = diag;
        for (int d = 3; d < 6; ++d)
            if (nb[d] >= 0) val[e++] = -t[d];
    }
}

// Position of entry (i, j) in row i for neighbour direction d (or the
// diagonal for d = -1), from the layout above.
__device__ __forceinline__ int32_t fv7_pos(const int32_t *__restrict__ rowptr, const int64_t (&nb)[6], int64_t i,
                                           int d) {
    int32_t p = rowptr[i];
    const int lower = (nb[0] >= 0) + (nb[1] >= 0) + (nb[2] >= 0);
    if (d < 0) return p + lower;
    if (d < 3) {
        for (int q = 0; q < d; ++q) p += nb[q] >= 0;
        return p;
    }
    p += lower + 1;
    for (int q = 3; q < d; ++q) p += nb[q] >= 0;
    return p;
}

// d log k_i of L from g = dL/dA (CSR order):
//   dL/dt (interior face a < b) = ((g_aa + g_bb) - g_ab) - g_ba,
//   dL/dt (boundary face of i)  = g_ii,
//   dt/dk_i = 2 k_j^2 / (k_i + k_j)^2 (interior), 2 (boundary),
//   dL/dlogk_i = k_i sum over the six faces of dL/dt dt/dk_i.
__global__ void __launch_bounds__(kBlock) k_fv7_adjoint(Fv7Grid G, const double *__restrict__ logk,
                                                        const int32_t *__restrict__ rowptr,
                                                        const double *__restrict__ g, double *__restrict__ glogk) {
    const int64_t n = (int64_t)G.nx * G.ny * G.nz;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += stride) {
        const double ki = exp(logk[i]);
        int64_t nb[6];
        fv7_nb(G, i, nb);
        const double gii = g[fv7_pos(rowptr, nb, i, -1)];
        double acc = 0.0;
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            const int64_t j = nb[d];
            if (j < 0) {
                acc = fma(gii, 2.0, acc);
                continue;
            }
            // row j's neighbour in the opposite direction (5 - d) is i
            int64_t nbj[6];
            fv7_nb(G, j, nbj);
            const double kj = exp(logk[j]);
            const double gjj = g[fv7_pos(rowptr, nbj, j, -1)];
            const double gij = g[fv7_pos(rowptr, nb, i, d)];
            const double gji = g[fv7_pos(rowptr, nbj, j, 5 - d)];
            const double dLdt = i < j ? ((gii + gjj) - gij) - gji : ((gjj + gii) - gji) - gij;
            const double s = ki + kj;
            acc = fma(dLdt, 2.0 * kj * kj / (s * s), acc);
        }
        glogk[i] = ki * acc;
    }
}

}  // namespace ssg
