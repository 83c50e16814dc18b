// Several right-hand sides, and several independent systems, solved together.
//
// K right-hand sides (K = 2, 4, 8 or 16) run Algorithm 3 side by side, each
// with its own alpha, beta and stopping test; the local matrices of the
// sub-structures are streamed once per iteration for all K columns, so the
// SpMV of Section 3.4.1 becomes a product with K vectors.  A column whose
// test has passed (or that broke down) is frozen: its alpha and beta are
// zero from then on, so x, r and the inner correction keep their bits.  Each
// column therefore follows the same sequence of operations as a solve of its
// right-hand side alone.
//
// Independent systems ("segments") are solved as one operator: the union of
// their sub-structures, block diagonal, with the subdomains of each system
// contiguous.  Every block of every kernel works inside one segment (the
// product's work list is cut per segment, the vector kernels run one block
// per chunk of one segment's local entries), each segment has its own state
// (ScalB) for its K columns, and a segment whose columns are all frozen
// skips its blocks.  One system with K columns is the case of one segment.
//
// Local vector blocks are interleaved: entry k of column j sits at k*K + j,
// so one local entry's K values are contiguous (K*8 bytes in FP64).
//
// Reductions stay deterministic: a block writes one partial per column, and
// every block of the next kernel sums its segment's partials of each column
// in the same fixed order.
#pragma once

#include "kernels.cuh"

namespace ssg {

constexpr int kMaxRhs = 16;
// Threads per block of the chunk kernels (one chunk of local entries per
// block, about one block per SM): every block sums its segment's partials of
// the previous kernel in FP64 (2 DFMA/clk/SM on this part), so fewer, larger
// chunks keep that sum small next to the chunk's own streaming.
constexpr int kBlockV = 1024;

// State of K solves, resident on the device.  Bit j of `act` is set while
// column j still iterates.
struct ScalB {
    double rho[kMaxRhs];     // (r, z)_w of the last completed iteration (z = r without a preconditioner)
    double rrt[kMaxRhs];     // (r, r)_w of the last completed iteration: the stopping test
    double rho_b[kMaxRhs];   // rho as the residual update saw it
    double alpha[kMaxRhs];
    double pq[kMaxRhs];
    double bnorm[kMaxRhs];
    double relres[kMaxRhs];
    double aux[kMaxRhs];     // true residual (b - S x, b - S x)_w at the end
    double rho0[kMaxRhs];    // inner solves: (r, r)_w at the start of the inner solve
    double tau[kMaxRhs];     // inner solves: relative tolerance of this inner solve
    int32_t iters[kMaxRhs];  // FP64: iterations; SSG_MIXED outer state: inner iterations summed
    int32_t outer[kMaxRhs];  // SSG_MIXED: refinements
    int32_t status[kMaxRhs];
    uint32_t act;
    uint32_t act_b;          // act as the residual update left it (hand-off to the x/p update)
    int32_t iter;            // completed loop iterations
    int32_t iter_b;
    int32_t max_iter;
    int32_t nrhs;            // columns in use (the rest are padding)
    double rtol;
    double inner_rtol;
    int32_t max_outer;
    int32_t guess;
    int32_t halt[2];
    int32_t done;
    int32_t loops;           // SSG_MIXED outer state: inner loop iterations summed (launch count)
};

template <typename T>
struct SpmmTraits;
template <>
struct SpmmTraits<double> {
    static constexpr int kBlocksPerSM = 2;  // K FP64 accumulators and two entries' rows in flight per lane
};
template <>
struct SpmmTraits<float> {
    static constexpr int kBlocksPerSM = 4;
};

// Sliced-ELL entries a lane loads at once in the K-vector product (before
// their x rows), the default of the autotuner (ssg_autotune_block times 1
// and 2): one with K >= 8 FP64 columns (register room), else two.
template <typename T, int K>
constexpr int spmm_nc_default() {
    return (sizeof(T) == 8 && K >= 8) ? 1 : 2;
}

// K contiguous values of one local entry.
template <int K>
__device__ __forceinline__ void load_row(const double *__restrict__ p, double (&v)[K]) {
    const double2 *p2 = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int q = 0; q < K / 2; ++q) {
        const double2 t = __ldg(p2 + q);
        v[2 * q] = t.x;
        v[2 * q + 1] = t.y;
    }
}
template <int K>
__device__ __forceinline__ void load_row(const float *__restrict__ p, float (&v)[K]) {
    if constexpr (K >= 4) {
        const float4 *p4 = reinterpret_cast<const float4 *>(p);
#pragma unroll
        for (int q = 0; q < K / 4; ++q) {
            const float4 t = __ldg(p4 + q);
            v[4 * q] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
        }
    } else {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = t.x;
        v[1] = t.y;
    }
}
template <int K>
__device__ __forceinline__ void store_row(double *__restrict__ p, const double (&v)[K]) {
    double2 *p2 = reinterpret_cast<double2 *>(p);
#pragma unroll
    for (int q = 0; q < K / 2; ++q) p2[q] = make_double2(v[2 * q], v[2 * q + 1]);
}
template <int K>
__device__ __forceinline__ void store_row(float *__restrict__ p, const float (&v)[K]) {
    if constexpr (K >= 4) {
        float4 *p4 = reinterpret_cast<float4 *>(p);
#pragma unroll
        for (int q = 0; q < K / 4; ++q) p4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    }
}

// Segment tables (host-built, see api.cu).
struct SegTab {
    const int32_t *blk_seg;    // [product grid] segment of each block of the K-vector product
    const int32_t *seg_blk;    // [nseg + 1] product blocks of each segment
    const int4 *chunk;         // [nchunks] (segment, first local entry, end local entry, 0)
    const int32_t *seg_chunk;  // [nseg + 1] chunks of each segment
    const int32_t *node_off;   // [nseg + 1] first global node of each segment
    const int64_t *rhs_off;    // [nseg] first value of the segment's right-hand sides in b / x
    const int32_t *nrhs;       // [nseg] right-hand sides of the segment (columns >= nrhs are padding)
    int32_t nseg;
};

// Lane layout of the K-vector product: each lane holds VW consecutive
// columns of one row (one 16-byte vector when K values take 16 bytes or
// more), LPR lanes cover a row, a warp covers RPP rows of a 32-row slice per
// pass and LPR passes cover the slice.  The x and y rows of one pass are
// then contiguous 16-byte pieces (a coalesced request per row) and the
// slice's value and column loads are broadcasts.
template <typename T, int K>
struct SpmmShape {
    static constexpr int VW = (K * (int)sizeof(T) >= 16) ? 16 / (int)sizeof(T) : K;
    static constexpr int LPR = K / VW;
    static constexpr int RPP = 32 / LPR;
};

template <int VW>
__device__ __forceinline__ void load_vec(const double *__restrict__ p, double (&v)[VW]) {
    const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
    v[0] = t.x;
    v[1] = t.y;
}
template <int VW>
__device__ __forceinline__ void load_vec(const float *__restrict__ p, float (&v)[VW]) {
    if constexpr (VW == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    } else {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = t.x, v[1] = t.y;
    }
}
template <int VW>
__device__ __forceinline__ void store_vec(double *__restrict__ p, const double (&v)[VW]) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}
template <int VW>
__device__ __forceinline__ void store_vec(float *__restrict__ p, const float (&v)[VW]) {
    if constexpr (VW == 4)
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
}

// NC consecutive sliced-ELL entries for the lane's LPR rows of a slice (row
// p * RPP + rl in pass p) and its VW columns: value and column loads
// (broadcast within a row's lanes), then the NC * LPR x pieces, then the FMAs
// in CSR order.
template <int NC, int LPR, int RPP, int VW, int K, typename T>
__device__ __forceinline__ void slice_chunk_v(const T *__restrict__ sv, const int32_t *__restrict__ sc,
                                              const T *__restrict__ X, int base, int k0, int col0,
                                              T (&acc)[LPR][VW]) {
    T v[NC][LPR];
    int c[NC][LPR];
#pragma unroll
    for (int e = 0; e < NC; ++e)
#pragma unroll
        for (int p = 0; p < LPR; ++p) {
            v[e][p] = __ldcs(sv + base + p * RPP + (k0 + e) * kSliceRows);
            c[e][p] = __ldcs(sc + base + p * RPP + (k0 + e) * kSliceRows);
        }
    T xv[NC][LPR][VW];
#pragma unroll
    for (int e = 0; e < NC; ++e)
#pragma unroll
        for (int p = 0; p < LPR; ++p) load_vec<VW>(X + (size_t)c[e][p] * K + col0, xv[e][p]);
#pragma unroll
    for (int e = 0; e < NC; ++e)
#pragma unroll
        for (int p = 0; p < LPR; ++p)
#pragma unroll
            for (int u = 0; u < VW; ++u) acc[p][u] = fma(v[e][p], xv[e][p][u], acc[p][u]);
}

// Sub-structured product with K vectors: Y = S X, then (with DOTS) each
// block's partial of (x_j, y_j)_w at partials[block * K + j].  The work list
// and the summation orders (CSR order inside a row, ascending subdomain at
// an interface node) are those of the single-vector kernel, so every column
// is bit-identical to it.  NC: sliced entries loaded at once; A.l2_ahead:
// slices ahead prefetched into L2 (neither changes the arithmetic).
template <typename T, int K, bool DOTS, int NC = spmm_nc_default<T, K>()>
__device__ __forceinline__ void spmm_body(const DevOp &A, const T *__restrict__ X, T *__restrict__ Y,
                                          double *partials) {
    using Sh = SpmmShape<T, K>;
    constexpr int VW = Sh::VW, LPR = Sh::LPR, RPP = Sh::RPP;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane % LPR, rl = lane / LPR, col0 = sub * VW;
    const int2 range = A.warp_range[blockIdx.x * kSpmvWarps + warp];
    const T *__restrict__ sv = slice_vals<T>(A);
    const T *__restrict__ val = row_vals<T>(A);
    const T *__restrict__ ival = copy_vals<T>(A);
    __shared__ T stage[kSpmvWarps][kSliceRows][K];  // copy-row products of an interface slice
    T dot[VW];
#pragma unroll
    for (int u = 0; u < VW; ++u) dot[u] = T(0);
    for (int it = range.x; it < range.y; ++it) {
        const WorkItem W = A.items[it];
        if (A.l2_ahead > 0 && it + A.l2_ahead < range.y) {
            const WorkItem Wp = A.items[it + A.l2_ahead];
            if (sliced_item(Wp.kind) && lane < Wp.e1) {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(sv + Wp.e0 + lane * kSliceRows));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(A.scol + Wp.e0 + lane * kSliceRows));
            }
        }
        if (sliced_item(W.kind)) {
            const bool iface = W.kind == kItemIfaceSlice;
            const bool sorted = W.kind == kItemSortedSlice;
            T acc[LPR][VW];
#pragma unroll
            for (int p = 0; p < LPR; ++p)
#pragma unroll
                for (int u = 0; u < VW; ++u) acc[p][u] = T(0);
            const int base = W.e0 + rl;
            int k = 0;
            for (; k + NC <= W.e1; k += NC)
                slice_chunk_v<NC, LPR, RPP, VW, K, T>(sv, A.scol, X, base, k, col0, acc);
            for (; k < W.e1; ++k) slice_chunk_v<1, LPR, RPP, VW, K, T>(sv, A.scol, X, base, k, col0, acc);
#pragma unroll
            for (int pass = 0; pass < LPR; ++pass) {
                const int sr = pass * RPP + rl;
                if (!iface) {
                    const int slot = W.a + sr;
                    if (slot < W.b) {
                        const int r = sorted ? __ldg(A.srow + slot) : slot;
                        store_vec<VW>(Y + (size_t)r * K + col0, acc[pass]);
                        if (DOTS) {
                            T xr[VW];
                            load_vec<VW>(X + (size_t)r * K + col0, xr);
#pragma unroll
                            for (int u = 0; u < VW; ++u) dot[u] = fma(xr[u], acc[pass][u], dot[u]);
                        }
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < VW; ++u) stage[warp][sr][col0 + u] = acc[pass][u];
                }
            }
            if (iface) {
                __syncwarp();
#pragma unroll
                for (int pass = 0; pass < LPR; ++pass) {
                    const int sr = pass * RPP + rl;
                    const int c = W.a + sr;
                    if (c < W.b) {
                        const int seg = __ldg(A.sseg + c);
                        const int l0 = seg & 0xff, m = seg >> 8;
                        T S[VW];
#pragma unroll
                        for (int u = 0; u < VW; ++u) S[u] = stage[warp][l0][col0 + u];
                        for (int t = 1; t < m; ++t)
#pragma unroll
                            for (int u = 0; u < VW; ++u) S[u] += stage[warp][l0 + t][col0 + u];
                        const int row = __ldg(A.icopy + c);
                        store_vec<VW>(Y + (size_t)row * K + col0, S);
                        if (DOTS) {
                            const T w = copy_weight<T>(A, m, row);
                            T xr[VW];
                            load_vec<VW>(X + (size_t)row * K + col0, xr);
#pragma unroll
                            for (int u = 0; u < VW; ++u) dot[u] = fma(w * xr[u], S[u], dot[u]);
                        }
                    }
                }
                __syncwarp();
            }
        } else if (W.kind == kItemLongRow) {
            // one long row, VW columns at a time: lane-strided partial sums and
            // the fixed warp tree of the single-vector kernel for every column
            for (int g0 = 0; g0 < K; g0 += VW) {
                T acc[VW];
#pragma unroll
                for (int u = 0; u < VW; ++u) acc[u] = T(0);
                for (int k = W.e0 + lane; k < W.e1; k += 32) {
                    const T v = val[k];
                    T xv[VW];
                    load_vec<VW>(X + (size_t)A.col[k] * K + g0, xv);
#pragma unroll
                    for (int u = 0; u < VW; ++u) acc[u] = fma(v, xv[u], acc[u]);
                }
#pragma unroll
                for (int u = 0; u < VW; ++u) acc[u] = T(warp_sum(double(acc[u])));  // valid in lane 0
                if (lane == 0) {
                    store_vec<VW>(Y + (size_t)W.a * K + g0, acc);
#pragma unroll
                    for (int u = 0; u < VW; ++u) stage[warp][0][g0 + u] = acc[u];
                }
            }
            __syncwarp();
            if (DOTS && rl == 0) {
                T xr[VW];
                load_vec<VW>(X + (size_t)W.a * K + col0, xr);
#pragma unroll
                for (int u = 0; u < VW; ++u) dot[u] = fma(xr[u], stage[warp][0][col0 + u], dot[u]);
            }
            __syncwarp();
        } else {
            // one interface node with long copy rows, VW columns at a time: each
            // copy row reduced by the warp (fixed tree), copies summed in
            // ascending s
            for (int g0 = 0; g0 < K; g0 += VW) {
                T S[VW];
#pragma unroll
                for (int u = 0; u < VW; ++u) S[u] = T(0);
                for (int c = W.c0; c < W.c1; ++c) {
                    T acc[VW];
#pragma unroll
                    for (int u = 0; u < VW; ++u) acc[u] = T(0);
                    for (int k = A.irp[c] + lane; k < A.irp[c + 1]; k += 32) {
                        const T v = ival[k];
                        T xv[VW];
                        load_vec<VW>(X + (size_t)A.icol[k] * K + g0, xv);
#pragma unroll
                        for (int u = 0; u < VW; ++u) acc[u] = fma(v, xv[u], acc[u]);
                    }
#pragma unroll
                    for (int u = 0; u < VW; ++u) S[u] += T(warp_sum(double(acc[u])));  // valid in lane 0
                }
                if (lane == 0) {
#pragma unroll
                    for (int u = 0; u < VW; ++u) stage[warp][0][g0 + u] = S[u];
                }
            }
            __syncwarp();
            if (rl == 0) {
                T Sv[VW];
#pragma unroll
                for (int u = 0; u < VW; ++u) Sv[u] = stage[warp][0][col0 + u];
                for (int c = W.c0; c < W.c1; ++c) {
                    const int row = A.icopy[c];
                    store_vec<VW>(Y + (size_t)row * K + col0, Sv);
                    if (DOTS) {
                        const T w = copy_weight<T>(A, W.c1 - W.c0, row);
                        T xr[VW];
                        load_vec<VW>(X + (size_t)row * K + col0, xr);
#pragma unroll
                        for (int u = 0; u < VW; ++u) dot[u] = fma(w * xr[u], Sv[u], dot[u]);
                    }
                }
            }
            __syncwarp();
        }
    }
    if (DOTS) {
        __shared__ double wsum[kSpmvWarps][K];
        // lanes holding the same columns (equal lane mod LPR) are summed by a fixed xor tree
        double dv[VW];
#pragma unroll
        for (int u = 0; u < VW; ++u) {
            dv[u] = double(dot[u]);
#pragma unroll
            for (int o = 16; o >= LPR; o >>= 1) dv[u] += __shfl_xor_sync(0xffffffffu, dv[u], o);
        }
        if (rl == 0) {
#pragma unroll
            for (int u = 0; u < VW; ++u) wsum[warp][col0 + u] = dv[u];
        }
        __syncthreads();
        if (threadIdx.x < K) {
            double bs = wsum[0][threadIdx.x];
#pragma unroll
            for (int w = 1; w < kSpmvWarps; ++w) bs += wsum[w][threadIdx.x];
            partials[(size_t)blockIdx.x * K + threadIdx.x] = bs;
        }
    }
}

// The K-vector product of ssg_spmm_assembled (no state, no partials).
template <typename T, int K>
__global__ void __launch_bounds__(kSpmvThreads, SpmmTraits<T>::kBlocksPerSM)
    k_spmm_asm(DevOp A, const T *__restrict__ X, T *__restrict__ Y) {
    spmm_body<T, K, false>(A, X, Y, nullptr);
}

// The K-vector product inside the solves: blocks of a segment whose columns
// are all frozen (segs given) return at once.
template <typename T, int K, bool DOTS, int NC>
__global__ void __launch_bounds__(kSpmvThreads, SpmmTraits<T>::kBlocksPerSM)
    k_spmm_seg(DevOp A, const T *__restrict__ X, T *__restrict__ Y, double *partials, SegTab tab,
               const ScalB *segs) {
    if (segs && segs[tab.blk_seg[blockIdx.x]].act == 0) return;
    spmm_body<T, K, DOTS, NC>(A, X, Y, partials);
}

// Sums of each column's partials over blocks [b0, b1) of the previous kernel
// (K per block), the same fixed order in every block: warp w takes the
// columns j = w mod 8; lane l adds the blocks b0 + l + 32 i into accumulator
// i mod 8 (eight loads in flight instead of a chain of dependent ones), the
// accumulators are combined as a fixed tree, then the lanes by a fixed
// shuffle tree.  Result in tot[K] (shared), valid after the call in every
// thread.
template <int K, int NT = kBlockV>
__device__ __forceinline__ void seg_sum_cols(const double *partials, int b0, int b1, double *tot) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = warp; j < K; j += NT / 32) {
        double a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = 0.0;
        int g = b0 + lane;
        for (; g + 7 * 32 < b1; g += 8 * 32) {
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] += __ldcg(partials + (size_t)(g + 32 * u) * K + j);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (g + 32 * u < b1) a[u] += __ldcg(partials + (size_t)(g + 32 * u) * K + j);
        double v = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
        v = warp_sum(v);
        if (lane == 0) tot[j] = v;
    }
    __syncthreads();
}

// Per-column block sum of thread accumulators.  Thread t holds acc[u] for
// the column (VW t + u) mod K (true when the element loop starts at a
// multiple of K and strides by a multiple of K, as all loops below do); the
// block's sums go to out[0..K).
template <int K, int VW, typename A>
__device__ __forceinline__ void block_cols_sum(const A (&acc)[VW], double *out) {
    __shared__ A red[kBlockV * VW];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < VW; ++u) red[threadIdx.x * VW + u] = acc[u];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kPer = kBlockV * VW / K;  // entries per column
    for (int j = warp; j < K; j += kBlockV / 32) {
        A v = A(0);
        for (int i = lane; i < kPer; i += 32) v += red[i * K + j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) out[j] = double(v);
    }
}

// One block: the loop condition of a segmented loop (any segment with an
// active column continues), the loop count in glob->iter (reset: set to 0
// instead of counted), and the running count of inner iterations in
// count->loops when count is given.
__global__ void __launch_bounds__(kBlock) k_seg_cond(const ScalB *segs, int nseg, ScalB *glob, ScalB *count,
                                                     int reset, cudaGraphConditionalHandle h, int use_cond) {
    int any = 0;
    for (int sg = threadIdx.x; sg < nseg; sg += kBlock) any |= segs[sg].act != 0;
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        glob->iter = reset ? 0 : glob->iter + 1;
        if (reset) glob->loops = 0;
        if (count && !reset) count->loops += 1;
        glob->done = !any;
        if (use_cond) cudaGraphSetConditional(h, any ? 1u : 0u);
    }
}

// Algorithm 3 lines 3 and 5 for K columns (FP64), one block per chunk:
// alpha_j = rho_j / (p_j, S p_j)_w for every active column of the chunk's
// segment (a column with (p, S p)_w <= 0 stops with a breakdown),
// r_j <- r_j - alpha_j q_j over the chunk and its partials of (r_j, r_j)_w
// at part_rr[chunk*K + j].  With the diagonal preconditioner (PC, dinv =
// 1 / diag(S) per local entry, shared by the K columns) also the partials of
// (r_j, z_j)_w, z = dinv r, at part_rr[(nchunks + chunk)*K + j].
template <int K, bool PC = false>
__global__ void __launch_bounds__(kBlockV, 1) k_update_rB(const double *__restrict__ q, double *__restrict__ r,
                                                      const uint8_t *__restrict__ mult,
                                                      const double *__restrict__ wtab,
                                                      const uint8_t *__restrict__ gflag, const double *part_pq,
                                                      double *part_rr, SegTab tab, ScalB *segs,
                                                      const double *__restrict__ dinv = nullptr) {
    __shared__ double tot[K];
    __shared__ double alpha_s[K];
    const int4 ch = tab.chunk[blockIdx.x];
    ScalB *s = segs + ch.x;
    const bool first = (int)blockIdx.x == tab.seg_chunk[ch.x];
    const uint32_t act = s->act;
    if (first && threadIdx.x == 0) {
        for (int j = 0; j < K; ++j) s->rho_b[j] = s->rho[j];
        s->iter_b = s->iter;
        if (!act) s->act_b = 0;
    }
    if (!act) return;
    const int j0 = (2 * threadIdx.x) % K;
    double a0 = 0.0, a1 = 0.0;
    double acc[2] = {0.0, 0.0}, acz[2] = {0.0, 0.0};
    double2 *__restrict__ r2 = reinterpret_cast<double2 *>(r);
    const double2 *__restrict__ q2 = reinterpret_cast<const double2 *>(q);
    struct Ld {
        double2 r, q;
        double d;
        uint8_t g;
    };
    stream_loop_after<PC ? 2 : 4>(
        (int64_t)ch.y * K / 2 + threadIdx.x, (int64_t)ch.z * K / 2, kBlockV,
        [&](int64_t i) {
            Ld l;
            l.r = r2[i];
            l.q = __ldcs(q2 + i);
            l.g = __ldg(gflag + (((2 * i) / K) >> 6));
            if (PC) l.d = __ldg(dinv + (2 * i) / K);  // local entry of both values
            return l;
        },
        [&]() {
            seg_sum_cols<K>(part_pq, tab.seg_blk[ch.x], tab.seg_blk[ch.x + 1], tot);
            if (threadIdx.x < K) {
                const int j = threadIdx.x;
                const double pq = tot[j];
                double a = 0.0;
                if (((act >> j) & 1u) && pq > 0.0 && isfinite(pq)) a = s->rho[j] / pq;
                alpha_s[j] = a;
            }
            __syncthreads();
            if (first && threadIdx.x == 0) {
                uint32_t ab = act;
                for (int j = 0; j < K; ++j) {
                    if (!((act >> j) & 1u)) continue;
                    const double pq = tot[j];
                    s->pq[j] = pq;
                    s->alpha[j] = alpha_s[j];
                    if (!(pq > 0.0) || !isfinite(pq)) {
                        s->status[j] = SSG_E_BREAKDOWN;
                        ab &= ~(1u << j);
                    }
                }
                s->act_b = ab;
            }
            a0 = alpha_s[j0];
            a1 = alpha_s[j0 + 1];
            return true;
        },
        [&](int64_t i, Ld l) {
            double2 rv = l.r;
            rv.x = fma(-a0, l.q.x, rv.x);
            rv.y = fma(-a1, l.q.y, rv.y);
            r2[i] = rv;
            // weight 1 (no lookup) in 64-entry groups without interface copies;
            // the group is the same for the whole warp, tested by a vote so the
            // multiplies are branched over rather than issued predicated off
            double wx = rv.x, wy = rv.y;
            if (__any_sync(__activemask(), l.g != 0)) {
                const double w = __ldg(wtab + mult[(2 * i) / K]);  // local entry of both values
                wx = w * rv.x;
                wy = w * rv.y;
            }
            acc[0] = fma(wx, rv.x, acc[0]);
            acc[1] = fma(wy, rv.y, acc[1]);
            if (PC) {
                acz[0] = fma(wx, rv.x * l.d, acz[0]);
                acz[1] = fma(wy, rv.y * l.d, acz[1]);
            }
        });
    block_cols_sum<K, 2>(acc, part_rr + (size_t)blockIdx.x * K);
    if (PC) block_cols_sum<K, 2>(acz, part_rr + (size_t)(gridDim.x + blockIdx.x) * K);
}

// Algorithm 3 lines 4, 7, 8 for K columns (FP64), one block per chunk:
// beta_j = (r_j, r_j)_w / rho_j, x_j <- x_j + alpha_j p_j, p_j <- r_j +
// beta_j p_j (alpha = beta = 0 for frozen columns); the segment's first chunk
// records each column's iteration and stopping decision.
template <int K, bool PC = false>
__global__ void __launch_bounds__(kBlockV, 1) k_update_xpB(double *__restrict__ x, double *__restrict__ p,
                                                       const double *__restrict__ r, const double *part_rr,
                                                       SegTab tab, ScalB *segs,
                                                       const double *__restrict__ dinv = nullptr) {
    __shared__ double tot[K], totz[K];
    __shared__ double alpha_s[K], beta_s[K];
    const int4 ch = tab.chunk[blockIdx.x];
    ScalB *s = segs + ch.x;
    const bool first = (int)blockIdx.x == tab.seg_chunk[ch.x];
    const uint32_t ab = s->act_b;
    if (!ab) {
        if (first && threadIdx.x == 0) s->act = 0;
        return;
    }
    const int k = s->iter_b;
    const int j0 = (2 * threadIdx.x) % K;
    double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
    double2 *x2 = reinterpret_cast<double2 *>(x);
    double2 *p2 = reinterpret_cast<double2 *>(p);
    const double2 *r2 = reinterpret_cast<const double2 *>(r);
    struct Ld {
        double2 p, x, r;  // r: z = dinv r with PC
    };
    stream_loop_after<PC ? 2 : 4>(
        (int64_t)ch.y * K / 2 + threadIdx.x, (int64_t)ch.z * K / 2, kBlockV,
        [&](int64_t i) {
            Ld l;
            l.p = p2[i];
            l.x = __ldcs(x2 + i);
            l.r = r2[i];
            if (PC) {
                const double dv = __ldg(dinv + (2 * i) / K);
                l.r.x *= dv;
                l.r.y *= dv;
            }
            return l;
        },
        [&]() {
            seg_sum_cols<K>(part_rr, tab.seg_chunk[ch.x], tab.seg_chunk[ch.x + 1], tot);
            if (PC) seg_sum_cols<K>(part_rr + (size_t)gridDim.x * K, tab.seg_chunk[ch.x], tab.seg_chunk[ch.x + 1], totz);
            if (threadIdx.x < K) {
                const int j = threadIdx.x;
                const bool on = (ab >> j) & 1u;
                alpha_s[j] = on ? s->alpha[j] : 0.0;
                beta_s[j] = on ? (PC ? totz[j] : tot[j]) / s->rho_b[j] : 0.0;
            }
            __syncthreads();
            a0 = alpha_s[j0];
            a1 = alpha_s[j0 + 1];
            b0 = beta_s[j0];
            b1 = beta_s[j0 + 1];
            return true;
        },
        [&](int64_t i, Ld l) {
            double2 xv = l.x;
            xv.x = fma(a0, l.p.x, xv.x);
            xv.y = fma(a1, l.p.y, xv.y);
            __stcs(x2 + i, xv);
            p2[i] = make_double2(fma(b0, l.p.x, l.r.x), fma(b1, l.p.y, l.r.y));
        });
    if (first && threadIdx.x == 0) {
        uint32_t na = ab;
        for (int j = 0; j < K; ++j) {
            if (!((ab >> j) & 1u)) continue;
            const double rr = tot[j];
            s->rho[j] = PC ? totz[j] : rr;
            s->rrt[j] = rr;
            s->iters[j] = k + 1;
            s->relres[j] = s->bnorm[j] > 0.0 ? sqrt(rr) / s->bnorm[j] : 0.0;
            if (sqrt(rr) <= s->rtol * s->bnorm[j]) {
                s->status[j] = SSG_OK;
                na &= ~(1u << j);
            }
        }
        s->iter = k + 1;
        if (na && k + 1 >= s->max_iter) {
            for (int j = 0; j < K; ++j)
                if ((na >> j) & 1u) s->status[j] = SSG_E_NOT_CONVERGED;
            na = 0;
        }
        s->act = na;
    }
}

// Setup of Algorithm 3 line 1 for K columns, one block per chunk: r = b - q
// (use_q; q = S x_1 with a guess, else zeros) or r = b, p = z when p is
// given (z = r, or z = dinv r with the diagonal preconditioner, PC), and the
// chunk's partials of (r_j, r_j)_w (part[chunk*K + j]), with with_b of
// (b_j, b_j)_w (part[(nchunks + chunk)*K + j]) and with PC of (r_j, z_j)_w
// (part[(2 nchunks + chunk)*K + j]).  With p == nullptr this is the FP64
// residual of the refinement; with r == nullptr only the norms are formed
// (the true residual at the end of a solve).
template <int K, bool PC = false>
__global__ void __launch_bounds__(kBlockV, 1) k_residualB(const double *__restrict__ b, const double *__restrict__ q,
                                                      double *__restrict__ r, double *__restrict__ p,
                                                      const uint8_t *__restrict__ mult,
                                                      const double *__restrict__ wtab, double *part, SegTab tab,
                                                      int use_q, int with_b, const double *__restrict__ dinv = nullptr) {
    const int4 ch = tab.chunk[blockIdx.x];
    double arr[2] = {0.0, 0.0}, abb[2] = {0.0, 0.0}, arz[2] = {0.0, 0.0};
    const double2 *b2 = reinterpret_cast<const double2 *>(b);
    const double2 *q2 = reinterpret_cast<const double2 *>(q);
    double2 *r2 = reinterpret_cast<double2 *>(r);
    double2 *p2 = reinterpret_cast<double2 *>(p);
    const int64_t i1 = (int64_t)ch.z * K / 2;
    for (int64_t i = (int64_t)ch.y * K / 2 + threadIdx.x; i < i1; i += kBlockV) {
        const double2 bv = b2[i];
        double2 rv = bv;
        if (use_q) {
            const double2 qv = q2[i];
            rv.x = bv.x - qv.x;
            rv.y = bv.y - qv.y;
        }
        double2 zv = rv;
        if (PC) {
            const double dv = __ldg(dinv + (2 * i) / K);
            zv.x *= dv;
            zv.y *= dv;
        }
        if (r) r2[i] = rv;
        if (p) p2[i] = zv;
        const double w = __ldg(wtab + mult[(2 * i) / K]);
        arr[0] = fma(w * rv.x, rv.x, arr[0]);
        arr[1] = fma(w * rv.y, rv.y, arr[1]);
        if (with_b) {
            abb[0] = fma(w * bv.x, bv.x, abb[0]);
            abb[1] = fma(w * bv.y, bv.y, abb[1]);
        }
        if (PC) {
            arz[0] = fma(w * rv.x, zv.x, arz[0]);
            arz[1] = fma(w * rv.y, zv.y, arz[1]);
        }
    }
    block_cols_sum<K, 2>(arr, part + (size_t)blockIdx.x * K);
    if (with_b) block_cols_sum<K, 2>(abb, part + (size_t)(gridDim.x + blockIdx.x) * K);
    if (PC) block_cols_sum<K, 2>(arz, part + (size_t)(2 * gridDim.x + blockIdx.x) * K);
}

// Parameters of every segment's solve (one thread per segment); nr_single > 0
// sets the right-hand-side count of a one-segment solve.
__global__ void k_set_paramsB(ScalB *segs, int nseg, double rtol, int32_t max_iter, int32_t guess,
                              double inner_rtol, int32_t max_outer, int32_t *nrhs, int nr_single) {
    if (nr_single > 0 && blockIdx.x == 0 && threadIdx.x == 0) nrhs[0] = nr_single;
    for (int sg = blockIdx.x * blockDim.x + threadIdx.x; sg < nseg; sg += gridDim.x * blockDim.x) {
        ScalB *s = segs + sg;
        s->rtol = rtol;
        s->max_iter = max_iter;
        s->guess = guess;
        s->inner_rtol = inner_rtol;
        s->max_outer = max_outer;
        s->done = 0;
    }
}

// One block per segment, after k_residualB (with_b) of the setup: rho_j,
// ||b_j||_w and the test before the first iteration.
template <int K, bool PC = false>
__global__ void __launch_bounds__(kBlock) k_init_finB(const double *part, int nchunks, SegTab tab, ScalB *segs) {
    __shared__ double rr[K], bb[K], rz[K];
    const int sg = blockIdx.x;
    ScalB *s = segs + sg;
    seg_sum_cols<K, kBlock>(part, tab.seg_chunk[sg], tab.seg_chunk[sg + 1], rr);
    seg_sum_cols<K, kBlock>(part + (size_t)nchunks * K, tab.seg_chunk[sg], tab.seg_chunk[sg + 1], bb);
    if (PC) seg_sum_cols<K, kBlock>(part + (size_t)2 * nchunks * K, tab.seg_chunk[sg], tab.seg_chunk[sg + 1], rz);
    if (threadIdx.x == 0) {
        const int nr = tab.nrhs[sg];
        uint32_t act = 0;
        for (int j = 0; j < K; ++j) {
            s->rho[j] = PC ? rz[j] : rr[j];
            s->rho_b[j] = s->rho[j];
            s->rrt[j] = rr[j];
            s->bnorm[j] = sqrt(bb[j]);
            s->relres[j] = s->bnorm[j] > 0.0 ? sqrt(rr[j]) / s->bnorm[j] : 0.0;
            s->iters[j] = 0;
            s->outer[j] = 0;
            s->alpha[j] = 0.0;
            s->pq[j] = 0.0;
            s->aux[j] = 0.0;
            if (j >= nr || sqrt(rr[j]) <= s->rtol * s->bnorm[j]) {
                s->status[j] = SSG_OK;
            } else {
                s->status[j] = SSG_E_NOT_CONVERGED;
                if (s->max_iter > 0) act |= 1u << j;
            }
        }
        s->nrhs = nr;
        s->act = act;
        s->act_b = act;
        s->iter = 0;
        s->iter_b = 0;
        s->loops = 0;
        s->done = act == 0;
    }
}

// ---------------------------------------------------------------------------
// SSG_MIXED for K columns: FP32 inner CG inside FP64 iterative refinement.
// Outer state so[seg] (act = columns still refining, iters = inner
// iterations summed, outer = refinements); inner state si[seg] (act = columns
// still in the current inner solve).
// ---------------------------------------------------------------------------

// Inner setup, one block per chunk: r32 = (float) r64, p32 = z32 (z32 = r32,
// or r32 * (1 / S_ii rounded to FP32) with the diagonal preconditioner, PC),
// d32 = 0 and the chunk's partials of (r32, r32)_w at part[chunk*K + j] and
// with PC of (r32, z32)_w at part[(nchunks + chunk)*K + j] (FP32 products and
// block sums).
template <int K, bool PC = false>
__global__ void __launch_bounds__(kBlockV, 1) k_inner_initB(const double *__restrict__ r64, float *__restrict__ r32,
                                                        float *__restrict__ p32, float *__restrict__ d32,
                                                        const uint8_t *__restrict__ mult,
                                                        const float *__restrict__ wtab, double *part, SegTab tab,
                                                        const float *__restrict__ dinv32 = nullptr) {
    const int4 ch = tab.chunk[blockIdx.x];
    float acc[2] = {0.f, 0.f}, acz[2] = {0.f, 0.f};
    const double2 *r2 = reinterpret_cast<const double2 *>(r64);
    float2 *rr2 = reinterpret_cast<float2 *>(r32);
    float2 *pp2 = reinterpret_cast<float2 *>(p32);
    float2 *dd2 = reinterpret_cast<float2 *>(d32);
    const int64_t i1 = (int64_t)ch.z * K / 2;
    for (int64_t i = (int64_t)ch.y * K / 2 + threadIdx.x; i < i1; i += kBlockV) {
        const double2 rv = r2[i];
        const float2 f = make_float2(float(rv.x), float(rv.y));
        float2 z = f;
        if (PC) {
            const float dv = __ldg(dinv32 + (2 * i) / K);
            z.x *= dv;
            z.y *= dv;
        }
        rr2[i] = f;
        pp2[i] = z;
        dd2[i] = make_float2(0.f, 0.f);
        const float w = __ldg(wtab + mult[(2 * i) / K]);
        acc[0] = fmaf(w * f.x, f.x, acc[0]);
        acc[1] = fmaf(w * f.y, f.y, acc[1]);
        if (PC) {
            acz[0] = fmaf(w * f.x, z.x, acz[0]);
            acz[1] = fmaf(w * f.y, z.y, acz[1]);
        }
    }
    block_cols_sum<K, 2>(acc, part + (size_t)blockIdx.x * K);
    if (PC) block_cols_sum<K, 2>(acz, part + (size_t)(gridDim.x + blockIdx.x) * K);
}

// One block per segment: rho0_j of the inner solves, their tolerances
// tau_j = max(inner_rtol, rtol ||b_j|| / ||r64_j||) and the active set.
template <int K, bool PC = false>
__global__ void __launch_bounds__(kBlock) k_inner_finB(const double *part, int nchunks, SegTab tab, ScalB *si,
                                                       const ScalB *so) {
    __shared__ double rr[K], rz[K];
    const int sg = blockIdx.x;
    seg_sum_cols<K, kBlock>(part, tab.seg_chunk[sg], tab.seg_chunk[sg + 1], rr);
    if (PC) seg_sum_cols<K, kBlock>(part + (size_t)nchunks * K, tab.seg_chunk[sg], tab.seg_chunk[sg + 1], rz);
    if (threadIdx.x == 0) {
        ScalB *i = si + sg;
        const ScalB *o = so + sg;
        uint32_t act = 0;
        for (int j = 0; j < K; ++j) {
            const double tot = rr[j];
            i->rho[j] = PC ? rz[j] : tot;
            i->rho_b[j] = i->rho[j];
            i->rrt[j] = tot;
            i->rho0[j] = tot;
            const double tau = o->bnorm[j] > 0.0 && o->rho[j] > 0.0 ? o->rtol * o->bnorm[j] / sqrt(o->rho[j]) : 0.0;
            i->tau[j] = tau > o->inner_rtol ? tau : o->inner_rtol;
            i->alpha[j] = 0.0;
            i->status[j] = SSG_OK;
            if (((o->act >> j) & 1u) && tot > 0.0 && o->iters[j] < o->max_iter) act |= 1u << j;
        }
        i->act = act;
        i->act_b = act;
        i->iter = 0;
        i->iter_b = 0;
        i->done = act == 0;
    }
}

// Inner Algorithm 3 lines 3 and 5 in FP32 for K columns, one block per chunk
// (alpha formed in FP64 from the FP64 sums of the partials, then rounded to
// FP32 once).
template <int K, bool PC = false>
__global__ void __launch_bounds__(kBlockV, 1) k_update_r32B(const float *__restrict__ q, float *__restrict__ r,
                                                        const uint8_t *__restrict__ mult,
                                                        const float *__restrict__ wtab,
                                                        const uint8_t *__restrict__ gflag128, const double *part_pq,
                                                        double *part_rr, SegTab tab, ScalB *si,
                                                        const float *__restrict__ dinv32 = nullptr) {
    constexpr int VW = K >= 4 ? 4 : 2;
    __shared__ double tot[K];
    __shared__ float alpha_s[K];
    const int4 ch = tab.chunk[blockIdx.x];
    ScalB *s = si + ch.x;
    const bool first = (int)blockIdx.x == tab.seg_chunk[ch.x];
    const uint32_t act = s->act;
    if (first && threadIdx.x == 0) {
        for (int j = 0; j < K; ++j) s->rho_b[j] = s->rho[j];
        s->iter_b = s->iter;
        if (!act) s->act_b = 0;
    }
    if (!act) return;
    const int j0 = (VW * threadIdx.x) % K;
    float a[VW];
    float acc[VW], acz[VW];
#pragma unroll
    for (int u = 0; u < VW; ++u) a[u] = acc[u] = acz[u] = 0.f;
    struct Ld {
        float r[VW], q[VW];
        float d;
        uint8_t g;
    };
    stream_loop_after<PC ? 2 : 4>(
        (int64_t)ch.y * K / VW + threadIdx.x, (int64_t)ch.z * K / VW, kBlockV,
        [&](int64_t i) {
            Ld l;
            if constexpr (VW == 4) {
                const float4 t = reinterpret_cast<const float4 *>(r)[i];
                const float4 u = __ldcs(reinterpret_cast<const float4 *>(q) + i);
                l.r[0] = t.x, l.r[1] = t.y, l.r[2] = t.z, l.r[3] = t.w;
                l.q[0] = u.x, l.q[1] = u.y, l.q[2] = u.z, l.q[3] = u.w;
            } else {
                const float2 t = reinterpret_cast<const float2 *>(r)[i];
                const float2 u = __ldcs(reinterpret_cast<const float2 *>(q) + i);
                l.r[0] = t.x, l.r[1] = t.y;
                l.q[0] = u.x, l.q[1] = u.y;
            }
            l.g = __ldg(gflag128 + (((VW * i) / K) >> 7));
            if (PC) l.d = __ldg(dinv32 + (VW * i) / K);  // local entry of the VW values
            return l;
        },
        [&]() {
            seg_sum_cols<K>(part_pq, tab.seg_blk[ch.x], tab.seg_blk[ch.x + 1], tot);
            if (threadIdx.x < K) {
                const int j = threadIdx.x;
                const double pq = tot[j];
                double a = 0.0;
                if (((act >> j) & 1u) && pq > 0.0 && isfinite(pq)) a = s->rho[j] / pq;
                alpha_s[j] = float(a);
                if (first && ((act >> j) & 1u)) {
                    s->pq[j] = pq;
                    s->alpha[j] = a;
                }
            }
            __syncthreads();
            if (first && threadIdx.x == 0) {
                uint32_t ab = act;
                for (int j = 0; j < K; ++j) {
                    if (!((act >> j) & 1u)) continue;
                    const double pq = tot[j];
                    if (!(pq > 0.0) || !isfinite(pq)) {
                        s->status[j] = SSG_E_BREAKDOWN;
                        ab &= ~(1u << j);
                    }
                }
                s->act_b = ab;
            }
#pragma unroll
            for (int u = 0; u < VW; ++u) a[u] = alpha_s[j0 + u];
            return true;
        },
        [&](int64_t i, Ld l) {
            float rv[VW];
#pragma unroll
            for (int u = 0; u < VW; ++u) rv[u] = fmaf(-a[u], l.q[u], l.r[u]);
            if constexpr (VW == 4)
                reinterpret_cast<float4 *>(r)[i] = make_float4(rv[0], rv[1], rv[2], rv[3]);
            else
                reinterpret_cast<float2 *>(r)[i] = make_float2(rv[0], rv[1]);
            float wr[VW];
#pragma unroll
            for (int u = 0; u < VW; ++u) wr[u] = rv[u];
            if (l.g != 0) {
                const float w = __ldg(wtab + mult[(VW * i) / K]);
#pragma unroll
                for (int u = 0; u < VW; ++u) wr[u] = w * rv[u];
            }
#pragma unroll
            for (int u = 0; u < VW; ++u) acc[u] = fmaf(wr[u], rv[u], acc[u]);
            if (PC) {
#pragma unroll
                for (int u = 0; u < VW; ++u) acz[u] = fmaf(wr[u], rv[u] * l.d, acz[u]);
            }
        });
    block_cols_sum<K, VW>(acc, part_rr + (size_t)blockIdx.x * K);
    if (PC) block_cols_sum<K, VW>(acz, part_rr + (size_t)(gridDim.x + blockIdx.x) * K);
}

// Inner Algorithm 3 lines 4, 7, 8 in FP32 for K columns, one block per chunk:
// d_j <- d_j + alpha_j p_j, p_j <- r_j + beta_j p_j; the segment's first chunk
// counts each active column's inner iteration and applies its inner test
// (sqrt(rho_j) <= tau_j sqrt(rho0_j), or its inner iterations summed reach
// max_iter).
template <int K, bool PC = false>
__global__ void __launch_bounds__(kBlockV, 1) k_update_dp32B(float *__restrict__ d, float *__restrict__ p,
                                                         const float *__restrict__ r, const double *part_rr,
                                                         SegTab tab, ScalB *si, ScalB *so,
                                                         const float *__restrict__ dinv32 = nullptr) {
    constexpr int VW = K >= 4 ? 4 : 2;
    __shared__ double tot[K], totz[K];
    __shared__ float alpha_s[K], beta_s[K];
    const int4 ch = tab.chunk[blockIdx.x];
    ScalB *s = si + ch.x;
    const bool first = (int)blockIdx.x == tab.seg_chunk[ch.x];
    const uint32_t ab = s->act_b;
    if (!ab) {
        if (first && threadIdx.x == 0) s->act = 0;
        return;
    }
    const int k = s->iter_b;
    const int j0 = (VW * threadIdx.x) % K;
    float a[VW], bt[VW];
    struct Ld {
        float p[VW], d[VW], r[VW];
    };
    stream_loop_after<2>(
        (int64_t)ch.y * K / VW + threadIdx.x, (int64_t)ch.z * K / VW, kBlockV,
        [&](int64_t i) {
            Ld l;
            if constexpr (VW == 4) {
                const float4 t = reinterpret_cast<const float4 *>(p)[i];
                const float4 u = reinterpret_cast<const float4 *>(d)[i];
                const float4 w = reinterpret_cast<const float4 *>(r)[i];
                l.p[0] = t.x, l.p[1] = t.y, l.p[2] = t.z, l.p[3] = t.w;
                l.d[0] = u.x, l.d[1] = u.y, l.d[2] = u.z, l.d[3] = u.w;
                l.r[0] = w.x, l.r[1] = w.y, l.r[2] = w.z, l.r[3] = w.w;
            } else {
                const float2 t = reinterpret_cast<const float2 *>(p)[i];
                const float2 u = reinterpret_cast<const float2 *>(d)[i];
                const float2 w = reinterpret_cast<const float2 *>(r)[i];
                l.p[0] = t.x, l.p[1] = t.y;
                l.d[0] = u.x, l.d[1] = u.y;
                l.r[0] = w.x, l.r[1] = w.y;
            }
            if (PC) {  // l.r becomes z = r * (1 / S_ii)
                const float dv = __ldg(dinv32 + (VW * i) / K);
#pragma unroll
                for (int u = 0; u < VW; ++u) l.r[u] *= dv;
            }
            return l;
        },
        [&]() {
            seg_sum_cols<K>(part_rr, tab.seg_chunk[ch.x], tab.seg_chunk[ch.x + 1], tot);
            if (PC) seg_sum_cols<K>(part_rr + (size_t)gridDim.x * K, tab.seg_chunk[ch.x], tab.seg_chunk[ch.x + 1], totz);
            if (threadIdx.x < K) {
                const int j = threadIdx.x;
                const bool on = (ab >> j) & 1u;
                alpha_s[j] = on ? float(s->alpha[j]) : 0.f;
                beta_s[j] = on ? float((PC ? totz[j] : tot[j]) / s->rho_b[j]) : 0.f;
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < VW; ++u) {
                a[u] = alpha_s[j0 + u];
                bt[u] = beta_s[j0 + u];
            }
            return true;
        },
        [&](int64_t i, Ld l) {
            float pv[VW], dv[VW];
#pragma unroll
            for (int u = 0; u < VW; ++u) {
                dv[u] = fmaf(a[u], l.p[u], l.d[u]);
                pv[u] = fmaf(bt[u], l.p[u], l.r[u]);
            }
            if constexpr (VW == 4) {
                reinterpret_cast<float4 *>(d)[i] = make_float4(dv[0], dv[1], dv[2], dv[3]);
                reinterpret_cast<float4 *>(p)[i] = make_float4(pv[0], pv[1], pv[2], pv[3]);
            } else {
                reinterpret_cast<float2 *>(d)[i] = make_float2(dv[0], dv[1]);
                reinterpret_cast<float2 *>(p)[i] = make_float2(pv[0], pv[1]);
            }
        });
    if (first && threadIdx.x == 0) {
        ScalB *o = so + ch.x;
        uint32_t na = ab;
        for (int j = 0; j < K; ++j) {
            if (!((ab >> j) & 1u)) continue;
            const double rr = tot[j];
            s->rho[j] = PC ? totz[j] : rr;
            s->rrt[j] = rr;
            const int t1 = o->iters[j] + 1;
            o->iters[j] = t1;
            if (sqrt(rr) <= s->tau[j] * sqrt(s->rho0[j]) || t1 >= o->max_iter) na &= ~(1u << j);
        }
        s->iter = k + 1;
        s->act = na;
    }
}

// One block per segment, after the refinement's residual (k_residualB
// without b): each refining column's outer decision (converged, inner
// breakdown, refinement or iteration cap).  With final_ != 0 it only stores
// the true residual of every column in aux.
template <int K>
__global__ void __launch_bounds__(kBlock) k_outer_finB(const double *part, SegTab tab, ScalB *so, const ScalB *si,
                                                       int final_) {
    __shared__ double rr[K];
    const int sg = blockIdx.x;
    seg_sum_cols<K, kBlock>(part, tab.seg_chunk[sg], tab.seg_chunk[sg + 1], rr);
    if (threadIdx.x != 0) return;
    ScalB *o = so + sg;
    if (final_) {
        for (int j = 0; j < K; ++j) o->aux[j] = rr[j];
        return;
    }
    const ScalB *i = si + sg;
    uint32_t na = o->act;
    for (int j = 0; j < K; ++j) {
        if (!((na >> j) & 1u)) continue;
        const double tot = rr[j];
        o->rho[j] = tot;
        o->outer[j] += 1;
        o->relres[j] = o->bnorm[j] > 0.0 ? sqrt(tot) / o->bnorm[j] : 0.0;
        int stop = 1;
        if (sqrt(tot) <= o->rtol * o->bnorm[j]) {
            o->status[j] = SSG_OK;
        } else if (i->status[j] == SSG_E_BREAKDOWN) {
            o->status[j] = SSG_E_BREAKDOWN;
        } else if (o->outer[j] >= o->max_outer || o->iters[j] >= o->max_iter) {
            o->status[j] = SSG_E_NOT_CONVERGED;
        } else {
            stop = 0;
        }
        if (stop) na &= ~(1u << j);
    }
    o->act = na;
    o->iter += 1;
}

// Global right-hand sides <-> interleaved local blocks (nloc x K), one block
// per chunk.  Segment sg's right-hand side j (< nrhs[sg]) starts at
// rhs_off[sg] + j * n_sg, node g of the segment at offset g - node_off[sg];
// columns nrhs..K-1 of the block are zero.
template <int K>
__global__ void __launch_bounds__(kBlockV, 1) k_scatterB(const int32_t *__restrict__ l2g, const double *__restrict__ xg,
                                                     double *__restrict__ xl, SegTab tab) {
    const int4 ch = tab.chunk[blockIdx.x];
    const int sg = ch.x;
    const int nr = tab.nrhs[sg];
    const int64_t n0 = tab.node_off[sg], ns = tab.node_off[sg + 1] - n0, ro = tab.rhs_off[sg];
    for (int64_t e = (int64_t)ch.y * K + threadIdx.x; e < (int64_t)ch.z * K; e += kBlockV) {
        const int64_t i = e / K;
        const int j = (int)(e % K);
        xl[e] = j < nr ? __ldg(xg + ro + j * ns + (l2g[i] - n0)) : 0.0;
    }
}

// Owner copies of the local blocks -> global right-hand-side layout.
template <int K>
__global__ void __launch_bounds__(kBlockV, 1) k_gatherB(const int32_t *__restrict__ l2g, const int32_t *__restrict__ own,
                                                    const double *__restrict__ xl, double *__restrict__ xg,
                                                    SegTab tab) {
    const int4 ch = tab.chunk[blockIdx.x];
    const int sg = ch.x;
    const int nr = tab.nrhs[sg];
    const int64_t n0 = tab.node_off[sg], ns = tab.node_off[sg + 1] - n0, ro = tab.rhs_off[sg];
    for (int64_t e = (int64_t)ch.y * K + threadIdx.x; e < (int64_t)ch.z * K; e += kBlockV) {
        const int64_t i = e / K;
        const int j = (int)(e % K);
        if (j >= nr) continue;
        const int32_t g = l2g[i];
        if (own[g] != i) continue;
        xg[ro + j * ns + (g - n0)] = xl[e];
    }
}

}  // namespace ssg
