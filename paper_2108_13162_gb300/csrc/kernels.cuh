// Device kernels of the sub-structured CG (sm_103a).
//
// Vectors are concatenated local vectors (Section 3.4.1): entry k belongs to
// one subdomain's V_s; interface nodes have one entry per subdomain holding
// them.  Inside each subdomain the interior rows come first and the
// interface rows last (Eq. 2.4:eqn0), so the interior rows of all subdomains
// form contiguous ranges that the SpMV tiles stream through.
//
// Reductions are deterministic: every block reduces its values in a fixed
// order, writes one partial, and the last block to arrive (an atomic ticket,
// no waiting) sums the partials in a fixed order and applies the scalar step
// of Algorithm 3 (alpha, beta, the stopping test).
//
// GB300 executes 2 FP64 FMAs per clock per SM, so every FP64 instruction
// counts: the block reduction runs its adds in one warp (12 warp-level adds
// per block) and interior entries (weight 1) skip the weight multiply.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ssg.h"

namespace ssg {

constexpr int kBlock = 256;       // threads per block, every kernel
constexpr int kSpmvWarps = 8;               // warps per SpMV block
constexpr int kSpmvThreads = 32 * kSpmvWarps;
constexpr int kSliceRows = 32;              // rows (or interface copy rows) per slice: one per lane
constexpr int kSliceMaxWidth = 64;          // longer rows are handled one per warp from the CSR arrays
constexpr int kGroupMaxCopies = 8;          // interface nodes with more copies are handled one per warp
// [spmv-source-begin] traits of the single-vector SpMV
template <typename T>
struct SpmvTraits;  // resident blocks per SM; slices ahead prefetched into L2
template <>
struct SpmvTraits<double> {
    static constexpr int kBlocksPerSM = 4;  // measured: 4 blocks without prefetch beat 3 with it
    static constexpr int kL2Ahead = 0;      // slices ahead whose lines are prefetched into L2 (0: none);
                                            // measured: 1 ahead 45.1 us, none 43.9 (the FP64 pipe is busy)
};
template <>
struct SpmvTraits<float> {
    static constexpr int kBlocksPerSM = 5;  // measured: 32.0 us vs 32.8 (4 blocks, with or without prefetch)
    static constexpr int kL2Ahead = 1;      // measured on the 128^3 system: 28.9 us (0: 31.8, 2: 29.9, 4: 31.7)
};
// [spmv-source-end]
constexpr int kVecBlocksPerSM = 4;
constexpr int kHostChunk = 32;    // iterations per host-loop chunk (SSG_DRIVER_HOST)

// Scalar state of one CG solve, resident on the device.
struct Scal {
    double rho;      // (r_k, z_k)_w (z = M^-1 r; z = r without a preconditioner)
    double rr;       // (r_k, r_k)_w: the stopping test
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
    // iterative refinement (SSG_MIXED): outer state uses iter as the
    // refinement count and total for the inner iterations summed; the inner
    // state stops at sqrt(rho) <= tau * sqrt(rho0)
    double rho0;
    double tau;
    double inner_rtol;
    int32_t total;
    int32_t max_outer;
    float alpha32;   // alpha and beta rounded to FP32 once (FP32 kernels read these:
    float beta32;    // a double-to-float conversion per thread costs FP64 pipe time)
    // Hand-offs inside an iteration.  No kernel reads a field that another
    // block of the same kernel writes: the residual update (block 0) copies
    // rho, iter and total into the *_b fields the direction update reads, and
    // the direction update (block 0) writes the new rho/iter/total and raises
    // halt[(k+1) & 1], while every kernel of iteration k reads halt[k & 1].
    double rho_b;
    int32_t iter_b;
    int32_t total_b;
    int32_t halt[2];
    int32_t brk;     // (S p, p) <= 0 seen: every later kernel returns at once
    int32_t passes;  // launches of the residual update (one per iteration copy the loop ran)
};

enum { kTicketSpmv = 0, kTicketR = 1, kTicketXP = 2, kTicketMisc = 3 };

// One unit of SpMV work (precomputed on the host, 32 bytes).
//   kind 0: slice of interior rows [a, b) (b - a <= 32), sliced-ELL data at
//           e0, width e1 (entries [e0 + k*32, e0 + k*32 + 32) are the k-th
//           nonzeros of the slice's rows, padded with zero values)
//   kind 1: slice of interface copy rows [a, b) in (node, copy) order, whole
//           nodes only, sliced-ELL data at e0, width e1
//   kind 2: one interior row a longer than kSliceMaxWidth, CSR nonzeros [e0, e1)
//   kind 3: one interface node a, copies [c0, c1), whose copy rows are too
//           long (in the list of kind-5 groups also: more than
//           kGroupMaxCopies copies)
//   kind 4: slice of interior rows taken from a window of one subdomain's
//           rows sorted by length (SELL-C-sigma): lane l holds row srow[a + l]
//           for a + l < b; sliced-ELL data at e0, width e1, as kind 0
//   kind 5: group of b <= 32 interface nodes of one multiplicity m = c0 <=
//           kGroupMaxCopies, one node per lane: the group's sliced-ELL data
//           at e0 of gval / gcol holds m sub-slices, the r-th with the lanes' r-th copy rows
//           (ascending subdomain) at width group_width(W, r) (8 bits each,
//           ranks 0-3 in c1, 4-7 in pad), e1 = their total width; lane l's
//           r-th copy is the local row gcopy[a + 32 r + l]
// A system carries its interface copy rows in both forms: kind 1 in the
// item list of every product, kind 5 in a second list that the FP64
// single-vector product takes when the groups store enough fewer padding
// entries (api.cu, make_plan).
struct WorkItem {
    int32_t kind, a, b, e0, e1, c0, c1, pad;
};

enum {
    kItemSlice = 0,
    kItemIfaceSlice = 1,
    kItemLongRow = 2,
    kItemLongIface = 3,
    kItemSortedSlice = 4,
    kItemIfaceGroup = 5
};

// Items streamed as sliced ELL (one row per lane); interface groups (kind
// 5, one node per lane) are sliced too, but only the single-vector product
// reads them and tests for them first.
__host__ __device__ __forceinline__ bool sliced_item(int kind) {
    return kind == kItemSlice || kind == kItemIfaceSlice || kind == kItemSortedSlice;
}

// Matrix-side arrays on the device (one arena, see api.cu).
struct DevOp {
    const int32_t *rowptr;  // [nloc+1] concatenated local CSR row pointers
    const int32_t *col;     // [nnz] concatenated column index (subdomain offset + local column)
    const double *val;      // [nnz]
    const float *val32;     // [nnz] values rounded to FP32 (mixed mode)
    const int32_t *irp;     // [ncopies+1] row pointers of the interface copy rows, (node, copy) order
    const int32_t *icol;    // copy-row columns (concatenated local index)
    const double *ival;     // copy-row values
    const float *ival32;    // copy-row values rounded to FP32
    const int32_t *iptr;    // [ngamma+1] copies of each interface node
    const int32_t *icopy;   // [ncopies] concatenated local index of each copy
    const double *sval;     // sliced-ELL values: slice k-th entries of its 32 rows contiguous
    const float *sval32;    // the same rounded to FP32
    const int32_t *scol;    // sliced-ELL columns (concatenated local index)
    const int32_t *sseg;    // interface slices, per copy: (lane of the node's first copy) | (m << 8)
    const int32_t *gcopy;   // interface groups: per group and copy rank, the 32 lanes' copy rows
    const double *gval;     // interface groups' sliced-ELL values (sub-slice layout as sval)
    const float *gval32;    // the same rounded to FP32
    const int32_t *gcol;    // their columns (concatenated local index)
    const int32_t *srow;    // sorted slices: the local row of each slot
    const WorkItem *items;  // SpMV work list
    const int2 *warp_range;  // [grid * kSpmvWarps] contiguous item range of each warp
    const uint8_t *mult;    // [nloc] weight code of each local entry: its node's multiplicity m (w = wtab[m] = 1/m),
                            // or with the owner mask 1 on owner copies and interior entries, 0 on other copies
    const uint8_t *wsel;    // owner mask: the same codes, read by the product's interface dot; null: w = 1/m of the
                            // node's copy count
    const double *wtab;     // [256] wtab[m] = 1/m
    const float *wtab32;    // [256] 1/m rounded to FP32
    const uint8_t *gflag;   // [ceil(nloc / 64)] 1 if entries [64 g, 64 g + 64) hold an interface copy
    const uint8_t *gflag128;  // [ceil(nloc / 128)] the same for groups of 128 entries
    int32_t l2_ahead;       // K-vector product: slices ahead whose lines are prefetched into L2 (0: none)
};

// kEpiStore: the (x, y)_w total is written to *out by the last block (ticket);
// kEpiPartials: each block only writes its partial, the next kernel sums them.
enum { kEpiStore = 0, kEpiPartials = 1 };

// Width of copy rank r's sub-slice in an interface group (kind 5).
__host__ __device__ __forceinline__ int group_width(const WorkItem &W, int r) {
    return static_cast<int>((static_cast<uint32_t>(r < 4 ? W.c1 : W.pad) >> (8 * (r & 3))) & 0xffu);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order block sum over NT threads, adds done by warp 0 only; result
// valid in thread 0.
template <int NT = kBlock>
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[NT];
    __syncthreads();  // protects red[] against a previous call
    red[threadIdx.x] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = red[threadIdx.x];
#pragma unroll
        for (int i = 1; i < NT / 32; ++i) t += red[threadIdx.x + 32 * i];
        t = warp_sum(t);
    }
    return t;
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// FP32 version for the FP32 kernels (one conversion to double per block).
__device__ __forceinline__ float block_sumf(float v) {
    __shared__ float redf[kBlock];
    __syncthreads();
    redf[threadIdx.x] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x < 32) {
        t = redf[threadIdx.x];
#pragma unroll
        for (int i = 1; i < kBlock / 32; ++i) t += redf[threadIdx.x + 32 * i];
        t = warp_sumf(t);
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

template <int NT = kBlock>
__device__ __forceinline__ double sum_partials(const double *partials, int G) {
    __threadfence();
    double v = 0.0;
    for (int i = threadIdx.x; i < G; i += NT) v += __ldcg(partials + i);
    return block_sum<NT>(v);
}

// Every block sums the previous kernel's block partials in the same fixed
// order (the partials are complete and visible at the kernel boundary), so
// all blocks hold the bitwise same total without a ticket or a last block.
__device__ __forceinline__ double all_sum_partials(const double *partials, int G) {
    double v = 0.0;
    for (int i = threadIdx.x; i < G; i += kBlock) v += __ldcg(partials + i);
    const double t = block_sum(v);
    __shared__ double bc;
    if (threadIdx.x == 0) bc = t;
    __syncthreads();
    return bc;
}

// num / den formed once by thread 0 and handed to the block: an FP64 division
// is a sequence of FP64 instructions, and every thread of every block
// dividing on its own kept the FP64 pipe (2 operations per clock per SM)
// busy for microseconds before the stream could start.  With to_f32 the
// quotient is also rounded to FP32 once (*q32).
__device__ __forceinline__ double block_quotient(double num, double den, float *q32 = nullptr) {
    __shared__ double q;
    __shared__ float qf;
    __syncthreads();  // a previous call's readers are done
    if (threadIdx.x == 0) {
        q = num / den;
        qf = float(q);
    }
    __syncthreads();
    if (q32) *q32 = qf;
    return q;
}

// Streams i = i0, i0 + step, ... < i1 through load(i) and apply(i, loaded),
// U indices at a time: the U loads are issued before the first apply, so a
// thread keeps U requests in flight instead of one, and the applies still run
// in ascending i (per-thread sums keep their order and bits).
template <int U, typename L, typename A>
__device__ __forceinline__ void stream_loop(int64_t i0, int64_t i1, int64_t step, L load, A apply) {
    using R = decltype(load(i0));
    int64_t i = i0;
    for (; i + (U - 1) * step < i1; i += U * step) {
        R v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = load(i + u * step);
#pragma unroll
        for (int u = 0; u < U; ++u) apply(i + u * step, v[u]);
    }
    for (; i < i1; i += step) apply(i, load(i));
}

// stream_loop whose first PRE loads are issued before prologue() runs: the
// prologue (summing the previous kernel's block partials, forming alpha or
// beta) then overlaps those loads instead of stalling the stream.  The
// applies run in the same ascending order as stream_loop's.  prologue() is
// called by every thread (it may hold barriers); when it returns false
// nothing is applied and false is returned.
template <int U, int PRE = (U < 2 ? U : 2), typename L, typename P, typename A>
__device__ __forceinline__ bool stream_loop_after(int64_t i0, int64_t i1, int64_t step, L load, P prologue, A apply) {
    constexpr int kPre = PRE;
    using R = decltype(load(i0));
    R v[kPre];
#pragma unroll
    for (int u = 0; u < kPre; ++u)
        if (i0 + u * step < i1) v[u] = load(i0 + u * step);
    if (!prologue()) return false;
#pragma unroll
    for (int u = 0; u < kPre; ++u)
        if (i0 + u * step < i1) apply(i0 + u * step, v[u]);
    stream_loop<U>(i0 + kPre * step, i1, step, load, apply);
    return true;
}

__device__ __forceinline__ void stop_loop(Scal *s, cudaGraphConditionalHandle h, int use_cond) {
    s->done = 1;
    if (use_cond) cudaGraphSetConditional(h, 0);
}

template <typename T>
__device__ __forceinline__ const T *slice_vals(const DevOp &A);
template <>
__device__ __forceinline__ const double *slice_vals<double>(const DevOp &A) { return A.sval; }
template <>
__device__ __forceinline__ const float *slice_vals<float>(const DevOp &A) { return A.sval32; }
template <typename T>
__device__ __forceinline__ const T *group_vals(const DevOp &A);
template <>
__device__ __forceinline__ const double *group_vals<double>(const DevOp &A) { return A.gval; }
template <>
__device__ __forceinline__ const float *group_vals<float>(const DevOp &A) { return A.gval32; }
template <typename T>
__device__ __forceinline__ const T *row_vals(const DevOp &A);
template <>
__device__ __forceinline__ const double *row_vals<double>(const DevOp &A) { return A.val; }
template <>
__device__ __forceinline__ const float *row_vals<float>(const DevOp &A) { return A.val32; }
template <typename T>
__device__ __forceinline__ const T *copy_vals(const DevOp &A);
template <>
__device__ __forceinline__ const double *copy_vals<double>(const DevOp &A) { return A.ival; }
template <>
__device__ __forceinline__ const float *copy_vals<float>(const DevOp &A) { return A.ival32; }

template <typename T>
__device__ __forceinline__ T wtab_of(const DevOp &A, int m);
template <>
__device__ __forceinline__ double wtab_of<double>(const DevOp &A, int m) { return __ldg(A.wtab + m); }
template <>
__device__ __forceinline__ float wtab_of<float>(const DevOp &A, int m) { return __ldg(A.wtab32 + m); }

// [spmv-source-begin] the single-vector SpMV kernel and its helpers
// Weight of interface copy `row` (of a node with m copies) in the product's
// weighted dot: 1/m, or the owner mask's 1 / 0 when the system uses it.
template <typename T>
__device__ __forceinline__ T copy_weight(const DevOp &A, int m, int row) {
    return wtab_of<T>(A, A.wsel ? __ldg(A.wsel + row) : m);
}

// The product's input x_j, gathered by column: through the read-only path,
// x being constant for the whole kernel (every product launch).  The
// one-cluster solve passes its own gather instead (cluster.cuh).
template <typename T>
struct XRead {
    const T *__restrict__ x;
    __device__ __forceinline__ T operator()(int j) const { return __ldg(x + j); }
};

// Matrix loads: streamed with L2 evict-first (every product launch: the
// matrix is read once per launch), or through L1 (STREAM = false: the
// one-cluster solve, whose CTAs read the same slices every iteration).
template <bool STREAM, typename U>
__device__ __forceinline__ U ldm(const U *p) {
    if constexpr (STREAM) return __ldcs(p);
    else return __ldg(p);
}

// N consecutive entries (k0 .. k0+N-1) of a lane's sliced-ELL row: all
// loads first (the value and column loads of a warp are contiguous and
// coalesced, streamed with L2 evict-first), then the FMA chain in order.
template <int N, bool STREAM, typename T, typename XL>
__device__ __forceinline__ T slice_chunk(const T *__restrict__ sv, const int32_t *__restrict__ sc, const XL &X,
                                         int base, int k0, T acc) {
    T vv[N], xv[N];
    int cc[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        vv[j] = ldm<STREAM>(sv + base + (k0 + j) * kSliceRows);
        cc[j] = ldm<STREAM>(sc + base + (k0 + j) * kSliceRows);
    }
#pragma unroll
    for (int j = 0; j < N; ++j) xv[j] = X(cc[j]);
#pragma unroll
    for (int j = 0; j < N; ++j) acc = fma(vv[j], xv[j], acc);
    return acc;
}

// Row product of lane `lane` of a slice (sliced-ELL data at `off`, width w,
// the same for the whole warp): the row's nonzeros in CSR order, then the
// zero-valued padding, which leaves the sum unchanged.  Every lane runs
// exactly w FMAs: on this part a predicated-off FP64 instruction still takes
// its issue slot, so nothing here is predicated.
template <bool STREAM, typename T, typename XL>
__device__ __forceinline__ T slice_row(const T *__restrict__ sv, const int32_t *__restrict__ sc, const XL &X,
                                       int off, int w, int lane) {
    const int base = off + lane;
    T acc = T(0);
    int k = 0;
    for (; k + 8 <= w; k += 8) acc = slice_chunk<8, STREAM>(sv, sc, X, base, k, acc);
    switch (w - k) {
        case 1: return slice_chunk<1, STREAM>(sv, sc, X, base, k, acc);
        case 2: return slice_chunk<2, STREAM>(sv, sc, X, base, k, acc);
        case 3: return slice_chunk<3, STREAM>(sv, sc, X, base, k, acc);
        case 4: return slice_chunk<4, STREAM>(sv, sc, X, base, k, acc);
        case 5: return slice_chunk<5, STREAM>(sv, sc, X, base, k, acc);
        case 6: return slice_chunk<6, STREAM>(sv, sc, X, base, k, acc);
        case 7: return slice_chunk<7, STREAM>(sv, sc, X, base, k, acc);
        default: return acc;
    }
}

// Writes of one slice's results: interior rows, or interface copy rows whose
// node sums are formed by shuffles in ascending subdomain order.
template <typename T, typename XL>
__device__ __forceinline__ void finish_slice(const DevOp &A, const WorkItem &W, T acc, const XL &X,
                                             T *__restrict__ y, int lane, T &dot) {
    if (W.kind == kItemSlice) {
        const int r = W.a + lane;
        if (r < W.b) {
            y[r] = acc;
            dot = fma(X(r), acc, dot);
        }
    } else if (W.kind == kItemSortedSlice) {
        if (W.a + lane < W.b) {
            const int r = __ldg(A.srow + W.a + lane);
            y[r] = acc;
            dot = fma(X(r), acc, dot);
        }
    } else {
        const int c = W.a + lane;
        const bool valid = c < W.b;
        const int seg = valid ? __ldg(A.sseg + c) : 0;
        const int l0 = seg & 0xff, m = seg >> 8;
        const int mmax = __reduce_max_sync(0xffffffffu, m);
        // the sum starts from the first copy, not from 0 (one FP64 add less
        // per slice: a predicated-off add still takes its FP64 issue slot);
        // the same sum in the same order, up to the sign of a zero total
        T S = __shfl_sync(0xffffffffu, acc, l0 & 31);
        for (int t = 1; t < mmax; ++t) {
            const T v = __shfl_sync(0xffffffffu, acc, (l0 + t) & 31);
            if (t < m) S += v;
        }
        if (valid) {
            const int row = __ldg(A.icopy + c);
            y[row] = S;
            dot = fma(copy_weight<T>(A, m, row) * X(row), S, dot);
        }
    }
}

// N consecutive entries (k0 .. k0+N-1) of the lane's rows in an interface
// group (kind 5): loads first, then the FMAs in order, where entry kend
// starts the next copy row: the finished row's product joins the node sum
// S (the first one is S), and the next row's chain starts from 0.  kend is
// the same in every lane (sub-slice boundaries), so the branch is uniform.
template <int N, bool STREAM, typename T, typename XL>
__device__ __forceinline__ void group_chunk(const T *__restrict__ sv, const int32_t *__restrict__ sc, const XL &X,
                                            const WorkItem &W, int base, int k0, int &r, int &kend, T &S, T &acc) {
    T vv[N], xv[N];
    int cc[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        vv[j] = ldm<STREAM>(sv + base + (k0 + j) * kSliceRows);
        cc[j] = ldm<STREAM>(sc + base + (k0 + j) * kSliceRows);
    }
#pragma unroll
    for (int j = 0; j < N; ++j) xv[j] = X(cc[j]);
#pragma unroll
    for (int j = 0; j < N; ++j) {
        while (k0 + j == kend) {
            if (r == 0) S = acc;
            else S += acc;
            acc = T(0);
            kend += group_width(W, ++r);
        }
        acc = fma(vv[j], xv[j], acc);
    }
}

// One interface group (kind 5), Algorithms 4/5 for its nodes: lane l's node
// has its m copy rows in sub-slices 0..m-1 (ascending subdomain); each row's
// product is an FMA chain over its nonzeros in CSR order (then zero-valued
// padding), the products are summed in ascending subdomain order starting
// from the first, and every copy receives the sum: the copy rows of one node
// meet in one lane, with no shuffle and no padding to another rank's width.
// The lane's copies' share of (x, y)_w is added to dot.  GC: entries loaded
// at once (8, or 4 where the node sum and the rank bookkeeping beside eight
// loads would spill: 48 registers a thread).
template <int GC, bool STREAM, typename T, typename XL>
__device__ __forceinline__ void iface_group(const DevOp &A, const WorkItem &W, const XL &X,
                                            T *__restrict__ y, int lane, T &dot) {
    const T *__restrict__ gv = group_vals<T>(A);
    const int base = W.e0 + lane, wsum = W.e1, m = W.c0;
    // the lane's first two copy rows, loaded before the chains so that their
    // latency overlaps them (most interface nodes have two copies)
    const int row0 = __ldg(A.gcopy + W.a + lane);
    const int row1 = m > 1 ? __ldg(A.gcopy + W.a + kSliceRows + lane) : row0;
    int r = 0, kend = group_width(W, 0);
    T S = T(0), acc = T(0);
    int k = 0;
    for (; k + GC <= wsum; k += GC) group_chunk<GC, STREAM>(gv, A.gcol, X, W, base, k, r, kend, S, acc);
    switch (wsum - k) {
        case 1: group_chunk<1, STREAM>(gv, A.gcol, X, W, base, k, r, kend, S, acc); break;
        case 2: group_chunk<2, STREAM>(gv, A.gcol, X, W, base, k, r, kend, S, acc); break;
        case 3: group_chunk<3, STREAM>(gv, A.gcol, X, W, base, k, r, kend, S, acc); break;
        case 4: if constexpr (GC > 4) group_chunk<4, STREAM>(gv, A.gcol, X, W, base, k, r, kend, S, acc); break;
        case 5: if constexpr (GC > 5) group_chunk<5, STREAM>(gv, A.gcol, X, W, base, k, r, kend, S, acc); break;
        case 6: if constexpr (GC > 6) group_chunk<6, STREAM>(gv, A.gcol, X, W, base, k, r, kend, S, acc); break;
        case 7: if constexpr (GC > 7) group_chunk<7, STREAM>(gv, A.gcol, X, W, base, k, r, kend, S, acc); break;
        default: break;
    }
    // the last row (and any empty ones after it)
    for (; r < m; ++r) {
        if (r == 0) S = acc;
        else S += acc;
        acc = T(0);
    }
    if (lane < W.b) {
        const T x0 = X(row0), w0 = copy_weight<T>(A, m, row0);
        T x1 = T(0), w1 = T(0);
        if (m > 1) {
            x1 = X(row1);
            w1 = copy_weight<T>(A, m, row1);
        }
        y[row0] = S;
        dot = fma(w0 * x0, S, dot);
        if (m > 1) {
            y[row1] = S;
            dot = fma(w1 * x1, S, dot);
        }
        for (int c = 2; c < m; ++c) {
            const int row = __ldg(A.gcopy + W.a + c * kSliceRows + lane);
            y[row] = S;
            dot = fma(copy_weight<T>(A, m, row) * X(row), S, dot);
        }
    }
}

// The work items [range.x, range.y) of one warp: y = S x on their rows, the
// interface sums, and the lane's share of (x, y)_w returned; x_j = X(j).
// AHEAD: slices ahead whose value and column lines are prefetched into L2
// (0: none); STREAM: how the slices are loaded (ldm); GROUPS: whether the
// list may hold interface groups (kind 5), GC their entries loaded at once
// (iface_group).
template <typename T, int AHEAD, bool STREAM = true, bool GROUPS = false, int GC = 8, typename XL>
__device__ __forceinline__ T spmv_items(const DevOp &A, int2 range, const XL &X, T *__restrict__ y, int lane) {
    const T *__restrict__ sv = slice_vals<T>(A);
    const T *__restrict__ val = row_vals<T>(A);
    const T *__restrict__ ival = copy_vals<T>(A);
    T dot = T(0);

    for (int it = range.x; it < range.y; ++it) {
        const WorkItem W = A.items[it];
        if (AHEAD > 0 && it + AHEAD < range.y) {
            // the value and column lines of a slice further ahead, one line per lane
            const WorkItem Wp = A.items[it + AHEAD];
            if (sliced_item(Wp.kind) && lane < Wp.e1) {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(sv + Wp.e0 + lane * kSliceRows));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(A.scol + Wp.e0 + lane * kSliceRows));
            } else if (GROUPS && Wp.kind == kItemIfaceGroup && lane < Wp.e1) {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(group_vals<T>(A) + Wp.e0 + lane * kSliceRows));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(A.gcol + Wp.e0 + lane * kSliceRows));
            }
        }
        if (GROUPS && W.kind == kItemIfaceGroup) {
            iface_group<GC, STREAM, T>(A, W, X, y, lane, dot);
        } else if (sliced_item(W.kind)) {
            const T acc = slice_row<STREAM, T>(sv, A.scol, X, W.e0, W.e1, lane);
            finish_slice<T>(A, W, acc, X, y, lane, dot);
        } else if (W.kind == kItemLongRow) {
            // one long row: lane-strided partial sums, fixed warp tree
            T acc = T(0);
            for (int k = W.e0 + lane; k < W.e1; k += 32) acc = fma(val[k], X(A.col[k]), acc);
            const T racc = T(warp_sum(double(acc)));
            if (lane == 0) {
                y[W.a] = racc;
                dot = fma(X(W.a), racc, dot);
            }
        } else {
            // one interface node with long copy rows: each copy row reduced by
            // the warp (fixed tree), copies summed in ascending s
            T S = T(0);
            for (int c = W.c0; c < W.c1; ++c) {
                T acc = T(0);
                for (int k = A.irp[c] + lane; k < A.irp[c + 1]; k += 32)
                    acc = fma(ival[k], X(A.icol[k]), acc);
                S += T(warp_sum(double(acc)));  // valid in lane 0
            }
            if (lane == 0) {
                for (int c = W.c0; c < W.c1; ++c) {
                    const int row = A.icopy[c];
                    y[row] = S;
                    dot = fma(copy_weight<T>(A, W.c1 - W.c0, row) * X(row), S, dot);
                }
            }
        }
    }
    return dot;
}

// BPS: resident blocks per SM the launch is built for (the grid and the
// register budget); AHEAD: slices ahead whose value and column lines are
// prefetched into L2 (0: none).  The defaults are the measured best on the
// 128^3 system; ssg_autotune times the other instances on a given system.
// GROUPS: the work list holds interface groups (kind 5) instead of slices.
template <int EPI, typename T, int BPS = SpmvTraits<T>::kBlocksPerSM, int AHEAD = SpmvTraits<T>::kL2Ahead,
          bool GROUPS = false>
__global__ void __launch_bounds__(kSpmvThreads, BPS)
    k_spmv_asm(DevOp A, const T *__restrict__ x, T *__restrict__ y, double *partials, Scal *s, double *out,
               cudaGraphConditionalHandle h, int use_cond) {
    if (EPI == kEpiPartials && (s->brk || s->halt[s->iter & 1])) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int2 range = A.warp_range[blockIdx.x * kSpmvWarps + warp];
    // GROUPS: the list holds interface groups (FP64 instances of systems
    // that use them; the group path, merely compiled in, slowed the slices:
    // FP32 8 % on 128^3, the FP64 loop of the 64^2 Poisson system 4 %)
    static_assert(!GROUPS || sizeof(T) == 8, "interface groups are read by the FP64 product only");
    constexpr int GC = BPS >= 5 ? 4 : 8;
    const T dot = spmv_items<T, AHEAD, true, GROUPS, GC>(A, range, XRead<T>{x}, y, lane);
    // fixed-order reduction.  FP32: lanes of each warp in FP32, then the
    // block's warps in order in FP64.  FP64: through shared memory, one warp
    // adding the block's 256 values (12 FP64 warp instructions per block
    // instead of 47 for a shuffle tree in every warp: each takes 16 cycles of
    // the SM's FP64 pipe, which the products keep busy; 41.5 -> 40.8 us on
    // the 128^3 system)
    double bs = 0.0;
    if constexpr (sizeof(T) == 4) {
        __shared__ double wsum[kSpmvWarps];
        const double wv = double(warp_sumf(dot));
        if (lane == 0) wsum[warp] = wv;
        __syncthreads();
        if (threadIdx.x == 0) {
            bs = wsum[0];
#pragma unroll
            for (int w = 1; w < kSpmvWarps; ++w) bs += wsum[w];
        }
    } else {
        bs = block_sum<kSpmvThreads>(double(dot));
    }
    if (EPI == kEpiPartials) {
        if (threadIdx.x == 0) partials[blockIdx.x] = bs;
        return;
    }
    if (publish_and_check_last(partials, bs, &s->ticket[kTicketSpmv])) {
        const double tot = sum_partials<kSpmvThreads>(partials, gridDim.x);
        if (threadIdx.x == 0) {
            s->ticket[kTicketSpmv] = 0;
            if (out) *out = tot;
        }
    }
}

// [spmv-source-end]

__device__ __forceinline__ double wsq(double r, unsigned int m, const double *__restrict__ wtab, double acc) {
    return m == 1u ? fma(r, r, acc) : fma(__ldg(wtab + m) * r, r, acc);
}

// Algorithm 3 lines 3 and 5: every block sums the SpMV's partials of
// (p, S p)_w, forms alpha = rho / (p, S p)_w (or stops on a breakdown), then
// r <- r - alpha q and its share of (r, r)_w.  With the diagonal
// preconditioner (PC, dinv = 1 / diag(S) per local entry) the block also
// forms its share of (r, z)_w, z = dinv r, into part_rz.
template <bool PC>
__global__ void __launch_bounds__(kBlock, kVecBlocksPerSM) k_update_r(int64_t N, double *__restrict__ r, const double *__restrict__ q,
                                                     const uint8_t *__restrict__ mult, const double *__restrict__ wtab,
                                                     const uint8_t *__restrict__ gflag, const double *part_pq,
                                                     int G1, double *part_rr, Scal *s, cudaGraphConditionalHandle h,
                                                     int use_cond, const double *__restrict__ dinv,
                                                     double *part_rz) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s->rho_b = s->rho;
        s->iter_b = s->iter;
        s->passes += 1;
    }
    if (s->brk || s->halt[s->iter & 1]) return;
    double pq = 0.0, alpha = 0.0;
    double acc = 0.0, acz = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    const int64_t N2 = N >> 1;
    double2 *__restrict__ r2 = reinterpret_cast<double2 *>(r);
    const double2 *__restrict__ q2 = reinterpret_cast<const double2 *>(q);
    const uchar2 *__restrict__ m2 = reinterpret_cast<const uchar2 *>(mult);
    const double2 *__restrict__ d2 = reinterpret_cast<const double2 *>(dinv);
    struct Ld {
        double2 r, q, d;
        uint8_t g;
    };
    const bool go = stream_loop_after<PC ? 2 : 4>(
        (int64_t)blockIdx.x * kBlock + threadIdx.x, N2, stride,
        [&](int64_t i) {
            Ld l;
            l.r = r2[i];
            l.q = __ldcs(q2 + i);
            l.g = __ldg(gflag + (i >> 5));
            if (PC) l.d = __ldg(d2 + i);
            return l;
        },
        [&]() {
            pq = all_sum_partials(part_pq, G1);
            if (!(pq > 0.0) || !isfinite(pq)) {
                if (blockIdx.x == 0 && threadIdx.x == 0) {
                    s->pq = pq;
                    s->status = SSG_E_BREAKDOWN;
                    s->brk = 1;
                    stop_loop(s, h, use_cond);
                }
                return false;
            }
            alpha = block_quotient(s->rho, pq);
            return true;
        },
        [&](int64_t i, Ld l) {
            double2 rv = l.r;
            rv.x = fma(-alpha, l.q.x, rv.x);
            rv.y = fma(-alpha, l.q.y, rv.y);
            r2[i] = rv;
            // a warp covers the 64 entries of group i >> 5; groups without an
            // interface copy have weight 1 everywhere and skip the weight lookup
            // (1.0 * r == r, so both forms give the same bits).  One FMA chain
            // for both cases (measured: 79.8 us per FP64 iteration against
            // 84.3 with the products in the two branches).  The test is a warp
            // vote, so the weight multiplies are skipped by a branch instead of
            // being issued predicated off (77.0 -> 75.5 us per iteration)
            double wx = rv.x, wy = rv.y;
            if (__any_sync(__activemask(), l.g != 0)) {
                const uchar2 mv = m2[i];
                wx = __ldg(wtab + mv.x) * rv.x;
                wy = __ldg(wtab + mv.y) * rv.y;
            }
            acc = fma(wx, rv.x, acc);
            acc = fma(wy, rv.y, acc);
            if (PC) {
                acz = fma(wx, rv.x * l.d.x, acz);
                acz = fma(wy, rv.y * l.d.y, acz);
            }
        });
    if (!go) return;
    if ((N & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        const double ri = fma(-alpha, q[N - 1], r[N - 1]);
        r[N - 1] = ri;
        const double wi = __ldg(wtab + mult[N - 1]) * ri;
        acc = fma(wi, ri, acc);
        if (PC) acz = fma(wi, ri * dinv[N - 1], acz);
    }
    const double bs = block_sum(acc);
    const double bz = PC ? block_sum(acz) : 0.0;
    if (threadIdx.x == 0) {
        part_rr[blockIdx.x] = bs;
        if (PC) part_rz[blockIdx.x] = bz;
        if (blockIdx.x == 0) {
            s->alpha = alpha;
            s->alpha32 = float(alpha);
            s->pq = pq;
        }
    }
}

// Algorithm 3 lines 4, 7, 8: every block sums the partials of (r_{k+1},
// r_{k+1})_w (and of (r_{k+1}, z_{k+1})_w with the diagonal preconditioner),
// forms beta = (r, z)_{k+1} / (r, z)_k, and x <- x + alpha p, p <- z + beta p
// (z = r without a preconditioner, z = dinv r with it); block 0 records the
// iteration and the stopping decision (recursive residual sqrt((r, r)_w) <=
// rtol ||b||, or max_iter reached), applied after this update.
template <bool PC>
__global__ void __launch_bounds__(kBlock, kVecBlocksPerSM) k_update_xp(int64_t N, double *__restrict__ x, double *__restrict__ p,
                                                      const double *__restrict__ r, const double *part_rr, int G2,
                                                      Scal *s, cudaGraphConditionalHandle h, int use_cond,
                                                      const double *__restrict__ dinv, const double *part_rz) {
    const int k = s->iter_b;
    if (s->brk || s->halt[k & 1]) return;
    double rr = 0.0, rz = 0.0, beta = 0.0;
    const double alpha = s->alpha;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    const int64_t N2 = N >> 1;
    double2 *x2 = reinterpret_cast<double2 *>(x);
    double2 *p2 = reinterpret_cast<double2 *>(p);
    const double2 *r2 = reinterpret_cast<const double2 *>(r);
    const double2 *__restrict__ d2 = reinterpret_cast<const double2 *>(dinv);
    struct Ld {
        double2 p, x, z;
    };
    stream_loop_after<PC ? 2 : 4>(
        (int64_t)blockIdx.x * kBlock + threadIdx.x, N2, stride,
        [&](int64_t i) {
            Ld l;
            l.p = p2[i];
            l.x = __ldcs(x2 + i);
            l.z = r2[i];
            if (PC) {
                const double2 dv = __ldg(d2 + i);
                l.z.x *= dv.x;
                l.z.y *= dv.y;
            }
            return l;
        },
        [&]() {
            rr = all_sum_partials(part_rr, G2);
            rz = PC ? all_sum_partials(part_rz, G2) : rr;
            beta = block_quotient(rz, s->rho_b);
            return true;
        },
        [&](int64_t i, Ld l) {
            double2 xv = l.x;
            xv.x = fma(alpha, l.p.x, xv.x);
            xv.y = fma(alpha, l.p.y, xv.y);
            __stcs(x2 + i, xv);
            p2[i] = make_double2(fma(beta, l.p.x, l.z.x), fma(beta, l.p.y, l.z.y));
        });
    if ((N & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        const double pi = p[N - 1];
        x[N - 1] = fma(alpha, pi, x[N - 1]);
        p[N - 1] = fma(beta, pi, PC ? r[N - 1] * dinv[N - 1] : r[N - 1]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s->rho = rz;
        s->rr = rr;
        s->beta = beta;
        s->iter = k + 1;
        s->relres = s->bnorm > 0.0 ? sqrt(rr) / s->bnorm : 0.0;
        int stop = 1;
        if (sqrt(rr) <= s->rtol * s->bnorm) s->status = SSG_OK;
        else if (k + 1 >= s->max_iter) s->status = SSG_E_NOT_CONVERGED;
        else stop = 0;
        if (stop) {
            s->halt[(k + 1) & 1] = 1;
            stop_loop(s, h, use_cond);
        }
    }
}

// Setup of Algorithm 3 line 1: r = b - q (q = S x_1 when a guess is given,
// else r = b), z = r (z = dinv r with the diagonal preconditioner, PC),
// p = z, rho = (r, z)_w, (r, r)_w, bnorm = sqrt((b, b)_w), and the stopping
// test before the first iteration.  Partials: (r, r)_w at [0, G), (b, b)_w
// at [G, 2G), (r, z)_w at [2G, 3G).
template <bool PC>
__global__ void __launch_bounds__(kBlock) k_cg_init(int64_t N, const double *__restrict__ b,
                                                    const double *__restrict__ q, double *__restrict__ r,
                                                    double *__restrict__ p, const uint8_t *__restrict__ mult,
                                                    const double *__restrict__ wtab, double *partials, Scal *s,
                                                    cudaGraphConditionalHandle h, int use_cond,
                                                    const double *__restrict__ dinv) {
    const int guess = s->guess;
    double arr = 0.0, abb = 0.0, arz = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < N; i += stride) {
        const double bi = b[i];
        const double ri = guess ? bi - q[i] : bi;
        const double zi = PC ? ri * dinv[i] : ri;
        r[i] = ri;
        if (p) p[i] = zi;
        const unsigned int m = mult[i];
        arr = wsq(ri, m, wtab, arr);
        abb = wsq(bi, m, wtab, abb);
        if (PC) arz = fma(__ldg(wtab + m) * ri, zi, arz);
    }
    const double srr = block_sum(arr);
    const double sbb = block_sum(abb);
    const double srz = PC ? block_sum(arz) : 0.0;
    if (threadIdx.x == 0) {
        partials[gridDim.x + blockIdx.x] = sbb;
        if (PC) partials[2 * gridDim.x + blockIdx.x] = srz;
    }
    if (publish_and_check_last(partials, srr, &s->ticket[kTicketMisc])) {
        const double rr = sum_partials(partials, gridDim.x);
        const double bb = sum_partials(partials + gridDim.x, gridDim.x);
        const double rz = PC ? sum_partials(partials + 2 * gridDim.x, gridDim.x) : rr;
        if (threadIdx.x == 0) {
            s->ticket[kTicketMisc] = 0;
            s->rho = rz;
            s->rr = rr;
            s->bnorm = sqrt(bb);
            s->iter = 0;
            s->total = 0;
            s->passes = 0;
            s->done = 0;
            s->stop_after_xp = 0;
            s->brk = 0;
            s->halt[1] = 0;
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
            s->halt[0] = stop;
            if (use_cond) cudaGraphSetConditional(h, stop ? 0u : 1u);
        }
    }
}

// dinv[k] = 1 / S_ii for the node i of local entry k (its diagonal entry sits
// at local entry dmap[k] of the concatenated local matrices); a missing or
// non-positive diagonal sets *bad and leaves dinv[k] = 0.
__global__ void __launch_bounds__(kBlock) k_dinv(int64_t N, const int32_t *__restrict__ dmap,
                                                 const double *__restrict__ val, double *__restrict__ dinv,
                                                 float *__restrict__ dinv32, int *bad) {
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < N; i += stride) {
        const int32_t e = dmap[i];
        const double d = e >= 0 ? val[e] : 0.0;
        double v = 0.0;
        if (d > 0.0 && isfinite(d)) v = 1.0 / d;
        else *bad = 1;
        dinv[i] = v;
        dinv32[i] = float(v);
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
        const unsigned int m = mult[i];
        if (DIFF) {
            acc = wsq(u[i] - v[i], m, wtab, acc);
        } else {
            acc = m == 1u ? fma(u[i], v[i], acc) : fma(__ldg(wtab + m) * u[i], v[i], acc);
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

// ===========================================================================
// Mixed precision (SSG_MIXED): FP32 inner CG inside FP64 iterative
// refinement.  Outer state `so` (FP64 residual r64, refinement count in
// so->iter, inner iterations summed in so->total); inner state `si`.
// ===========================================================================

// Inner setup: r32 = (float) r64, p32 = r32, d32 = 0, rho0 = (r32, r32)_w and
// the inner tolerance tau = max(inner_rtol, rtol ||b|| / ||r64||), so the last
// refinement is not solved further than the outer test needs.
template <bool PC>
__global__ void __launch_bounds__(kBlock) k_inner_init(int64_t N, const double *__restrict__ r64,
                                                       float *__restrict__ r32, float *__restrict__ p32,
                                                       float *__restrict__ d32, const uint8_t *__restrict__ mult,
                                                       const float *__restrict__ wtab, double *partials, Scal *si,
                                                       const Scal *so, cudaGraphConditionalHandle h, int use_cond,
                                                       const float *__restrict__ dinv32) {
    float acc = 0.f, acz = 0.f;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < N; i += stride) {
        const float ri = float(r64[i]);
        const float zi = PC ? ri * __ldg(dinv32 + i) : ri;
        r32[i] = ri;
        p32[i] = zi;
        d32[i] = 0.f;
        const unsigned int m = mult[i];
        const float wr = __ldg(wtab + m) * ri;
        acc = fmaf(wr, ri, acc);
        if (PC) acz = fmaf(wr, zi, acz);
    }
    const double bs = double(block_sumf(acc));
    const double bz = PC ? double(block_sumf(acz)) : 0.0;
    if (PC && threadIdx.x == 0) partials[gridDim.x + blockIdx.x] = bz;
    if (publish_and_check_last(partials, bs, &si->ticket[kTicketMisc])) {
        const double tot = sum_partials(partials, gridDim.x);
        const double trz = PC ? sum_partials(partials + gridDim.x, gridDim.x) : tot;
        if (threadIdx.x == 0) {
            si->ticket[kTicketMisc] = 0;
            si->rho = trz;
            si->rr = tot;
            si->rho0 = tot;
            double tau = so->bnorm > 0.0 && so->rho > 0.0 ? so->rtol * so->bnorm / sqrt(so->rho) : 0.0;
            si->tau = tau > so->inner_rtol ? tau : so->inner_rtol;
            si->iter = 0;
            si->alpha = 0.0;
            si->beta = 0.0;
            si->alpha32 = 0.f;
            si->beta32 = 0.f;
            si->status = SSG_OK;
            si->stop_after_xp = 0;
            const int stop = !(tot > 0.0) || so->total >= so->max_iter;
            si->done = stop;
            si->brk = 0;
            si->halt[0] = stop;
            si->halt[1] = 0;
            if (use_cond) cudaGraphSetConditional(h, stop ? 0u : 1u);
        }
    }
}

// Inner Algorithm 3 lines 3 and 5 in FP32: every block sums the FP32 SpMV's
// partials of (p, S p)_w (FP64), forms alpha (or stops on a breakdown), then
// r32 <- r32 - alpha q32 and its share of (r32, r32)_w (products and block
// sums in FP32).  A warp covers the 128 entries of flag group i >> 5 (float4
// per lane); groups without interface copies skip the weights.
// The block's part of it; false when the loop has stopped (every block
// returns at the same point: all read the same state and partials).
template <bool PC>
__device__ __forceinline__ bool update_r32_step(int64_t N, float *__restrict__ r, const float *__restrict__ q,
                                                const uint8_t *__restrict__ mult, const float *__restrict__ wtab,
                                                const uint8_t *__restrict__ gflag128, const double *part_pq, int G1,
                                                double *part_rr, Scal *si, Scal *so,
                                                cudaGraphConditionalHandle h, int use_cond,
                                                const float *__restrict__ dinv32, double *part_rz) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        si->rho_b = si->rho;
        si->iter_b = si->iter;
        si->total_b = so->total;
        so->passes += 1;
    }
    const int k = si->iter;
    if (si->brk || si->halt[k & 1]) return false;
    double pq = 0.0, alpha_d = 0.0;
    float alpha = 0.f;
    float acc = 0.f, acz = 0.f;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    const int64_t N4 = N >> 2;
    float4 *__restrict__ r4 = reinterpret_cast<float4 *>(r);
    const float4 *__restrict__ q4 = reinterpret_cast<const float4 *>(q);
    const uchar4 *__restrict__ m4 = reinterpret_cast<const uchar4 *>(mult);
    const float4 *__restrict__ z4 = reinterpret_cast<const float4 *>(dinv32);
    struct Ld {
        float4 r, q, d;
        uint8_t g;
    };
    // a thread streams about four items on the 128^3 system: all of them
    // are in flight before the prologue
    const bool go = stream_loop_after<PC ? 2 : 4, PC ? 2 : 4>(
        (int64_t)blockIdx.x * kBlock + threadIdx.x, N4, stride,
        [&](int64_t i) {
            Ld l;
            l.r = r4[i];
            l.q = __ldcs(q4 + i);
            l.g = __ldg(gflag128 + (i >> 5));
            if (PC) l.d = __ldg(z4 + i);
            return l;
        },
        [&]() {
            pq = all_sum_partials(part_pq, G1);
            if (!(pq > 0.0) || !isfinite(pq)) {
                if (blockIdx.x == 0 && threadIdx.x == 0) {
                    si->pq = pq;
                    si->status = SSG_E_BREAKDOWN;
                    si->brk = 1;
                    stop_loop(si, h, use_cond);
                }
                return false;
            }
            alpha_d = block_quotient(si->rho, pq, &alpha);
            return true;
        },
        [&](int64_t i, Ld l) {
            float4 rv = l.r;
            rv.x = fmaf(-alpha, l.q.x, rv.x);
            rv.y = fmaf(-alpha, l.q.y, rv.y);
            rv.z = fmaf(-alpha, l.q.z, rv.z);
            rv.w = fmaf(-alpha, l.q.w, rv.w);
            r4[i] = rv;
            float4 w = make_float4(1.f, 1.f, 1.f, 1.f);
            if (l.g != 0) {
                const uchar4 mv = m4[i];
                w = make_float4(__ldg(wtab + mv.x), __ldg(wtab + mv.y), __ldg(wtab + mv.z), __ldg(wtab + mv.w));
            }
            if (l.g == 0) {
                acc = fmaf(rv.x, rv.x, acc);
                acc = fmaf(rv.y, rv.y, acc);
                acc = fmaf(rv.z, rv.z, acc);
                acc = fmaf(rv.w, rv.w, acc);
            } else {
                acc = fmaf(w.x * rv.x, rv.x, acc);
                acc = fmaf(w.y * rv.y, rv.y, acc);
                acc = fmaf(w.z * rv.z, rv.z, acc);
                acc = fmaf(w.w * rv.w, rv.w, acc);
            }
            if (PC) {
                acz = fmaf(w.x * rv.x, rv.x * l.d.x, acz);
                acz = fmaf(w.y * rv.y, rv.y * l.d.y, acz);
                acz = fmaf(w.z * rv.z, rv.z * l.d.z, acz);
                acz = fmaf(w.w * rv.w, rv.w * l.d.w, acz);
            }
        });
    if (!go) return false;
    if (blockIdx.x == 0 && threadIdx.x < (N & 3)) {
        const int64_t i = (N & ~int64_t(3)) + threadIdx.x;
        const float ri = fmaf(-alpha, q[i], r[i]);
        r[i] = ri;
        const float wi = __ldg(wtab + mult[i]) * ri;
        acc = fmaf(wi, ri, acc);
        if (PC) acz = fmaf(wi, ri * dinv32[i], acz);
    }
    const double bs = double(block_sumf(acc));
    const double bz = PC ? double(block_sumf(acz)) : 0.0;
    if (threadIdx.x == 0) {
        part_rr[blockIdx.x] = bs;
        if (PC) part_rz[blockIdx.x] = bz;
        if (blockIdx.x == 0) {
            si->alpha = alpha_d;
            si->alpha32 = alpha;
            si->pq = pq;
        }
    }
    return true;
}

template <bool PC>
__global__ void __launch_bounds__(kBlock, kVecBlocksPerSM) k_update_r32(int64_t N, float *__restrict__ r, const float *__restrict__ q,
                                                       const uint8_t *__restrict__ mult, const float *__restrict__ wtab,
                                                       const uint8_t *__restrict__ gflag128, const double *part_pq, int G1,
                                                       double *part_rr, Scal *si, Scal *so,
                                                       cudaGraphConditionalHandle h, int use_cond,
                                                       const float *__restrict__ dinv32, double *part_rz) {
    update_r32_step<PC>(N, r, q, mult, wtab, gflag128, part_pq, G1, part_rr, si, so, h, use_cond, dinv32, part_rz);
}

// Inner Algorithm 3 lines 4, 7, 8 in FP32: every block sums the partials of
// (r32, r32)_w, forms beta, and d32 <- d32 + alpha p32, p32 <- r32 + beta p32;
// block 0 records the iteration and the inner stopping decision
// (sqrt((r, r)_w) <= tau sqrt(rho0), or the inner iterations summed over
// refinements reach max_iter).
// The block's part of it for iteration k, with alpha (FP32), the summed
// inner iteration count and rho_k handed in by the caller.
template <bool PC>
__device__ __forceinline__ void update_dp32_step(int64_t N, float *__restrict__ d, float *__restrict__ p,
                                                 const float *__restrict__ r, const double *part_rr, int G2,
                                                 Scal *si, Scal *so, cudaGraphConditionalHandle h, int use_cond,
                                                 const float *__restrict__ dinv32, const double *part_rz, int k, float alpha, int total1,
                                                 double rho_b) {
    double rr = 0.0, rz = 0.0, beta_d = 0.0;
    float beta = 0.f;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    const int64_t N4 = N >> 2;
    float4 *__restrict__ d4 = reinterpret_cast<float4 *>(d);
    float4 *__restrict__ p4 = reinterpret_cast<float4 *>(p);
    const float4 *__restrict__ r4 = reinterpret_cast<const float4 *>(r);
    const float4 *__restrict__ z4 = reinterpret_cast<const float4 *>(dinv32);
    struct Ld {
        float4 p, d, z;
    };
    stream_loop_after<2>(
        (int64_t)blockIdx.x * kBlock + threadIdx.x, N4, stride,
        [&](int64_t i) {
            Ld l;
            l.p = p4[i];
            l.d = d4[i];
            l.z = r4[i];
            if (PC) {
                const float4 dv = __ldg(z4 + i);
                l.z.x *= dv.x;
                l.z.y *= dv.y;
                l.z.z *= dv.z;
                l.z.w *= dv.w;
            }
            return l;
        },
        [&]() {
            rr = all_sum_partials(part_rr, G2);
            rz = PC ? all_sum_partials(part_rz, G2) : rr;
            beta_d = block_quotient(rz, rho_b, &beta);
            return true;
        },
        [&](int64_t i, Ld l) {
            float4 dv = l.d;
            const float4 pv = l.p, zv = l.z;
            dv.x = fmaf(alpha, pv.x, dv.x);
            dv.y = fmaf(alpha, pv.y, dv.y);
            dv.z = fmaf(alpha, pv.z, dv.z);
            dv.w = fmaf(alpha, pv.w, dv.w);
            d4[i] = dv;
            p4[i] = make_float4(fmaf(beta, pv.x, zv.x), fmaf(beta, pv.y, zv.y), fmaf(beta, pv.z, zv.z),
                                fmaf(beta, pv.w, zv.w));
        });
    if (blockIdx.x == 0 && threadIdx.x < (N & 3)) {
        const int64_t i = (N & ~int64_t(3)) + threadIdx.x;
        const float pi = p[i];
        d[i] = fmaf(alpha, pi, d[i]);
        p[i] = fmaf(beta, pi, PC ? r[i] * dinv32[i] : r[i]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        si->rho = rz;
        si->rr = rr;
        si->beta = beta_d;
        si->beta32 = beta;
        si->iter = k + 1;
        so->total = total1;
        if (sqrt(rr) <= si->tau * sqrt(si->rho0) || total1 >= so->max_iter) {
            si->halt[(k + 1) & 1] = 1;
            stop_loop(si, h, use_cond);
        }
    }
}

template <bool PC>
__global__ void __launch_bounds__(kBlock, kVecBlocksPerSM) k_update_dp32(int64_t N, float *__restrict__ d, float *__restrict__ p,
                                                        const float *__restrict__ r, const double *part_rr, int G2,
                                                        Scal *si, Scal *so, cudaGraphConditionalHandle h, int use_cond,
                                                        const float *__restrict__ dinv32, const double *part_rz) {
    const int k = si->iter_b;
    if (si->brk || si->halt[k & 1]) return;
    update_dp32_step<PC>(N, d, p, r, part_rr, G2, si, so, h, use_cond, dinv32, part_rz, k, si->alpha32,
                         si->total_b + 1, si->rho_b);
}

// x64 <- x64 + (double) d32 (the refinement update).
__global__ void __launch_bounds__(kBlock) k_ir_correct(int64_t N, double *__restrict__ x, const float *__restrict__ d) {
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < N; i += stride) x[i] += double(d[i]);
}

// r64 = b - q64 (q64 = S x64 from the FP64 SpMV), (r64, r64)_w, and the outer
// decision: converged, inner breakdown, refinement or iteration cap.
__global__ void __launch_bounds__(kBlock) k_ir_residual(int64_t N, const double *__restrict__ b,
                                                        const double *__restrict__ q, double *__restrict__ r,
                                                        const uint8_t *__restrict__ mult,
                                                        const double *__restrict__ wtab, double *partials, Scal *so,
                                                        const Scal *si, cudaGraphConditionalHandle h, int use_cond) {
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < N; i += stride) {
        const double ri = b[i] - q[i];
        r[i] = ri;
        acc = wsq(ri, mult[i], wtab, acc);
    }
    const double bs = block_sum(acc);
    if (publish_and_check_last(partials, bs, &so->ticket[kTicketMisc])) {
        const double tot = sum_partials(partials, gridDim.x);
        if (threadIdx.x == 0) {
            so->ticket[kTicketMisc] = 0;
            so->rho = tot;
            so->iter += 1;
            so->relres = so->bnorm > 0.0 ? sqrt(tot) / so->bnorm : 0.0;
            int stop = 1;
            if (si->status == SSG_E_TIMEOUT) {
                so->status = SSG_E_TIMEOUT;  // the inner iterate is not to be trusted
            } else if (sqrt(tot) <= so->rtol * so->bnorm) {
                so->status = SSG_OK;
            } else if (si->status == SSG_E_BREAKDOWN) {
                so->status = SSG_E_BREAKDOWN;
            } else if (so->iter >= so->max_outer || so->total >= so->max_iter) {
                so->status = SSG_E_NOT_CONVERGED;
            } else {
                stop = 0;
            }
            so->done = stop;
            if (use_cond) cudaGraphSetConditional(h, stop ? 0u : 1u);
        }
    }
}

__global__ void k_set_mixed(Scal *s, double inner_rtol, int32_t max_outer) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        s->inner_rtol = inner_rtol;
        s->max_outer = max_outer;
    }
}

}  // namespace ssg
