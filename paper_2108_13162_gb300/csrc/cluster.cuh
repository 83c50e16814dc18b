// A small system solved by one thread-block cluster: Algorithm 3 (M = I, or
// the diagonal preconditioner) with all its iterations inside one kernel.
//
// On a system whose vectors and matrix sit in L2 (tens of thousands of
// local entries) an iteration of the three-kernel loop costs the latency of
// three kernel boundaries, not bandwidth.  Here the CTAs of one cluster (up
// to 16, one per SM) run the iteration with two cluster barriers instead:
// the product's work items are split among the cluster's warps (the same
// items, rows in the same order and interface copies summed in the same
// order as the multi-block product), each CTA sums its share of a dot in a
// fixed order and publishes it in its shared memory, and after the barrier
// warp 0 of every CTA reads the CTAs' sums through distributed shared memory
// and adds them in the same fixed order — so every CTA holds bitwise the same
// totals, forms the same scalars and takes the same branches, and no CTA
// leaves the loop alone.
#pragma once

#include <cooperative_groups.h>

#include "kernels.cuh"

namespace ssg {

constexpr int kClusterThreads = 1024;  // threads per CTA
constexpr int kClusterWarps = kClusterThreads / 32;
constexpr int kClusterMaxCtas = 16;

// The scalars of the iteration, formed by thread 0 of each CTA from the
// cluster-wide sums (the same bits in every CTA) and read by its threads
// after the next block barrier.
struct ClusterScal {
    double rho, rr, pq, alpha, beta, bnorm;
    int status, k, run;
};

// Sum over the first 16 lanes of a warp (the CTAs of a cluster), by the
// fixed tree of offsets 8, 4, 2, 1; valid in lane 0.
__device__ __forceinline__ double warp_sum16(double v) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Cluster-wide sums of NV <= 3 values per thread, in every CTA; thread 0 then
// runs fin(tot) with the NV totals (red: the CTA's [3][kClusterThreads]
// staging buffer).  Each CTA adds its warps [0, wact) (the others hold no
// entry) lane by lane, warp w into chain w mod 4, the four chains then
// pairwise, then the 32 lanes by the fixed shuffle tree, into slot[phase &
// 1] of its shared memory.  (On this part a dependent FP64 add costs about
// 80 cycles: the four chains cut the critical path of 32 warps from 31 adds
// to 9.)  The cluster barrier (release / acquire at cluster scope: it also
// publishes the phase's global-memory writes to the other CTAs), then lane r
// of warp 0 reads CTA r's sums through distributed shared memory and the 16
// lanes are added by a fixed tree.  The slots alternate: a CTA writes a slot
// again only after the next cluster barrier, which no CTA passes before every
// CTA has read this phase's sums.  Ends with a block barrier (fin's results
// visible).
template <int NV, typename F>
__device__ __forceinline__ void cluster_sums(cooperative_groups::cluster_group &cl, double (*red)[kClusterThreads],
                                             double (*slot)[4], int phase, int wact, const double (&v)[NV], F fin) {
    double *mine = slot[phase & 1];
#pragma unroll
    for (int j = 0; j < NV; ++j) red[j][threadIdx.x] = v[j];
    __syncthreads();
    if (threadIdx.x < 32) {
        const int l = threadIdx.x;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            double a[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) a[c] = c < wact ? red[j][l + 32 * c] : 0.0;
            for (int w = 4; w < wact; w += 4) {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (w + c < wact) a[c] += red[j][l + 32 * (w + c)];
            }
            const double t = warp_sum((a[0] + a[1]) + (a[2] + a[3]));
            if (l == 0) mine[j] = t;
        }
    }
    cl.sync();
    if (threadIdx.x < 32) {
        const unsigned int n = cl.num_blocks();
        const unsigned int lane = threadIdx.x;
        double tot[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            double t = 0.0;
            if (lane < n) t = cl.map_shared_rank(mine, lane)[j];
            tot[j] = warp_sum16(t);
        }
        if (lane == 0) fin(tot);
    }
    __syncthreads();
}

// The stopping test of Algorithm 3 as the loop takes it, sqrt(rr) <= t,
// without the square root (a chain of dependent FP64 operations) when rr is
// clearly on one side of t^2: lo and hi bracket t^2 by a relative 2^-48,
// far beyond the rounding of t^2 and of the square root, so outside
// [lo, hi] the answer is that of the correctly rounded square root; inside,
// and whenever t^2 is not a normal number, the square root decides.
struct StopTest {
    double t, lo, hi;
    bool bracket;
    __device__ __forceinline__ void init(double t_) {
        t = t_;
        const double T = t_ * t_;
        bracket = isfinite(T) && T >= 0x1p-1000;
        lo = T * (1.0 - 0x1p-48);
        hi = T * (1.0 + 0x1p-48);
    }
    __device__ __forceinline__ bool operator()(double rr) const {
        if (bracket) {
            if (rr <= lo) return true;
            if (rr > hi) return false;
        }
        return sqrt(rr) <= t;
    }
};

// The direction the product gathers in iteration k, formed where it is
// read: p_k[j] = z_k[j] + beta_{k-1} p_{k-1}[j] (Algorithm 3 line 8, z = r,
// or dinv r with the diagonal preconditioner), the same FMA on the same
// operands as the update that stores p_k, so the same bits.  r and p are
// rewritten by other CTAs between products and are read through L2.
template <bool PC>
struct PNext {
    const double *r, *p, *dinv;
    double beta;
    __device__ __forceinline__ double operator()(int j) const {
        const double rj = __ldcg(r + j);
        return fma(beta, __ldcg(p + j), PC ? rj * __ldg(dinv + j) : rj);
    }
};

// One solve of S x = b on the concatenated local vectors.  The caller has
// scattered b into b, x holds x_1 (zero, or the scattered guess) and, with a
// guess, q = S x_1.  Launched as one cluster of gridDim.x CTAs.  Product
// items: warp w of CTA c takes A.warp_range[w * gridDim.x + c] (ranges cut
// for the whole cluster, dealt out to the CTAs in turn); the non-empty
// ranges are the first `nranges`.  Vector entries: CTA c takes a contiguous
// run of whole warps' worth.
//
// Iteration k: q = S p_k with p_k formed as the product gathers it (PNext),
// then one cluster-wide sum gives alpha_k; each CTA stores p_k on its
// entries (the product's gathers of p_{k-1} are over: they precede that
// sum), x <- x + alpha_k p_k, r <- r - alpha_k q, and a second cluster-wide
// sum gives (r, r)_w (and (r, z)_w), beta_k and the stopping test.  Two
// cluster barriers per iteration; the operations and their operands are
// those of the three-kernel loop, in its order for every entry.  The setup,
// the stopping rule (recursive residual sqrt((r, r)_w) <= rtol ||b||_w after
// an iteration, or max_iter), the breakdown test and the state written to s
// at the end are the loop's; p is left holding the last p_k, not p_{k+1}.
template <bool PC>
__global__ void __launch_bounds__(kClusterThreads, 1)
    k_cg_cluster(DevOp A, int64_t N, int nranges, const double *__restrict__ b, double *__restrict__ x,
                 double *r, double *p, double *q, const double *__restrict__ dinv, Scal *s) {
    namespace cgr = cooperative_groups;
    constexpr int NZ = PC ? 2 : 1;  // sums after the residual update: (r, r)_w [, (r, z)_w]
    cgr::cluster_group cl = cgr::this_cluster();
    __shared__ double red[3][kClusterThreads];
    __shared__ double slot[2][4];
    __shared__ ClusterScal cs;
    __shared__ StopTest stop;  // read by thread 0 only
    const int nc = static_cast<int>(cl.num_blocks());
    const int rank = static_cast<int>(cl.block_rank());
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int2 range = A.warp_range[warp * nc + rank];
    // warps of this CTA holding product items (ranges [0, nranges) non-empty)
    const int wspmv = min(kClusterWarps, max(0, (nranges - rank + nc - 1) / nc));
    // this CTA's vector entries [e0, e1), whole warps
    const int64_t chunk = ((N + nc - 1) / nc + 31) / 32 * 32;
    const int64_t e0 = min(N, static_cast<int64_t>(rank) * chunk), e1 = min(N, e0 + chunk);
    const int wvec = static_cast<int>(min(static_cast<int64_t>(kClusterWarps), (e1 - e0 + 31) / 32));
    const uint8_t *__restrict__ mult = A.mult;
    const double *__restrict__ wtab = A.wtab;
    const double rtol = s->rtol;
    const int max_iter = s->max_iter;
    int phase = 0;

    // Algorithm 3 line 1: r = b - S x_1, z = r (z = dinv r), p = z
    const int guess = s->guess;
    double arr = 0.0, abb = 0.0, arz = 0.0;
    for (int64_t i = e0 + threadIdx.x; i < e1; i += kClusterThreads) {
        const double bi = b[i];
        const double ri = guess ? bi - q[i] : bi;
        const double zi = PC ? ri * dinv[i] : ri;
        r[i] = ri;
        p[i] = zi;
        const unsigned int m = mult[i];
        arr = wsq(ri, m, wtab, arr);
        abb = wsq(bi, m, wtab, abb);
        if (PC) arz = fma(__ldg(wtab + m) * ri, zi, arz);
    }
    const double v0[3] = {arr, abb, arz};
    cluster_sums<3>(cl, red, slot, phase++, wvec, v0, [&](const double(&t)[3]) {
        cs.rr = t[0];
        cs.rho = PC ? t[2] : t[0];
        cs.bnorm = sqrt(t[1]);
        stop.init(rtol * cs.bnorm);
        // p_0 = z_0 = fma(0, p, z_0): the gather's form with beta = 0
        cs.pq = cs.alpha = cs.beta = 0.0;
        cs.k = 0;
        cs.status = SSG_E_NOT_CONVERGED;
        cs.run = 1;
        if (stop(cs.rr)) {
            cs.status = SSG_OK;
            cs.run = 0;
        } else if (max_iter <= 0) {
            cs.run = 0;
        }
    });
    // every CTA reads the same cs.run after the same barrier
    while (cs.run) {
        // lines 2-3: q = S p_k, alpha = rho / (p_k, S p_k)_w; r and p complete
        // in every CTA (the previous cluster barrier)
        const double beta = cs.beta;
        const double v1[1] = {spmv_items<double, 0, false>(A, range, PNext<PC>{r, p, dinv, beta}, q, lane)};
        cluster_sums<1>(cl, red, slot, phase++, wspmv, v1, [&](const double(&t)[1]) {
            cs.pq = t[0];
            if (!(cs.pq > 0.0) || !isfinite(cs.pq)) {
                cs.status = SSG_E_BREAKDOWN;
                cs.run = 0;
            } else {
                cs.alpha = cs.rho / cs.pq;
            }
        });
        if (!cs.run) break;
        // lines 4-5 and this CTA's share of line 8's p_k: p_k = z_k + beta
        // p_{k-1}, x <- x + alpha p_k, r <- r - alpha q and (r, r)_w (and
        // (r, z)_w); q was written by other CTAs' warps and is read through L2
        const double alpha = cs.alpha;
        double acc = 0.0, acz = 0.0;
        for (int64_t i = e0 + threadIdx.x; i < e1; i += kClusterThreads) {
            const double r0 = r[i];
            const double pk = fma(beta, p[i], PC ? r0 * dinv[i] : r0);
            p[i] = pk;
            x[i] = fma(alpha, pk, x[i]);
            const double ri = fma(-alpha, __ldcg(q + i), r0);
            r[i] = ri;
            const unsigned int m = mult[i];
            const double wi = m == 1u ? ri : __ldg(wtab + m) * ri;
            acc = fma(wi, ri, acc);
            if (PC) acz = fma(wi, ri * dinv[i], acz);
        }
        double v2[NZ];
        v2[0] = acc;
        if constexpr (PC) v2[NZ - 1] = acz;
        // line 6 and the stopping test: beta = (r, z)_{k+1} / (r, z)_k
        cluster_sums<NZ>(cl, red, slot, phase++, wvec, v2, [&](const double(&t)[NZ]) {
            const double rz = t[NZ - 1];
            cs.rr = t[0];
            cs.beta = rz / cs.rho;
            cs.rho = rz;
            cs.k += 1;
            if (stop(cs.rr)) {
                cs.status = SSG_OK;
                cs.run = 0;
            } else if (cs.k >= max_iter) {
                cs.run = 0;
            }
        });
    }
    // no CTA exits while another may still read its shared memory
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) {
        s->iter = cs.k;
        s->status = cs.status;
        s->brk = cs.status == SSG_E_BREAKDOWN;
        s->rr = cs.rr;
        s->rho = cs.rho;
        s->pq = cs.pq;
        s->alpha = cs.alpha;
        s->beta = cs.beta;
        s->bnorm = cs.bnorm;
        s->relres = cs.bnorm > 0.0 ? sqrt(cs.rr) / cs.bnorm : 0.0;
        s->total = 0;
        s->passes = 0;
        s->done = 1;
    }
}

}  // namespace ssg
