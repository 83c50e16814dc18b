/*
 * ssg.h - sub-structured Conjugate Gradient on one GPU (C ABI).
 *
 * Cheik Ahamed & Magoules, "Parallel Sub-Structuring Methods for solving
 * Sparse Linear Systems on a cluster of GPU".  The problem statement the ABI
 * follows: a sparse symmetric positive-definite system S u = f in CSR form
 * (Section 1.2, Section 2.4 Eq. linear_systems) is split into sub-structures
 * (Section 2.4: local matrices S_i whose interface blocks sum to S_33,
 * Eq. mat_subdomains / interface_summation) and solved with the Conjugate
 * Gradient (Algorithm 3) whose SpMV is the two-step local product plus
 * interface assembly (Section 3.4.1, Algorithms 4 and 5) and whose dot
 * products are interface-weighted (Section 3.4.2).  All subdomains live on
 * one GPU; the interface exchange is an on-device gather-sum-scatter.
 *
 * Conventions for every call:
 *   - Return value: SSG_OK (0) or one of the SSG_E_* codes below.  No C++
 *     exception crosses the ABI.  ssg_last_error() gives a thread-local
 *     message for the last failing call on the calling thread.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory on the context's device.  The library never takes
 *     ownership of caller memory; it owns (and frees in *_destroy) every
 *     buffer it allocates.
 *   - Device work is ordered on the context's stream (ssg_create).  Calls
 *     that return host results (ssg_solve*, ssg_copy_maps) synchronise that
 *     stream before returning; the others are asynchronous, and caller device
 *     buffers must stay valid until the stream has passed them.
 *   - Integer types are fixed width; all indices are 0-based int32.
 *   - Local vectors ("x_loc") are the concatenation over subdomains
 *     s = 0..P-1 of the local vectors of V_s (length nloc, ssg_sizes).  Every
 *     interface node has one entry per subdomain holding it; a vector is
 *     "consistent" when all copies of a node are equal.
 */
#ifndef SSG_H
#define SSG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SSG_OK 0
#define SSG_E_INVALID 1       /* bad argument, shape, index, partition id or asymmetric matrix */
#define SSG_E_OOM 2           /* host or device allocation failed */
#define SSG_E_CUDA 3          /* a CUDA runtime call failed (message in ssg_last_error) */
#define SSG_E_BREAKDOWN 4     /* (S p, p) <= 0 or not finite: matrix not SPD (Algorithm 3 line 3) */
#define SSG_E_NOT_CONVERGED 5 /* max_iter reached; x and stats hold the last iterate */
#define SSG_E_TIMEOUT 6       /* reserved: a bounded device wait expired */

/* solve modes */
#define SSG_FP64 0  /* Algorithm 3 in FP64 throughout */
#define SSG_MIXED 1 /* FP32 inner CG inside FP64 iterative refinement */
#define SSG_FP64_JACOBI 2  /* Algorithm 3 with the diagonal preconditioner M = diag(S) of the \
                              paper's experiments (Section 3.1), FP64 */
#define SSG_MIXED_JACOBI 3 /* SSG_MIXED with the diagonal preconditioner in the FP32 inner solves */

/* driver modes (ssg_set_driver) */
#define SSG_DRIVER_GRAPH 0 /* one CUDA-graph launch per solve, device-side while loop */
#define SSG_DRIVER_HOST 1  /* host loop of direct launches, done-flag polled every 32 iterations */

typedef struct ssg_ctx ssg_ctx;
typedef struct ssg_system ssg_system;

typedef struct {
    int32_t n;        /* global unknowns */
    int32_t P;        /* subdomains */
    int64_t nnz;      /* stored nonzeros of S (= sum of local nonzeros) */
    int64_t nloc;     /* sum over s of |V_s| (length of local vectors) */
    int32_t ngamma;   /* interface nodes (multiplicity >= 2) */
    int32_t max_mult; /* largest multiplicity */
    int64_t ncopies;  /* sum of multiplicities over interface nodes */
} ssg_sizes;

typedef struct {
    int32_t status;          /* SSG_OK, SSG_E_BREAKDOWN or SSG_E_NOT_CONVERGED for this right-hand side */
    int32_t iters;           /* CG iterations (mixed mode: inner iterations summed over refinements) */
    int32_t outer;           /* refinement steps (mixed mode); 1 in FP64 mode */
    int32_t block;           /* right-hand sides that iterated together with this one (1, 2, 4, 8 or 16) */
    double relres;           /* final recursive residual sqrt((r,r)_w) / sqrt((b,b)_w) */
    double true_relres;      /* ||b - S x|| / ||b|| recomputed in FP64 after the solve */
    double solve_ms;         /* device time of this solve (CUDA events on the context stream); for a
                                block of right-hand sides, the time of the whole block; for a
                                batch, of its longest column group (the groups overlap) */
    int64_t kernel_launches; /* kernels executed on the device for this solve (or block, or batch) */
} ssg_stats;

/*
 * Create a context on CUDA device `device`; work is issued on `stream`
 * (a cudaStream_t, or NULL for the legacy default stream).  The stream is
 * borrowed and must outlive the context.
 */
int ssg_create(ssg_ctx **ctx, int device, void *stream);
/* Change the stream later calls on this context use (borrowed). */
int ssg_set_stream(ssg_ctx *ctx, void *stream);
/* Pick how ssg_solve drives the iteration (SSG_DRIVER_*); default GRAPH. */
int ssg_set_driver(ssg_ctx *ctx, int driver);
/* CG iterations per pass of the body of a single-vector solve's loop graph
 * (1..8, default 4): the body holds that many copies of one iteration's
 * kernels; once the loop has stopped, the later copies of the last pass
 * return at once (the host-loop driver relies on the same flags).  Results
 * are unchanged.  Each pass of a conditional loop costs about 1.9 us on
 * GB300: on the 128^3 system 4 copies per pass take 39.7 us per mixed inner
 * iteration and 73.0 us per FP64 iteration, against 41.5 and 74.7 with one.
 * Applies to systems partitioned on this context afterwards. */
int ssg_set_unroll(ssg_ctx *ctx, int32_t iters);
/* Layout of the local matrices' interior rows in the sliced-ELL copy the
 * products stream (Section 3.4.1's local SpMV; the layout is this library's,
 * the products are unchanged): a slice holds 32 rows, one per lane, padded
 * to its longest row.  window = 1: a slice is 32 consecutive rows; > 1: each
 * window of that many consecutive rows is ordered by decreasing length first
 * (SELL-C-sigma), so rows of equal length share slices and padding shrinks,
 * at the cost of a 4-byte row index per row; -1: the window is the whole
 * subdomain; 0 (default): per subdomain, the window of {1, 128, 256, 512}
 * rows whose slices move the fewest bytes by its row-length histogram,
 * sorting only when it saves at least 2 %.  Each row's entries keep their
 * order, so the product's entries are the same bits in every layout (the
 * block partial sums of its weighted dot group rows differently).  Applies
 * to systems partitioned on this context afterwards; SSG_E_INVALID for
 * window < -1. */
int ssg_set_slice_sort(ssg_ctx *ctx, int32_t window);
/*
 * One-cluster solve of small systems (Algorithm 3 of Section 3.4, the whole
 * iteration loop in one kernel launch).  Under the graph driver, a
 * single-right-hand-side SSG_FP64 or SSG_FP64_JACOBI solve of a system with
 * at most max_nloc local entries (|V_1| + ... + |V_P|) runs as one thread-block
 * cluster of up to 16 CTAs, one per SM, instead of three kernels per
 * iteration.  Its CTAs exchange the weighted dots' per-CTA sums through
 * distributed shared memory and add them in one fixed order in every CTA,
 * and meet at two cluster barriers per iteration.  The product's rows and
 * interface sums are the same bits as the multi-kernel loop's.  The dots'
 * partial sums are grouped differently, so iterates agree to rounding and the
 * iteration count may differ by a few.  max_nloc = 0 turns it off; default
 * 12288 (on GB300 the one-cluster solve takes 7.1 us per FP64 iteration on
 * the 64 x 64 Poisson system against 13.3 for the loop; its 16 SMs' FP64
 * rate makes it the slower one beyond about 12-16 thousand entries).  ctas: CTAs per cluster (2, 4, 8 or 16, capped at what the device
 * places), or 0 for the device's largest.  max_nloc applies to solves issued
 * afterwards; ctas to systems partitioned on this context afterwards.
 * SSG_E_INVALID for max_nloc < 0 or another ctas.
 */
int ssg_set_cluster_solve(ssg_ctx *ctx, int64_t max_nloc, int32_t ctas);
/* The current limit, and the most CTAs per cluster the device places (0: the
 * one-cluster solve is unavailable and never used).  Either pointer may be
 * NULL. */
int ssg_get_cluster_solve(const ssg_ctx *ctx, int64_t *max_nloc, int32_t *ctas);
/*
 * Parameters of SSG_MIXED solves on this context (not a method of the paper;
 * its experiments are FP64 only): the inner FP32 CG stops when its residual
 * has dropped by inner_rtol (or by the factor the outer test still needs, if
 * that is larger), and at most max_outer refinements run.  Defaults 1e-4, 30.
 * SSG_E_INVALID unless 0 < inner_rtol < 1 and max_outer >= 1.
 */
int ssg_set_mixed(ssg_ctx *ctx, double inner_rtol, int32_t max_outer);
/*
 * How many right-hand sides of one ssg_solve call iterate together: kmax =
 * 1, 2, 4, 8 or 16 (default 16).  A group of k > 1 right-hand sides runs K
 * Algorithm 3 iterations side by side (K = the power of two >= k, the extra
 * columns zero), each with its own alpha, beta and stopping test, and reads
 * the local matrices once per iteration for all of them (the product of
 * Section 3.4.1 with K vectors).  A right-hand side whose test has passed
 * stops changing, so each one gets the iterates of its own solve up to the
 * order of the floating-point sums.  kmax = 1 solves them one after another.
 */
int ssg_set_rhs_block(ssg_ctx *ctx, int32_t kmax);
/* Free a context.  Refused with SSG_E_INVALID (nothing freed) while systems
 * created on it are still alive: destroy those first. */
int ssg_destroy(ssg_ctx *ctx);

/*
 * Sub-structuring of Section 2.4 (Eq. 2.4:eqn0, mat_subdomains,
 * interface_summation) for an assembled matrix, plus the interface lists of
 * Section 3.4.2 (for every interface node, the subdomains that hold it).
 *
 * Inputs (host, copied): S in 0-based CSR (rowptr[n+1], colidx[nnz],
 * val[nnz]); columns sorted and unique in each row; the pattern and the values
 * symmetric (exactly); part[n] gives the subdomain 0..P-1 of every node.
 * Rules (where the paper only treats finite-element assembly, the reading for
 * an assembled matrix):
 *   V_s = {i : part(i) = s} U {j : A_ij stored for some i with part(i) = s < part(j)}
 *   m_j = number of V_s holding j; interface nodes have m_j >= 2 (m_j <= 255)
 *   local order in V_s: nodes with m = 1 ascending by id, then interface nodes
 *   ascending by id (interior first, interface last, as in Eq. 2.4:eqn0)
 *   entry (i,i) belongs to S^(part(i)); entry (i,j), i != j, to
 *   S^(min(part(i), part(j))), so the local matrices sum exactly to S.
 *   Interface copies of a node are listed in ascending subdomain order.
 * With ctx == NULL only the host maps are built (ssg_get_sizes,
 * ssg_copy_maps and ssg_get_layout, with the default layout rule, work;
 * device calls return SSG_E_INVALID).  Otherwise the
 * device arena is allocated and filled on the context stream.
 * Errors: SSG_E_INVALID for any malformed input, SSG_E_OOM, SSG_E_CUDA.
 */
int ssg_partition(ssg_ctx *ctx, int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                  const int32_t *part, int32_t P, ssg_system **sys);

/*
 * Sub-structures from finite elements, as Section 2.4 builds them: subdomain
 * s owns the elements e with epart[e] = s; V_s is the set of free nodes of its
 * elements; its local matrix is the sum of its own element matrices in local
 * numbering (S_s = sum over e in s of K_e, each entry summed in ascending
 * element order), so the interface blocks of the local matrices add up to the
 * global one (Eq. interface_summation) and every S_s is a Neumann matrix.
 * Inputs (host, copied): ne elements of nv nodes, elem[e*nv + a] in [0, n)
 * or -1 for an eliminated (Dirichlet) node whose row and column are dropped;
 * kel[(e*nv + a)*nv + b] the symmetric element matrices; epart[e] in [0, P).
 * Numbering, multiplicities, interface lists and weights follow
 * ssg_partition; the owner copy of a node is its copy in the lowest
 * subdomain; SSG_FP64_JACOBI uses the assembled diagonal (the copies'
 * diagonal entries summed in ascending s).  Such a system has no input-CSR
 * values: ssg_set_values, ssg_pattern_grad and ssg_fv7_* refuse it.
 * SSG_E_INVALID for part ids or node ids out of range, a non-symmetric
 * element matrix, or a node that belongs to no element.
 */
int ssg_partition_fe(ssg_ctx *ctx, int32_t n, int32_t ne, int32_t nv, const int32_t *elem, const double *kel,
                     const int32_t *epart, int32_t P, ssg_system **sys);

/*
 * A batch of independent systems solved together (not in the paper; its
 * method is one system).  The caller passes the union of the systems as one
 * block-diagonal CSR (the input conventions of ssg_partition): system s owns
 * the nodes [sys_node_off[s], sys_node_off[s+1]) and the subdomain ids
 * [sys_sub_off[s], sys_sub_off[s+1]) (every one of its nodes' part values
 * lies there; no stored entry couples two systems), and has sys_nrhs[s]
 * right-hand sides (1..16).  nsys + 1 offsets, both starting at 0, strictly
 * increasing.  The sub-structures are built as by ssg_partition for the
 * union; the product's work is cut per system so that every block of every
 * kernel works inside one system.  SSG_E_INVALID for bad tables, a node whose
 * subdomain lies outside its system's range or an entry coupling two systems.
 */
int ssg_partition_batch(ssg_ctx *ctx, int32_t nsys, const int32_t *sys_node_off, const int32_t *sys_sub_off,
                        const int32_t *sys_nrhs, const int32_t *rowptr, const int32_t *colidx, const double *val,
                        const int32_t *part, ssg_system **sys);
/*
 * Solve every system of a batch for its right-hand sides in one graph
 * launch: each (system, right-hand side) runs its own Algorithm 3 (SSG_FP64,
 * SSG_FP64_JACOBI) or its own refinement (SSG_MIXED, SSG_MIXED_JACOBI) with
 * the readings of ssg_solve.  Systems are grouped by column count K (the
 * power of two >= their sys_nrhs, at least 2); the columns of all systems of
 * a group iterate together, every group's loop is a branch of one graph
 * launched once (groups side by side), and a finished system's blocks
 * return at once.  b and x
 * (device, rhs_off[nsys] doubles each, caller-allocated: the library cannot
 * check their length) hold system s's right-hand side j at rhs_off[s] + j * n_s, with
 * rhs_off[s] = sum over s' < s of sys_nrhs[s'] * n_s' (n_s = its node count);
 * stats (host, may be NULL) receives one entry per (system, right-hand side)
 * in that order.  max_iter <= 0 means the largest n_s.  Returns SSG_OK when
 * every right-hand side converged, else the first non-OK status.
 */
int ssg_solve_batch(ssg_system *sys, const double *b, double *x, int32_t x_is_guess, double rtol, int32_t max_iter,
                    int32_t mode, ssg_stats *stats);
/*
 * How a batch whose systems fall into several column groups runs with the
 * graph driver (not in the paper): one_graph != 0 (the default) launches one
 * graph whose parallel branches are the groups' loops; 0 launches each
 * group's own loop graph on a stream of its own, side by side.  The second
 * form is also what a solve falls back to when the one-graph form cannot be
 * built.  Both give the same bits.  SSG_E_INVALID for a null system.
 */
int ssg_set_batch_graph(ssg_system *sys, int32_t one_graph);

/*
 * This GPU's FP64 fused multiply-add rate, measured (not in the paper): the
 * denominator of the rooflines of FP64-bound kernels.  Eight 256-thread
 * blocks per SM each keep 8 independent FMA chains per thread going for
 * `iters` steps; the best of `reps` timed launches (CUDA events on the
 * context's stream, after one untimed launch) gives *tflops (2 flops per FMA)
 * and *best_ms (may be NULL).  Allocates and frees a small sink buffer.
 * SSG_E_INVALID for a null context or result, iters or reps < 1.
 */
int ssg_measure_fp64_rate(ssg_ctx *ctx, int32_t iters, int32_t reps, double *tflops, double *best_ms);
int ssg_get_sizes(const ssg_system *sys, ssg_sizes *out);
/* The interior slice layout a system got (ssg_set_slice_sort): out[0] =
 * entries stored in interior slices (padding included), out[1] = nonzeros
 * they hold, out[2] = subdomains whose slices are sorted by row length,
 * out[3] = the largest sorting window (1: none).  Host memory, 4 int64. */
int ssg_get_layout(const ssg_system *sys, int64_t *out);
/* The interface layout of a system's products (Algorithms 4/5 fused into
 * them).  Every product can read the interface copy rows as slices of whole
 * nodes, up to 32 copy rows in (node, copy) order, one copy row per lane, the
 * node sums formed by warp shuffles; a slice pads every copy row to its
 * longest, and a node's copies in the lower subdomains hold only the entries
 * those own (one on a face of the 7-point grids, against six in the owner's
 * row).  The FP64 single-vector product can instead read groups of up to 32
 * nodes of one multiplicity m, one node per lane, its m copy rows in m
 * sub-slices padded rank by rank, the node sum formed in the lane (the same
 * operations in the same order: the same products).  It takes the groups
 * when they store at least 4 % of all its sliced entries fewer; the FP32
 * and K-vector products and the one-cluster solve always read the slices.
 * out[0] = entries stored in interface slices, out[1] = in interface groups
 * (both with padding), out[2] = 1 if the FP64 single-vector product reads
 * the groups.
 * Host memory, 3 int64; SSG_E_INVALID for a null argument. */
int ssg_get_iface_layout(const ssg_system *sys, int64_t *out);

/*
 * Copy the sub-structure maps into caller host buffers (any pointer may be
 * NULL to skip it).  Sizes from ssg_sizes:
 *   off[P+1]      first concatenated local index of each subdomain
 *   nint[P]       interior (m = 1) nodes of each subdomain (they come first)
 *   l2g[nloc]     global node of each local entry (the local-to-global map, Section 2)
 *   mult[n]       multiplicity of every global node
 *   lrowptr[nloc+1], lcol[nnz], lval[nnz]
 *                 local matrices, concatenated; lcol holds the column's local
 *                 index inside its own subdomain; values copied unchanged
 *   gamma[ngamma] interface nodes, ascending global id
 *   iptr[ngamma+1], icopy[ncopies]
 *                 concatenated local indices of each interface node's copies,
 *                 ascending subdomain
 *   own[n]        local index of node i's copy in subdomain part(i)
 */
int ssg_copy_maps(const ssg_system *sys, int32_t *off, int32_t *nint, int32_t *l2g, int32_t *mult,
                  int32_t *lrowptr, int32_t *lcol, double *lval, int32_t *gamma, int32_t *iptr, int32_t *icopy,
                  int32_t *own);

/* Global -> local: x_loc[k] = x_glob[l2g[k]] (device pointers, n and nloc long). */
int ssg_scatter(ssg_system *sys, const double *x_glob, double *x_loc);
/* Local -> global: x_glob[i] = x_loc[own[i]] (device pointers). */
int ssg_gather(ssg_system *sys, const double *x_loc, double *x_glob);

/*
 * The sub-structured SpMV of Section 3.4.1: local products y_s = S_s x_s for
 * every subdomain, then assembly of the interface contributions (the
 * collect/send and receive/update of Algorithms 4 and 5, done on the device):
 * every copy of an interface node receives the sum of its copies' local
 * values, summed in ascending subdomain order.  x_loc must be consistent for
 * y_loc to be the global product.  Device pointers, nloc long, must not
 * overlap.  If xSx_dev is not NULL it receives (x, S x)_w on the device (the
 * launch then ends with a last-block sum of the block partials); with NULL
 * the launch is the solver loop's own instance (block partials only).
 */
int ssg_spmv_assembled(ssg_system *sys, const double *x_loc, double *y_loc, double *xSx_dev);

/*
 * The same sub-structured SpMV with the values rounded to FP32 and FP32
 * vectors and arithmetic (the inner operator of SSG_MIXED solves; the paper
 * itself computes in FP64).  Rows summed in CSR order with FP32 FMAs,
 * interface copies summed in ascending subdomain order in FP32; xSx_dev (may
 * be NULL) receives (x, S x)_w summed in FP64.  Device pointers, nloc floats,
 * must not overlap.
 */
int ssg_spmv_assembled_f32(ssg_system *sys, const float *x_loc, float *y_loc, double *xSx_dev);

/* Result of ssg_autotune: per precision, the launch shape (blocks per SM)
 * and L2 prefetch distance of every candidate, its mean launch time, and the
 * index chosen. */
#define SSG_TUNE_CANDIDATES 6
typedef struct {
    int32_t fp64_choice, fp32_choice;
    int32_t fp64_blocks_per_sm[SSG_TUNE_CANDIDATES], fp64_l2_ahead[SSG_TUNE_CANDIDATES];
    int32_t fp32_blocks_per_sm[SSG_TUNE_CANDIDATES], fp32_l2_ahead[SSG_TUNE_CANDIDATES];
    double fp64_us[SSG_TUNE_CANDIDATES], fp32_us[SSG_TUNE_CANDIDATES];
} ssg_tune;
/*
 * Time the single-vector SpMV instances (launch shapes of 3 to 6 blocks per
 * SM, L2 prefetch of the next slices on or off; six per precision) on this
 * system as the solver loop launches them (block partials, no last-block
 * sum), reps launches each (reps <= 0: 20), and use the fastest for the
 * following solves and products.  The choice changes only the order of the
 * block partial sums (results within the same rounding bounds; bit-for-bit
 * repeatable once chosen).  Without a call the defaults are entry 0, the
 * measured best on the 128^3 finite-volume system.  Blocks until done;
 * graphs built earlier are rebuilt on the next solve.
 */
int ssg_autotune(ssg_system *sys, int32_t reps, ssg_tune *out);

/* Result of ssg_autotune_block: the column count tuned for, each
 * candidate's entries loaded at once and L2 look-ahead, its mean launch time
 * per precision, and the index chosen. */
#define SSG_TUNE_BLOCK_CANDIDATES 6
typedef struct {
    int32_t k;
    int32_t fp64_choice, fp32_choice;
    int32_t nc[SSG_TUNE_BLOCK_CANDIDATES], l2_ahead[SSG_TUNE_BLOCK_CANDIDATES];
    double fp64_us[SSG_TUNE_BLOCK_CANDIDATES], fp32_us[SSG_TUNE_BLOCK_CANDIDATES];
} ssg_tune_block;
/*
 * Tune the product with k vectors (Section 3.4.1's SpMV with several
 * right-hand sides; not in the paper) as ssg_solve and ssg_solve_batch launch
 * it: sliced entries loaded at once per lane (1 or 2) x slices ahead whose
 * lines are prefetched into L2 (0, 1, 2), timed in FP64 and FP32 (reps
 * launches each, reps <= 0: 20), the fastest kept for the following solves
 * with that k.  Neither changes the arithmetic: results are the same bits
 * with every candidate.  A batch of systems tunes every column group for its
 * own K (k is then ignored) and reports the group with the most columns.
 * Allocates the K-column vectors if needed; blocks until done; graphs built
 * earlier are rebuilt on the next solve.  SSG_E_INVALID for another k.
 */
int ssg_autotune_block(ssg_system *sys, int32_t k, int32_t reps, ssg_tune_block *out);

/*
 * The sub-structured product of ssg_spmv_assembled with k vectors at once
 * (k = 2, 4, 8 or 16): x_loc and y_loc are device blocks of nloc*k doubles,
 * interleaved (entry i of vector j at i*k + j), aligned to 16 bytes.  The
 * local matrices are read once for all k vectors; each column of y_loc is
 * bit-identical to ssg_spmv_assembled of that column (same summation
 * order).  SSG_E_INVALID for another k, null, aliased or misaligned blocks.
 */
int ssg_spmm_assembled(ssg_system *sys, int32_t k, const double *x_loc, double *y_loc);
/* The same in FP32 (values rounded to FP32 once, FP32 arithmetic; columns
 * bit-identical to ssg_spmv_assembled_f32); blocks aligned to
 * min(16, 4k) bytes. */
int ssg_spmm_assembled_f32(ssg_system *sys, int32_t k, const float *x_loc, float *y_loc);

/*
 * Interface-weighted dot of Section 3.4.2: result = sum_k w_k u_k v_k over the
 * nloc local entries with w_k the system's weight of entry k (ssg_set_weights:
 * 1/m of the entry's node by default; either weighting equals the global dot
 * for consistent vectors).  Device pointers; *result_dev is written on the
 * device.  Deterministic for a given system.
 */
int ssg_wdot(ssg_system *sys, const double *u_loc, const double *v_loc, double *result_dev);

/* weightings of the weighted dots (ssg_set_weights) */
#define SSG_WEIGHT_INV_MULT 0 /* w = 1/m on each of a node's m copies (the default) */
#define SSG_WEIGHT_OWNER 1    /* w = 1 on the node's owner copy, 0 on its other copies */
/*
 * The weights of every weighted dot the system forms (Section 3.4.2 combines
 * the subdomains' sums with weights it does not give): the solves' (r, r)_w,
 * (r, z)_w, (p, S p)_w and ||b||_w, the true residual and ssg_wdot.
 * SSG_WEIGHT_INV_MULT: w = 1/m on each copy of a node of multiplicity m.
 * SSG_WEIGHT_OWNER: the owner mask, w = 1 on the node's owner copy (the copy
 * ssg_copy_maps reports in own: in subdomain part(i) for ssg_partition, in the
 * lowest subdomain for ssg_partition_fe) and 0 on its other copies, so that
 * each node is counted once with no division.  Both sum to 1 over a node's
 * copies: for consistent vectors both dots are the global dot in exact
 * arithmetic, and the solves' iterates agree to rounding.  Applies to later
 * calls (loop graphs built before are rebuilt; for a batch, every column
 * group); blocks until the context's stream is idle.  SSG_E_INVALID for
 * another mode or a system without device data.
 */
int ssg_set_weights(ssg_system *sys, int32_t mode);

/*
 * Solve S x = b for k right-hand sides with Algorithm 3 (M = I) on the
 * sub-structured operator.  b and x are device pointers to n*k doubles,
 * right-hand side j at offset j*n.  If x_is_guess is nonzero x holds the
 * initial guess x_1, else the iteration starts from 0.  Readings where the
 * paper is silent: stop after the first iteration with
 * sqrt((r,r)_w) <= rtol * sqrt((b,b)_w) (recursive residual) or after
 * max_iter iterations (max_iter <= 0 means n).  mode = SSG_FP64, SSG_MIXED or
 * SSG_FP64_JACOBI.  SSG_FP64_JACOBI: z = M^-1 r with M = diag(S) (stored as
 * the reciprocal 1 / S_ii per local entry), alpha = (r, z)_w / (S p, p)_w,
 * beta = (r, z)_w(k+1) / (r, z)_w(k), p = z + beta p; the stopping test stays
 * on (r, r)_w; SSG_E_INVALID if a diagonal entry is missing or not positive.
 * SSG_MIXED_JACOBI: the refinement of SSG_MIXED whose inner FP32 solves use
 * the same preconditioner (z = r * 1/S_ii rounded to FP32, the inner test on
 * (r, r)_w).
 * SSG_MIXED: iterative refinement in FP64 (r = b - S x with the FP64
 * sub-structured SpMV, x += d, the stopping test on that true residual)
 * around an inner Algorithm 3 in FP32 (values, vectors and SpMV in FP32, dot
 * products summed in FP64) on S d = r; max_iter then caps the inner
 * iterations summed over refinements (ssg_set_mixed sets the inner tolerance
 * and the refinement cap).
 * Groups of up to ssg_set_rhs_block right-hand sides iterate together.
 * stats (host, may be NULL) receives k entries.  Blocks until done.
 * Returns SSG_OK when every right-hand side converged, else the first
 * non-OK per-RHS status (x still holds the last iterates).
 */
int ssg_solve(ssg_system *sys, int32_t k, const double *b, double *x, int32_t x_is_guess, double rtol,
              int32_t max_iter, int32_t mode, ssg_stats *stats);

/* Same as ssg_solve with b and x in host memory (copied in and out on the
 * context stream inside the call). */
int ssg_solve_host(ssg_system *sys, int32_t k, const double *b_host, double *x_host, int32_t x_is_guess,
                   double rtol, int32_t max_iter, int32_t mode, ssg_stats *stats);

/*
 * Differentiable solves (not in the paper; its method is the forward solve).
 *
 * ssg_set_values: new matrix values for the same pattern.  val (device, nnz
 * doubles) is in the order of the CSR given to ssg_partition; every device
 * copy of the local matrices (FP64 and the FP32 rounding of SSG_MIXED) is
 * refreshed on the context stream.  The values must stay symmetric and the
 * matrix positive definite (a solve reports SSG_E_BREAKDOWN otherwise); the
 * host maps of ssg_copy_maps keep the values given at partition time.
 *
 * ssg_pattern_grad: g[e] = -sum_{j<k} lam[j*n + i] * x[j*n + c] for each
 * stored entry e = (i, c) of that CSR (device, nnz doubles): the gradient of
 * a loss L(x) with respect to the stored entries of S when S x_j = b_j and
 * S lam_j = dL/dx_j (S symmetric).  lam and x: device, n*k, column j at j*n.
 */
int ssg_set_values(ssg_system *sys, const double *val);
int ssg_pattern_grad(ssg_system *sys, int32_t k, const double *lam, const double *x, double *g);
/*
 * 7-point finite-volume diffusion on an nx x ny x nz cell grid (the synthetic
 * workloads): cell (ix, iy, iz) = ix + nx (iy + ny iz), kappa = exp(logk),
 * an interior face carries the harmonic mean 2 k_a k_b / (k_a + k_b), a
 * boundary face 2 k; A_ij = -t of the shared face, A_ii = sum of the cell's
 * six face coefficients.  ssg_fv7_values writes the nnz values (device, CSR
 * order, columns ascending in each row); ssg_fv7_adjoint maps g = dL/dA
 * (device, CSR order) to dL/dlogk (device, n).  The system's matrix must
 * have this grid's 7-point pattern (checked on the host at the first call
 * for a grid: SSG_E_INVALID otherwise).
 */
int ssg_fv7_values(ssg_system *sys, int32_t nx, int32_t ny, int32_t nz, const double *logk, double *val);
int ssg_fv7_adjoint(ssg_system *sys, int32_t nx, int32_t ny, int32_t nz, const double *logk, const double *g,
                    double *glogk);

int ssg_system_destroy(ssg_system *sys);

/*
 * Interface-weighted dot, (u, v)_w = sum_k w_k u_k v_k with w_k = 1/mult_loc[k],
 * for callers that cannot let a library allocate device memory (this call
 * has no counterpart in the paper).  Such callers: programs whose own
 * allocator owns the device memory under a fixed budget, where an allocation
 * made behind its back can fail or starve it; loops that must not take the
 * implicit device synchronisation cudaMalloc/cudaFree can cause.
 *
 * No system is needed.  All arguments are device pointers owned by the
 * caller: u_loc, v_loc (nloc doubles), mult_loc (nloc bytes, the multiplicity
 * 1..255 of each local entry's node, i.e. mult[l2g[k]] from ssg_copy_maps;
 * an entry with multiplicity 0 gets weight 0, as in the system path),
 * result_dev (one double, written on the device).  The library cannot see
 * the buffers' lengths: each must hold nloc elements (result_dev one) on the
 * current device, or the kernel reads out of bounds.  Work goes to `stream`
 * (cudaStream_t or NULL) on the calling thread's current device.
 * Scratch: a 64 KB static __device__ array that every GPU loading this
 * library keeps until the process exits; nothing is allocated or freed.
 * Limit: nloc <= 33,554,432 (8192 partial sums of 4096 entries); larger
 * nloc, a negative nloc or a null pointer returns SSG_E_INVALID.
 * The first call on a device looks up the scratch address on that device
 * (cudaGetSymbolAddress); later calls on it reuse the address.  Every call shares the one
 * scratch array: calls that can overlap on the GPU (different streams, or
 * threads) race and must be serialised by the caller.
 */
int ssg_wdot_noalloc(const double *u_loc, const double *v_loc, const uint8_t *mult_loc, int64_t nloc,
                     double *result_dev, void *stream);

/*
 * Band splittings (Sections 2.1 and 2.2, Algorithms 1 and 2): the paper's
 * two other ways of sharing a matrix among processors, kept here as
 * comparison operators for the sub-structured product.  Band p of nb
 * (0-based) covers q = floor(n / nb) rows (SSG_BAND_ROW) or columns
 * (SSG_BAND_COL) starting at displ = p q; the last band takes the rest.
 *   SSG_BAND_ROW: band p is the N_p x n CSR matrix of rows [displ, displ +
 *     N_p): A's row pointers shifted to start at 0, A's global column ids and
 *     values copied in order (Algorithm 1).  y = A x: each band writes its
 *     block of y from the whole of x.
 *   SSG_BAND_COL: band p is the n x N_p CSR matrix of the entries of every
 *     row whose column lies in [displ, displ + N_p), column ids shifted by
 *     displ (Algorithm 2; reading: the listing's column offset is the band's
 *     first column).  y = A x is the sum of the bands' partial products
 *     A_p x[displ .. displ + N_p), taken in ascending p (reading: the paper
 *     gives no order for that sum; a fixed one keeps y reproducible).
 * On one GPU every band lives in the same memory, so the device keeps A once
 * (the bands of either splitting are row or column ranges of it) and one
 * kernel computes all bands' products; each row's entries are summed left to
 * right with fused multiply-adds, per band for SSG_BAND_COL.
 *
 * ssg_band_split: inputs (host, copied): A in 0-based CSR with columns sorted
 *   and unique in each row (no symmetry needed; empty rows allowed), 1 <= nb
 *   <= n.  SSG_E_INVALID otherwise.  Uploads A and the kernel's tile table.
 * ssg_band_get: band p's sizes (sizes[0] = N_p, sizes[1] = displ, sizes[2] =
 *   nnz of the band) and, when the pointers are not NULL, its CSR arrays into
 *   caller host buffers (rowptr: N_p + 1 or n + 1 entries; colidx, val: nnz).
 * ssg_band_spmv: y = A x through the band's splitting; x and y are device
 *   vectors of n doubles (not overlapping), ordered on the context stream.
 * ssg_band_set_variant: which kernel computes the product:
 *   SSG_BAND_AUTO (the row-length rule: one thread per row while the mean
 *   row length is at most 8, else lanes per row = the power of two >= half
 *   the mean row length, from 2 to 32; band-column: one thread per row),
 *   SSG_BAND_STAGED (tiles of whole rows staged in shared
 *   memory by bulk asynchronous copies, one thread per row: the left-to-right
 *   order), 1 (one thread per row from global memory, left to right), or
 *   2, 4, 8, 16, 32 lanes per row (strided partial sums, then a fixed
 *   shuffle tree: same products, another summation order; SSG_BAND_ROW only).
 * ssg_band_autotune: times every variant valid for the splitting (reps
 *   launches each, CUDA events on the context stream), keeps the fastest and
 *   reports each variant's mean time in microseconds (us[i] for variant
 *   code[i], 0 where not valid).
 */
#define SSG_BAND_ROW 0
#define SSG_BAND_COL 1
#define SSG_BAND_AUTO 0
#define SSG_BAND_STAGED (-1)
typedef struct ssg_band ssg_band;
typedef struct {
    int32_t variant;      /* the variant now in use */
    int32_t rule_variant; /* what SSG_BAND_AUTO picks for this matrix */
    int32_t code[7];      /* SSG_BAND_STAGED, 1, 2, 4, 8, 16, 32 */
    float us[7];
} ssg_band_tune;
int ssg_band_split(ssg_ctx *ctx, int32_t kind, int32_t n, const int32_t *rowptr, const int32_t *colidx,
                   const double *val, int32_t nb, ssg_band **out);
int ssg_band_get(const ssg_band *band, int32_t p, int64_t *sizes, int32_t *rowptr, int32_t *colidx, double *val);
int ssg_band_spmv(ssg_band *band, const double *x, double *y);
int ssg_band_set_variant(ssg_band *band, int32_t variant);
int ssg_band_autotune(ssg_band *band, int32_t reps, ssg_band_tune *out);
/*
 * ssg_band_check_timeout: runs the staged kernel's bounded wait once on an
 * mbarrier phase that nothing completes (no copy issued, nothing in flight):
 * the wait gives up after one second, raises the operator's error flag, and
 * the call returns SSG_E_TIMEOUT (then clears the flag; the context and the
 * operator stay usable).  Any other status means the failure path did not
 * work.  A test of failure detection without a GPU fault.
 */
int ssg_band_check_timeout(ssg_band *band);
int ssg_band_destroy(ssg_band *band);

const char *ssg_error_string(int status);
const char *ssg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SSG_H */
