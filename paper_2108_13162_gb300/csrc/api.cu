// C ABI of the sub-structured CG library: contexts, device upload of the
// sub-structures, the SpMV/dot entry points and the solve driver.
//
// The solve runs Algorithm 3 (M = I) with the whole iteration on the device:
// one CUDA graph holds the setup kernel and a conditional WHILE node whose
// body is {sub-structured SpMV + alpha, residual update + beta, x/p update};
// the kernels decide convergence and clear the loop condition themselves, so
// the host synchronises once per solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "adjoint.cuh"
#include "block.cuh"
#include "cluster.cuh"
#include "kernels.cuh"
#include "ssg_ctx.h"
#include "ssg_internal.h"

namespace ssg {

static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }

}  // namespace ssg

using namespace ssg;

struct ssg_system {
    ssg_ctx *ctx = nullptr;
    HostMaps maps;
    bool on_device = false;
    // device arena
    void *arena = nullptr;
    size_t arena_bytes = 0;
    DevOp op{};    // FP64 SpMV launch (warp ranges for grid_spmv blocks)
    DevOp op32{};  // FP32 SpMV launch (warp ranges for grid_spmv32 blocks)
    int32_t *d_l2g = nullptr;
    int32_t *d_own = nullptr;
    // solver state
    double *d_bl = nullptr, *d_xl = nullptr, *d_r = nullptr, *d_p = nullptr, *d_q = nullptr;
    float *d_r32 = nullptr, *d_p32 = nullptr, *d_q32 = nullptr, *d_d32 = nullptr;  // SSG_MIXED inner vectors
    Scal *d_scal_in = nullptr;  // SSG_MIXED inner CG state
    double *d_partials = nullptr;
    int32_t n_partials = 0;
    Scal *d_scal = nullptr;     // CG state
    int32_t *d_dmap = nullptr;  // local entry holding the diagonal of each local entry's node
    double *d_dinv = nullptr;   // 1 / diag(S) per local entry (SSG_FP64_JACOBI)
    float *d_dinv32 = nullptr;
    int *d_diag_bad = nullptr;  // set by k_dinv on a missing or non-positive diagonal
    int diag_state = -1;        // host copy of *d_diag_bad: -1 not read since the values changed
    Scal *d_scal_op = nullptr;  // state for the stand-alone SpMV / dot calls
    double *d_xg = nullptr, *d_bg = nullptr;  // global staging for ssg_solve_host
    int unroll = 4;     // iterations per pass of the single-vector loop bodies
    // the interior slice layout (make_plan): entries stored with padding, real
    // entries, subdomains sorted by row length, the largest sorting window
    int64_t slice_slots = 0, slice_entries = 0;
    int32_t sorted_subdomains = 0, max_window = 1;
    // the interface layout: entries stored in interface slices and in
    // interface groups (padding included)
    int64_t iface_slots = 0, group_slots = 0;
    int grid_spmv = 0;
    int grid_spmv32 = 0;
    int grid_bps[7] = {0, 0, 0, 0, 0, 0, 0};        // single-vector grids for 3 to 6 blocks per SM
    const int2 *range_bps[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int grid_bps32[7] = {0, 0, 0, 0, 0, 0, 0};      // the same for the FP32 product (interface slices)
    const int2 *range_bps32[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int var64 = 0, var32 = 0;                       // chosen SpMV instances (ssg_autotune)
    // weights of the weighted dots (ssg_set_weights): the multiplicity codes
    // (w = 1/m) and the owner-mask codes; the operators read one of them
    const uint8_t *d_mult = nullptr, *d_wown = nullptr;
    int32_t weight_mode = SSG_WEIGHT_INV_MULT;
    int grid_vec = 0;
    // one-cluster solve: warp ranges for cluster_ctas CTAs (warp w of CTA c
    // takes range w * cluster_ctas + c), the first cluster_nranges non-empty
    const int2 *range_cluster = nullptr;
    int32_t cluster_ctas = 0, cluster_nranges = 0;
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle cond = 0;
    cudaGraph_t graph_pc = nullptr;  // SSG_FP64_JACOBI
    cudaGraphExec_t exec_pc = nullptr;
    cudaGraphConditionalHandle cond_pc = 0;
    cudaGraph_t graph_m[2] = {nullptr, nullptr};  // SSG_MIXED, SSG_MIXED_JACOBI: nested loops
    cudaGraphExec_t exec_m[2] = {nullptr, nullptr};
    cudaGraphConditionalHandle cond_out[2] = {0, 0}, cond_in[2] = {0, 0};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // new values for the same pattern (ssg_set_values): the input-CSR entry
    // each device value copies (-1: padding)
    int32_t *d_vmap = nullptr, *d_imap = nullptr, *d_smap = nullptr, *d_gmap = nullptr;
    int64_t n_gval = 0;  // interface groups' sliced entries (d_gmap)
    int64_t n_ival = 0, n_sval = 0;
    int32_t *d_growptr = nullptr;  // 7-point grid row pointers (ssg_fv7_*), after the pattern check
    int fv7_dims[3] = {0, 0, 0};
    // several right-hand sides and independent systems together (block.cuh):
    // segments = independent systems (one for a system from ssg_partition)
    DevOp opB64{}, opB32{};  // K-vector product launches (warp ranges cut inside each segment)
    const WorkItem *items_slices = nullptr;  // the item list with interface slices (kind 1)
    bool iface_groups = false;               // op.items holds interface groups (kind 5) instead
    // the K-vector product's entries loaded at once (1 or 2) and L2 look-ahead
    // per precision (0: FP64, 1: FP32) and log2 K - 1 (ssg_autotune_block)
    int8_t spmm_nc[2][4] = {{2, 2, 1, 1}, {2, 2, 2, 2}};
    int8_t spmm_ahead[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    int grid_spmmB = 0;
    int32_t nseg = 1, nchunks = 0;
    std::vector<int32_t> seg_sub, seg_node, seg_nrhs;  // [nseg+1], [nseg+1], [nseg]
    std::vector<int64_t> seg_rhs_off;                  // [nseg]
    int32_t batch_k = 0;       // largest right-hand-side count of a batch (0: not a batch)
    // A batch whose systems need different column counts K is also held as
    // one batch per K class (systems grouped by the power of two >= their
    // right-hand-side count, at least 2), each reading and writing the
    // caller's b and x at the original offsets; the solves run through these.
    std::vector<ssg_system *> kclass;
    std::vector<std::vector<int32_t>> kclass_sys;  // original system indices of each class, ascending
    ssg_ctx *own_ctx = nullptr;    // a class's own context (its own stream), owned by the class
    // a block solve enqueued and not yet finished (solve_block_enqueue)
    ScalB *h_states = nullptr;     // pinned copy of the segment states, nseg + 1
    int64_t pending_launches = 0;
    int pending_k = 0, pending_mode = 0, pending_nr = 0;
    SegTab tab{};              // device copies of the segment tables
    struct BlockGraph {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphConditionalHandle c_out = 0, c_in = 0;
    };
    struct BlockState {
        void *mem = nullptr;  // one allocation for kcap columns
        int kcap = 0;
        double *bl = nullptr, *xl = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
        double *part_a = nullptr, *part_b = nullptr;
        float *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr;
        double *bg = nullptr, *xg = nullptr;  // global staging for ssg_solve_host (n x kcap)
        ScalB *so = nullptr, *si = nullptr;  // [nseg + 1]: one state per segment, then the loop counters
        BlockGraph graph[4][5];  // by mode (SSG_FP64 .. SSG_MIXED_JACOBI) and log2 K
    } blk;
    BlockGraph classes_graph[4];  // per mode: every K class's loop as a parallel branch of one graph
    bool classes_graph_refused[4] = {false, false, false, false};  // building it failed: streams instead
};

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Launch through a kernel pointer (one instance chosen at run time), with
// the arguments converted to the kernel's parameter types.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), int grid, int block, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = nullptr;
    cfg.numAttrs = 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Single-vector SpMV instances ssg_autotune chooses from (launch shape x L2
// prefetch distance); entry 0 is the default, the measured best on the 128^3
// system.
template <typename T>
struct SpmvVariant {
    int bps, ahead;
    void (*part)(DevOp, const T *, T *, double *, Scal *, double *, cudaGraphConditionalHandle, int);
    void (*store)(DevOp, const T *, T *, double *, Scal *, double *, cudaGraphConditionalHandle, int);
};
constexpr int kSpmvVariants = SSG_TUNE_CANDIDATES;
const SpmvVariant<double> kSpmv64Variants[kSpmvVariants] = {
    {4, 0, k_spmv_asm<kEpiPartials, double, 4, 0>, k_spmv_asm<kEpiStore, double, 4, 0>},
    {4, 1, k_spmv_asm<kEpiPartials, double, 4, 1>, k_spmv_asm<kEpiStore, double, 4, 1>},
    {3, 0, k_spmv_asm<kEpiPartials, double, 3, 0>, k_spmv_asm<kEpiStore, double, 3, 0>},
    {3, 1, k_spmv_asm<kEpiPartials, double, 3, 1>, k_spmv_asm<kEpiStore, double, 3, 1>},
    {5, 0, k_spmv_asm<kEpiPartials, double, 5, 0>, k_spmv_asm<kEpiStore, double, 5, 0>},
    {5, 1, k_spmv_asm<kEpiPartials, double, 5, 1>, k_spmv_asm<kEpiStore, double, 5, 1>},
};
// the same instances reading interface groups (systems that use them)
const SpmvVariant<double> kSpmv64VariantsG[kSpmvVariants] = {
    {4, 0, k_spmv_asm<kEpiPartials, double, 4, 0, true>, k_spmv_asm<kEpiStore, double, 4, 0, true>},
    {4, 1, k_spmv_asm<kEpiPartials, double, 4, 1, true>, k_spmv_asm<kEpiStore, double, 4, 1, true>},
    {3, 0, k_spmv_asm<kEpiPartials, double, 3, 0, true>, k_spmv_asm<kEpiStore, double, 3, 0, true>},
    {3, 1, k_spmv_asm<kEpiPartials, double, 3, 1, true>, k_spmv_asm<kEpiStore, double, 3, 1, true>},
    {5, 0, k_spmv_asm<kEpiPartials, double, 5, 0, true>, k_spmv_asm<kEpiStore, double, 5, 0, true>},
    {5, 1, k_spmv_asm<kEpiPartials, double, 5, 1, true>, k_spmv_asm<kEpiStore, double, 5, 1, true>},
};
const SpmvVariant<float> kSpmv32Variants[kSpmvVariants] = {
    {5, 1, k_spmv_asm<kEpiPartials, float, 5, 1>, k_spmv_asm<kEpiStore, float, 5, 1>},
    {5, 0, k_spmv_asm<kEpiPartials, float, 5, 0>, k_spmv_asm<kEpiStore, float, 5, 0>},
    {4, 1, k_spmv_asm<kEpiPartials, float, 4, 1>, k_spmv_asm<kEpiStore, float, 4, 1>},
    {4, 2, k_spmv_asm<kEpiPartials, float, 4, 2>, k_spmv_asm<kEpiStore, float, 4, 2>},
    {6, 1, k_spmv_asm<kEpiPartials, float, 6, 1>, k_spmv_asm<kEpiStore, float, 6, 1>},
    {6, 2, k_spmv_asm<kEpiPartials, float, 6, 2>, k_spmv_asm<kEpiStore, float, 6, 2>},
};

// The FP64 instances a system launches: reading its interface groups, or
// its slices.
const SpmvVariant<double> *v64(const ssg_system *S) { return S->iface_groups ? kSpmv64VariantsG : kSpmv64Variants; }

// SpMV work list (see WorkItem in kernels.cuh) and the sliced-ELL copy of
// the local matrices it streams.  Interior slices: up to 32 consecutive
// interior rows of one subdomain, width = their longest row; a row longer
// than kSliceMaxWidth is an item of its own (read from the CSR arrays).
// Interface slices: whole interface nodes, up to 32 copy rows in (node,
// copy) order; a node with more than 32 copies or a copy row longer than
// kSliceMaxWidth is an item of its own.  The FP64 single-vector product may
// take a second list in which interface groups replace the slices
// (make_plan).
// Padding entries have value 0 and a column inside the same subdomain.
// Interface items are spread evenly among
// the interior ones, and the list is cut into one contiguous slice of about
// equal cost per warp.
struct WorkPlan {
    std::vector<int32_t> irp, icol;  // interface copy rows in CSR form (long nodes)
    std::vector<double> ival;
    std::vector<int32_t> isrc, ssrc;  // local entry each copy-row / sliced value copies (-1: padding)
    std::vector<double> sval;        // sliced-ELL values
    std::vector<int32_t> scol, sseg;
    std::vector<int32_t> gcopy;      // interface groups: per group and copy rank, the 32 lanes' copy rows
    std::vector<double> gval;        // interface groups' sliced values (their own arrays: the slices'
    std::vector<int32_t> gcol, gsrc;  // stay as they are), columns, local entry (-1: padding)
    std::vector<int32_t> srow;       // sorted slices: the local row of each slot
    int64_t slice_slots = 0;         // interior slice entries stored (padding included)
    int64_t slice_entries = 0;       // interior nonzeros in slices
    int32_t sorted_subdomains = 0;   // subdomains whose interior slices are sorted by row length
    int32_t max_window = 1;          // the largest sorting window used
    std::vector<WorkItem> items;
    std::vector<WorkItem> items_g;   // the same with interface groups (empty: the product keeps items)
    int64_t iface_slots = 0;         // interface slice entries stored (padding included)
    int64_t group_slots = 0;         // the same in interface groups
    std::vector<int2> range_bps[7];  // per warp of a single-vector launch sized for 3 to 6 blocks per SM
    std::vector<int2> range_bps32[7];  // the same over the slices' list (the FP32 product)
    std::vector<int2> warp_rangeB;   // per warp of the K-vector product: cut inside each segment
    std::vector<int2> range_cluster;  // per warp of the one-cluster solve (cluster_ctas CTAs)
    int32_t cluster_nranges = 0;      // its non-empty ranges (a prefix)
    std::vector<int32_t> blk_seg, seg_blk;  // segment of each K-vector product block; blocks per segment
    std::vector<int4> chunk;                // vector-kernel chunks (segment, first entry, end entry, 0)
    std::vector<int32_t> seg_chunk;         // chunks per segment
    int grid_bps[7] = {0, 0, 0, 0, 0, 0, 0};
    int grid_bps32[7] = {0, 0, 0, 0, 0, 0, 0};
    int gridB = 0;
};

double item_cost(const WorkItem &w) {
    double cost = 64.0;
    if (sliced_item(w.kind) || w.kind == kItemIfaceGroup) cost += 32.0 * w.e1;
    else cost += 4.0 * (w.e1 - w.e0);
    return cost;
}

// Cut items [lo0, hi0) into one contiguous range of about equal cost per warp
// of `blocks` blocks; the ranges are appended to R (absolute item indices).
void cut_ranges(const std::vector<WorkItem> &items, int lo0, int hi0, int blocks, std::vector<int2> &R) {
    const int n = hi0 - lo0;
    const int G = blocks * kSpmvWarps;
    std::vector<double> prefix(static_cast<size_t>(n) + 1, 0.0);
    for (int i = 0; i < n; ++i) prefix[i + 1] = prefix[i] + item_cost(items[lo0 + i]);
    int lo = 0;
    for (int b = 0; b < G; ++b) {
        const double target = prefix[n] * (b + 1) / G;
        int hi = lo;
        while (hi < n && (prefix[hi + 1] <= target || hi == lo)) ++hi;
        if (b == G - 1) hi = n;
        R.push_back(make_int2(lo0 + lo, lo0 + hi));
        lo = hi;
    }
}

std::vector<int2> cut_ranges(const std::vector<WorkItem> &items, int blocks) {
    std::vector<int2> R;
    cut_ranges(items, 0, static_cast<int>(items.size()), blocks, R);
    return R;
}

// Interior slice entries stored for rows lens[0..n) (runs of rows no longer
// than kSliceMaxWidth) cut into windows of `win` rows sorted by decreasing
// length, 32 rows per slice (win <= 1: no sorting).
int64_t slice_slots_for(const std::vector<int32_t> &lens, int win) {
    int64_t slots = 0;
    const int n = static_cast<int>(lens.size());
    const int step = win <= 1 ? n : win;
    std::vector<int32_t> w;
    for (int w0 = 0; w0 < n; w0 += std::max(step, 1)) {
        w.assign(lens.begin() + w0, lens.begin() + std::min(n, w0 + std::max(step, 1)));
        if (win > 1) std::stable_sort(w.begin(), w.end(), [](int32_t x, int32_t y) { return x > y; });
        for (size_t i = 0; i < w.size(); i += kSliceRows)
            slots += static_cast<int64_t>(kSliceRows) *
                     *std::max_element(w.begin() + i, w.begin() + std::min(w.size(), i + kSliceRows));
    }
    return slots;
}

// Sorting window of subdomain s's interior rows.  policy: 1 = none, > 1 = a
// window of that many rows, -1 = the whole subdomain, 0 = chosen from the
// row lengths: the window of {1, 128, 256, 512} rows whose slices move the
// fewest bytes, counting 12 bytes per stored entry (value and column) and,
// for a sorted layout, 4 bytes per row for its row index; sorting is taken
// only when it saves at least 2 % (its row indices scatter the stores).
// Windows of at most 512 rows keep each slice's column gathers within a few
// grid lines of the subdomain.
int slice_window(const HostMaps &M, int32_t s, int policy) {
    if (policy == 1) return 1;
    if (policy == -1) return std::max<int32_t>(M.nint[s], 2);
    if (policy > 1) return policy;
    std::vector<int32_t> lens;
    for (int64_t r = M.off[s]; r < M.off[s] + M.nint[s]; ++r) {
        const int32_t L = M.lrowptr[r + 1] - M.lrowptr[r];
        if (L <= kSliceMaxWidth) lens.push_back(L);
    }
    const double base = 12.0 * static_cast<double>(slice_slots_for(lens, 1));
    int best = 1;
    double best_bytes = base;
    for (int win : {128, 256, 512}) {
        const double b = 12.0 * static_cast<double>(slice_slots_for(lens, win)) + 4.0 * lens.size();
        if (b < best_bytes) {
            best = win;
            best_bytes = b;
        }
    }
    return best_bytes <= 0.98 * base ? best : 1;
}

// CTAs per cluster of a system's one-cluster solve: the count asked for on
// the context, else the most the device places.
int cluster_ctas_for(const ssg_ctx *C) {
    if (C->cluster_ctas <= 0) return 0;
    return C->cluster_ctas_set > 0 ? std::min(C->cluster_ctas_set, C->cluster_ctas) : C->cluster_ctas;
}

// seg_sub: subdomains of each segment (independent systems), [nseg + 1];
// sort_policy: the sorting window of the interior slices (slice_window).
WorkPlan make_plan(const HostMaps &M, int num_sms, const std::vector<int32_t> &seg_sub, int sort_policy,
                   int cluster_ctas) {
    WorkPlan W;
    std::vector<int32_t> sub_of(static_cast<size_t>(M.nloc));
    for (int32_t s = 0; s < M.P; ++s)
        for (int64_t r = M.off[s]; r < M.off[s + 1]; ++r) sub_of[r] = s;
    auto rlen = [&](int32_t r) { return M.lrowptr[r + 1] - M.lrowptr[r]; };
    // interface copy rows in (node, copy) order, columns as concatenated index
    W.irp.assign(static_cast<size_t>(M.ncopies) + 1, 0);
    for (int64_t c = 0; c < M.ncopies; ++c) {
        const int32_t row = M.icopy[c];
        const int32_t o = M.off[sub_of[row]];
        for (int32_t k = M.lrowptr[row]; k < M.lrowptr[row + 1]; ++k) {
            W.icol.push_back(o + M.lcol[k]);
            W.ival.push_back(M.lval[k]);
            W.isrc.push_back(k);
        }
        W.irp[c + 1] = static_cast<int32_t>(W.icol.size());
    }
    W.sseg.assign(static_cast<size_t>(M.ncopies), 0);
    std::vector<WorkItem> rows, iface;
    // interior slices: the rows no longer than kSliceMaxWidth, in runs
    // between long rows; unsorted (window 1), a slice is 32 consecutive rows
    // of a run; sorted, each window of a run is ordered by decreasing row
    // length (ties in row order) and sliced 32 rows at a time, so that short
    // rows stop padding to a long neighbour's width (SELL-C-sigma); its lanes
    // find their rows in srow.  Padding entries: value 0, a column of the
    // same subdomain.
    std::vector<int32_t> order;
    auto emit_slice = [&](const int32_t *rws, int32_t cnt, int32_t o, bool sorted) {
        int32_t w = 0;
        for (int32_t i = 0; i < cnt; ++i) w = std::max(w, rlen(rws[i]));
        const int32_t off = static_cast<int32_t>(W.sval.size());
        for (int32_t k = 0; k < w; ++k)
            for (int32_t lane = 0; lane < kSliceRows; ++lane) {
                const int32_t row = lane < cnt ? rws[lane] : rws[0];
                if (lane < cnt && k < rlen(row)) {
                    const int32_t e = M.lrowptr[row] + k;
                    W.sval.push_back(M.lval[e]);
                    W.scol.push_back(o + M.lcol[e]);
                    W.ssrc.push_back(e);
                    W.slice_entries++;
                } else {
                    W.sval.push_back(0.0);
                    W.scol.push_back(row);
                    W.ssrc.push_back(-1);
                }
            }
        W.slice_slots += static_cast<int64_t>(w) * kSliceRows;
        if (sorted) {
            const int32_t slot0 = static_cast<int32_t>(W.srow.size());
            W.srow.insert(W.srow.end(), rws, rws + cnt);
            rows.push_back({kItemSortedSlice, slot0, slot0 + cnt, off, w, 0, 0, 0});
        } else {
            rows.push_back({kItemSlice, rws[0], rws[0] + cnt, off, w, 0, 0, 0});
        }
    };
    for (int32_t s = 0; s < M.P; ++s) {
        int32_t r = M.off[s];
        const int32_t rend = M.off[s] + M.nint[s];
        const int32_t o = M.off[s];
        const int win = slice_window(M, s, sort_policy);
        if (win > 1 && rend > r) {
            W.sorted_subdomains++;
            W.max_window = std::max(W.max_window, win);
        }
        while (r < rend) {
            if (rlen(r) > kSliceMaxWidth) {
                rows.push_back({kItemLongRow, r, r + 1, M.lrowptr[r], M.lrowptr[r + 1], 0, 0, 0});
                ++r;
                continue;
            }
            int32_t r1 = r;
            while (r1 < rend && rlen(r1) <= kSliceMaxWidth) ++r1;
            const int32_t step = win > 1 ? win : kSliceRows;
            for (int32_t w0 = r; w0 < r1; w0 += step) {
                const int32_t w1 = std::min(r1, w0 + step);
                order.resize(static_cast<size_t>(w1 - w0));
                for (int32_t i = w0; i < w1; ++i) order[i - w0] = i;
                if (win > 1)
                    std::stable_sort(order.begin(), order.end(),
                                     [&](int32_t x, int32_t y) { return rlen(x) > rlen(y); });
                for (int32_t i = 0; i < w1 - w0; i += kSliceRows)
                    emit_slice(order.data() + i, std::min<int32_t>(kSliceRows, w1 - w0 - i), o, win > 1);
            }
            r = r1;
        }
    }
    // segments (independent systems): every item stays inside one
    const int nseg = static_cast<int>(seg_sub.size()) - 1;
    std::vector<int32_t> seg_of_sub(static_cast<size_t>(M.P), 0);
    for (int sg = 0; sg < nseg; ++sg)
        for (int32_t sd = seg_sub[sg]; sd < seg_sub[sg + 1]; ++sd) seg_of_sub[sd] = sg;
    auto node_seg = [&](int32_t gg) { return seg_of_sub[sub_of[M.icopy[M.iptr[gg]]]]; };
    // interface slices (whole nodes, one segment)
    int32_t g = 0;
    while (g < M.ngamma) {
        auto long_node = [&](int32_t gg) {
            if (M.iptr[gg + 1] - M.iptr[gg] > kSliceRows) return true;
            for (int32_t c = M.iptr[gg]; c < M.iptr[gg + 1]; ++c)
                if (W.irp[c + 1] - W.irp[c] > kSliceMaxWidth) return true;
            return false;
        };
        if (long_node(g)) {
            const int32_t c0 = M.iptr[g], c1 = M.iptr[g + 1];
            iface.push_back({kItemLongIface, g, g + 1, W.irp[c0], W.irp[c1], c0, c1, 0});
            ++g;
            continue;
        }
        const int32_t c0 = M.iptr[g];
        int32_t g1 = g, w = 0;
        while (g1 < M.ngamma && !long_node(g1) && M.iptr[g1 + 1] - c0 <= kSliceRows && node_seg(g1) == node_seg(g)) {
            for (int32_t c = M.iptr[g1]; c < M.iptr[g1 + 1]; ++c) w = std::max(w, W.irp[c + 1] - W.irp[c]);
            ++g1;
        }
        const int32_t c1 = M.iptr[g1];
        for (int32_t gg = g; gg < g1; ++gg)
            for (int32_t c = M.iptr[gg]; c < M.iptr[gg + 1]; ++c)
                W.sseg[c] = (M.iptr[gg] - c0) | ((M.iptr[gg + 1] - M.iptr[gg]) << 8);
        const int32_t off = static_cast<int32_t>(W.sval.size());
        for (int32_t k = 0; k < w; ++k)
            for (int32_t lane = 0; lane < kSliceRows; ++lane) {
                const int32_t c = c0 + lane;
                if (c < c1 && k < W.irp[c + 1] - W.irp[c]) {
                    W.sval.push_back(W.ival[W.irp[c] + k]);
                    W.scol.push_back(W.icol[W.irp[c] + k]);
                    W.ssrc.push_back(W.isrc[W.irp[c] + k]);
                } else {
                    W.sval.push_back(0.0);
                    W.scol.push_back(M.icopy[c < c1 ? c : c0]);
                    W.ssrc.push_back(-1);
                }
            }
        iface.push_back({kItemIfaceSlice, c0, c1, off, w, 0, 0, 0});
        W.iface_slots += static_cast<int64_t>(w) * kSliceRows;
        g = g1;
    }
    // interface groups (kind 5), for the FP64 single-vector product only: a
    // node with more than kGroupMaxCopies copies or a copy row longer than
    // kSliceMaxWidth is an item of its own (kind 3); the others go in groups
    // of up to 32 nodes of one multiplicity m, one node per lane, per
    // segment.  A group's data holds m sub-slices, the r-th with the r-th
    // copy rows of its nodes at the width of the longest, so that a node's
    // copies meet in one lane and a short copy row (a node's copies in the
    // lower subdomains hold only the entries those own: one on the faces of
    // the 7-point grids) never pads to a long one's width.  Within windows
    // of kGroupWindow nodes of one multiplicity the nodes are ordered by
    // decreasing copy-row lengths (rank 0 first; ties in node order).  The
    // groups are built, and the product takes them, only when they store at
    // least kGroupGain of all the product's sliced entries fewer than the
    // slices (measured on the 128^3 system, where they save 4.9 %: the FP64
    // product 2 % and the FP64 solve 3 % faster; on the P1 mesh, 2.6 %: no
    // gain.  The FP32 products, the K-vector products and the one-cluster
    // solve, no faster or slower with them, keep the slices)
    std::vector<WorkItem> iface_g;
    constexpr double kGroupGain = 0.04;
    for (int pass = 0; pass < 2; ++pass) {
        const bool emit = pass == 1;
        if (emit && !(W.iface_slots > W.group_slots &&
                      static_cast<double>(W.iface_slots - W.group_slots) >=
                          kGroupGain * static_cast<double>(W.slice_slots + W.iface_slots)))
            break;
        constexpr size_t kGroupWindow = 512;
        auto clen = [&](int32_t c) { return W.irp[c + 1] - W.irp[c]; };
        auto long_node_g = [&](int32_t gg) {
            if (M.iptr[gg + 1] - M.iptr[gg] > kGroupMaxCopies) return true;
            for (int32_t c = M.iptr[gg]; c < M.iptr[gg + 1]; ++c)
                if (clen(c) > kSliceMaxWidth) return true;
            return false;
        };
        std::vector<int32_t> by_mult[kGroupMaxCopies + 1];
        g = 0;
        while (g < M.ngamma) {
            const int sg = node_seg(g);
            int32_t g1 = g;
            while (g1 < M.ngamma && node_seg(g1) == sg) ++g1;
            for (std::vector<int32_t> &v : by_mult) v.clear();
            for (int32_t gg = g; gg < g1; ++gg) {
                if (long_node_g(gg)) {
                    const int32_t c0 = M.iptr[gg], c1 = M.iptr[gg + 1];
                    if (emit) iface_g.push_back({kItemLongIface, gg, gg + 1, W.irp[c0], W.irp[c1], c0, c1, 0});
                } else {
                    by_mult[M.iptr[gg + 1] - M.iptr[gg]].push_back(gg);
                }
            }
            for (int m = 1; m <= kGroupMaxCopies; ++m) {
                std::vector<int32_t> &nodes = by_mult[m];
                for (size_t w0 = 0; w0 < nodes.size(); w0 += kGroupWindow) {
                    const size_t w1 = std::min(nodes.size(), w0 + kGroupWindow);
                    std::stable_sort(nodes.begin() + w0, nodes.begin() + w1, [&](int32_t x, int32_t y) {
                        for (int r = 0; r < m; ++r) {
                            const int32_t lx = clen(M.iptr[x] + r), ly = clen(M.iptr[y] + r);
                            if (lx != ly) return lx > ly;
                        }
                        return false;
                    });
                }
                for (size_t i0 = 0; i0 < nodes.size(); i0 += kSliceRows) {
                    if (!emit) {
                        for (int r = 0; r < m; ++r) {
                            int32_t w = 0;
                            for (size_t l = i0; l < std::min(nodes.size(), i0 + kSliceRows); ++l)
                                w = std::max(w, clen(M.iptr[nodes[l]] + r));
                            W.group_slots += static_cast<int64_t>(w) * kSliceRows;
                        }
                        continue;
                    }
                    const int cnt = static_cast<int>(std::min<size_t>(kSliceRows, nodes.size() - i0));
                    const int32_t *nd = nodes.data() + i0;
                    auto copy_of = [&](int lane, int r) { return M.iptr[nd[lane < cnt ? lane : 0]] + r; };
                    const int32_t a = static_cast<int32_t>(W.gcopy.size());
                    const int32_t off = static_cast<int32_t>(W.gval.size());
                    int32_t wsum = 0;
                    uint32_t wpack[2] = {0u, 0u};
                    for (int r = 0; r < m; ++r) {
                        int32_t w = 0;
                        for (int l = 0; l < cnt; ++l) w = std::max(w, clen(copy_of(l, r)));
                        wpack[r >> 2] |= static_cast<uint32_t>(w) << (8 * (r & 3));
                        wsum += w;
                        for (int l = 0; l < kSliceRows; ++l) W.gcopy.push_back(M.icopy[copy_of(l, r)]);
                        for (int32_t k = 0; k < w; ++k)
                            for (int l = 0; l < kSliceRows; ++l) {
                                const int32_t c = copy_of(l, r);
                                if (l < cnt && k < clen(c)) {
                                    W.gval.push_back(W.ival[W.irp[c] + k]);
                                    W.gcol.push_back(W.icol[W.irp[c] + k]);
                                    W.gsrc.push_back(W.isrc[W.irp[c] + k]);
                                } else {
                                    W.gval.push_back(0.0);
                                    W.gcol.push_back(M.icopy[c]);
                                    W.gsrc.push_back(-1);
                                }
                            }
                    }
                    iface_g.push_back({kItemIfaceGroup, a, cnt, off, wsum, m, static_cast<int32_t>(wpack[0]),
                                     static_cast<int32_t>(wpack[1])});
                }
            }
            g = g1;
        }
    }
    // per segment, interface item j goes after interior item floor((j+1) *
    // nrows / (niface+1)) of the segment
    auto item_seg = [&](const WorkItem &w) {
        if (w.kind == kItemSlice || w.kind == kItemLongRow) return seg_of_sub[sub_of[w.a]];
        if (w.kind == kItemSortedSlice) return seg_of_sub[sub_of[W.srow[w.a]]];
        if (w.kind == kItemIfaceGroup) return seg_of_sub[sub_of[W.gcopy[w.a]]];
        const int32_t c = w.kind == kItemIfaceSlice ? w.a : w.c0;
        return seg_of_sub[sub_of[M.icopy[c]]];
    };
    std::vector<int32_t> seg_item(static_cast<size_t>(nseg) + 1, 0);
    auto interleave = [&](const std::vector<WorkItem> &ifc, std::vector<WorkItem> &out) {
        size_t ir = 0, ii = 0;
        for (int sg = 0; sg < nseg; ++sg) {
            size_t r0 = ir, i0 = ii;
            while (ir < rows.size() && item_seg(rows[ir]) == sg) ++ir;
            while (ii < ifc.size() && item_seg(ifc[ii]) == sg) ++ii;
            const size_t nr = ir - r0, ni = ii - i0;
            size_t j = 0;
            for (size_t i = 0; i <= nr; ++i) {
                while (j < ni && (j + 1) * nr <= i * (ni + 1)) out.push_back(ifc[i0 + j++]);
                if (i < nr) out.push_back(rows[r0 + i]);
            }
            while (j < ni) out.push_back(ifc[i0 + j++]);
            seg_item[sg + 1] = static_cast<int32_t>(out.size());
        }
    };
    if (!iface_g.empty()) interleave(iface_g, W.items_g);
    interleave(iface, W.items);  // last: seg_item is this list's
    // single-vector launches: FP64 the list with interface groups when
    // built, FP32 the slices (latency-bound, it gains nothing from them:
    // measured slower on the 96^3 system)
    for (int prec = 0; prec < 2; ++prec) {
        const std::vector<WorkItem> &items1 = prec == 0 && !W.items_g.empty() ? W.items_g : W.items;
        const int per = (static_cast<int>(items1.size()) + kSpmvWarps - 1) / kSpmvWarps;
        for (int bps = 3; bps <= 6; ++bps) {
            int &grid = prec == 0 ? W.grid_bps[bps] : W.grid_bps32[bps];
            grid = std::max(1, std::min(per, num_sms * bps));
            (prec == 0 ? W.range_bps[bps] : W.range_bps32[bps]) = cut_ranges(items1, grid);
        }
    }
    if (cluster_ctas > 0) {
        // kClusterWarps warps per CTA: cut for the equivalent number of
        // kSpmvWarps-warp blocks
        W.range_cluster = cut_ranges(W.items, cluster_ctas * kClusterWarps / kSpmvWarps);
        for (const int2 &r : W.range_cluster) W.cluster_nranges += r.y > r.x ? 1 : 0;
    }
    // K-vector product: blocks shared out among the segments by cost, at
    // least one each, every block inside one segment
    std::vector<double> seg_cost(static_cast<size_t>(nseg), 0.0);
    double total = 0.0;
    for (int sg = 0; sg < nseg; ++sg) {
        for (int i = seg_item[sg]; i < seg_item[sg + 1]; ++i) seg_cost[sg] += item_cost(W.items[i]);
        total += seg_cost[sg];
    }
    constexpr int kSpmmBlocks = SpmmTraits<double>::kBlocksPerSM > SpmmTraits<float>::kBlocksPerSM
                                    ? SpmmTraits<double>::kBlocksPerSM
                                    : SpmmTraits<float>::kBlocksPerSM;
    const int perB = (static_cast<int>(W.items.size()) + kSpmvWarps - 1) / kSpmvWarps;
    const int target = std::max(1, std::min(perB, num_sms * kSpmmBlocks * (nseg > 1 ? 4 : 1)));
    W.seg_blk.assign(static_cast<size_t>(nseg) + 1, 0);
    for (int sg = 0; sg < nseg; ++sg) {
        const int nit = seg_item[sg + 1] - seg_item[sg];
        int gs = nseg == 1 ? target
                           : static_cast<int>(std::floor(target * (total > 0 ? seg_cost[sg] / total : 0.0) + 0.5));
        gs = std::max(1, std::min(gs, std::max(1, (nit + kSpmvWarps - 1) / kSpmvWarps)));
        cut_ranges(W.items, seg_item[sg], seg_item[sg + 1], gs, W.warp_rangeB);
        for (int b = 0; b < gs; ++b) W.blk_seg.push_back(sg);
        W.seg_blk[sg + 1] = W.seg_blk[sg] + gs;
    }
    W.gridB = W.seg_blk[nseg];
    // vector-kernel chunks: about one per SM in all for one system (every
    // chunk's block sums the system's product partials per column), four for
    // a batch (a large system then spreads over more SMs once the small ones
    // have converged); a multiple of 64 entries, at least one per segment
    const int per_sm = nseg > 1 ? 4 : 1;
    const int64_t ch = std::max<int64_t>(64, (M.nloc / (num_sms * per_sm) + 63) / 64 * 64);
    W.seg_chunk.assign(static_cast<size_t>(nseg) + 1, 0);
    for (int sg = 0; sg < nseg; ++sg) {
        const int64_t e0 = M.off[seg_sub[sg]], e1 = M.off[seg_sub[sg + 1]];
        for (int64_t e = e0; e < e1; e += ch)
            W.chunk.push_back(make_int4(sg, static_cast<int>(e), static_cast<int>(std::min(e + ch, e1)), 0));
        if (e1 == e0) W.chunk.push_back(make_int4(sg, static_cast<int>(e0), static_cast<int>(e0), 0));
        W.seg_chunk[sg + 1] = static_cast<int32_t>(W.chunk.size());
    }
    return W;
}

// Partials of the loop reductions, three slots of n_partials / 3: the SpMV
// writes (p, S p)_w, the residual update (r, r)_w and, with the diagonal
// preconditioner, (r, z)_w; each is read by the next kernel.
double *part_pq(ssg_system *S) { return S->d_partials; }
double *part_rr(ssg_system *S) { return S->d_partials + S->n_partials / 3; }
double *part_rz(ssg_system *S) { return S->d_partials + 2 * (S->n_partials / 3); }

int launch_body(ssg_system *S, cudaStream_t st, int use_cond, bool pc) {
    const int64_t N = S->maps.nloc;
    const cudaGraphConditionalHandle h = pc ? S->cond_pc : S->cond;
    SSG_CUDA_TRY(launch_k(v64(S)[S->var64].part, S->grid_spmv, kSpmvThreads, st, S->op, S->d_p,
                          S->d_q, part_pq(S), S->d_scal, (double *)nullptr, h, use_cond));
    SSG_CUDA_TRY(launch_k(pc ? k_update_r<true> : k_update_r<false>, S->grid_vec, kBlock, st, N, S->d_r,
                          S->d_q, S->op.mult, S->op.wtab, S->op.gflag, (const double *)part_pq(S), S->grid_spmv,
                          part_rr(S), S->d_scal, h, use_cond, (const double *)S->d_dinv, part_rz(S)));
    SSG_CUDA_TRY(launch_k(pc ? k_update_xp<true> : k_update_xp<false>, S->grid_vec, kBlock, st, N, S->d_xl,
                          S->d_p, S->d_r, (const double *)part_rr(S), S->grid_vec, S->d_scal, h, use_cond,
                          (const double *)S->d_dinv, (const double *)part_rz(S)));
    return SSG_OK;
}

int launch_init(ssg_system *S, cudaStream_t st, int use_cond, bool pc) {
    const cudaGraphConditionalHandle h = pc ? S->cond_pc : S->cond;
    if (pc)
        k_cg_init<true><<<S->grid_vec, kBlock, 0, st>>>(S->maps.nloc, S->d_bl, S->d_q, S->d_r, S->d_p, S->op.mult,
                                                        S->op.wtab, S->d_partials, S->d_scal, h, use_cond, S->d_dinv);
    else
        k_cg_init<false><<<S->grid_vec, kBlock, 0, st>>>(S->maps.nloc, S->d_bl, S->d_q, S->d_r, S->d_p, S->op.mult,
                                                         S->op.wtab, S->d_partials, S->d_scal, h, use_cond, nullptr);
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

int launch_mixed_init(ssg_system *S, cudaStream_t st, int use_cond, bool pc) {
    k_cg_init<false><<<S->grid_vec, kBlock, 0, st>>>(S->maps.nloc, S->d_bl, S->d_q, S->d_r, nullptr, S->op.mult,
                                                     S->op.wtab, S->d_partials, S->d_scal, S->cond_out[pc], use_cond,
                                                     nullptr);
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

int launch_inner_init(ssg_system *S, cudaStream_t st, int use_cond, bool pc) {
    auto kern = pc ? k_inner_init<true> : k_inner_init<false>;
    kern<<<S->grid_vec, kBlock, 0, st>>>(S->maps.nloc, S->d_r, S->d_r32, S->d_p32, S->d_d32, S->op.mult, S->op.wtab32,
                                         S->d_partials, S->d_scal_in, S->d_scal, S->cond_in[pc], use_cond,
                                         S->d_dinv32);
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

int launch_inner_body(ssg_system *S, cudaStream_t st, int use_cond, bool pc) {
    const int64_t N = S->maps.nloc;
    const cudaGraphConditionalHandle h = S->cond_in[pc];
    SSG_CUDA_TRY(launch_k(kSpmv32Variants[S->var32].part, S->grid_spmv32, kSpmvThreads, st, S->op32,
                          S->d_p32, S->d_q32, part_pq(S), S->d_scal_in, (double *)nullptr, h, use_cond));
    SSG_CUDA_TRY(launch_k(pc ? k_update_r32<true> : k_update_r32<false>, S->grid_vec, kBlock, st, N,
                          S->d_r32, S->d_q32, S->op.mult, S->op.wtab32, S->op.gflag128, (const double *)part_pq(S),
                          S->grid_spmv32, part_rr(S), S->d_scal_in, S->d_scal, h, use_cond,
                          (const float *)S->d_dinv32, part_rz(S)));
    SSG_CUDA_TRY(launch_k(pc ? k_update_dp32<true> : k_update_dp32<false>, S->grid_vec, kBlock, st, N,
                          S->d_d32, S->d_p32, S->d_r32, (const double *)part_rr(S), S->grid_vec, S->d_scal_in,
                          S->d_scal, h, use_cond, (const float *)S->d_dinv32, (const double *)part_rz(S)));
    return SSG_OK;
}

int launch_outer_tail(ssg_system *S, cudaStream_t st, int use_cond, bool pc) {
    const int64_t N = S->maps.nloc;
    k_ir_correct<<<S->grid_vec, kBlock, 0, st>>>(N, S->d_xl, S->d_d32);
    v64(S)[S->var64].store<<<S->grid_spmv, kSpmvThreads, 0, st>>>(
        S->op, S->d_xl, S->d_q, S->d_partials, S->d_scal_op, nullptr, 0, 0);
    k_ir_residual<<<S->grid_vec, kBlock, 0, st>>>(N, S->d_bl, S->d_q, S->d_r, S->op.mult, S->op.wtab, S->d_partials,
                                                  S->d_scal, S->d_scal_in, S->cond_out[pc], use_cond);
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

// Capture `fn` into `g` after `deps`; returns the nodes `g` holds afterwards
// that have no dependents (the capture's sink).
template <typename F>
cudaError_t capture_into(cudaStream_t cap, cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, F fn, int *rc) {
    cudaError_t e = cudaStreamBeginCaptureToGraph(cap, g, deps, nullptr, ndeps, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    *rc = fn(cap);
    cudaGraph_t out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &out);
    return e2;
}

cudaError_t last_node(cudaGraph_t g, cudaGraphNode_t *out) {
    size_t nn = 0;
    cudaError_t e = cudaGraphGetNodes(g, nullptr, &nn);
    if (e != cudaSuccess) return e;
    std::vector<cudaGraphNode_t> nodes(nn);
    e = cudaGraphGetNodes(g, nodes.data(), &nn);
    if (e != cudaSuccess) return e;
    for (cudaGraphNode_t n : nodes) {
        size_t nd = 0;
        e = cudaGraphNodeGetDependentNodes(n, nullptr, nullptr, &nd);
        if (e != cudaSuccess) return e;
        if (nd == 0) {
            *out = n;
            return cudaSuccess;
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t add_while(cudaGraph_t g, const cudaGraphNode_t *dep, cudaGraphConditionalHandle h, cudaGraphNode_t *node,
                      cudaGraph_t *body) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaError_t e = cudaGraphAddNode(node, g, dep, nullptr, dep ? 1 : 0, &cp);
    if (e == cudaSuccess) *body = cp.conditional.phGraph_out[0];
    return e;
}

// Build the FP64 graph (with or without the diagonal preconditioner).
int build_graph(ssg_system *S, bool pc) {
    if (pc ? S->exec_pc : S->exec) return SSG_OK;
    cudaGraph_t &graph = pc ? S->graph_pc : S->graph;
    cudaGraphExec_t &exec = pc ? S->exec_pc : S->exec;
    cudaGraphConditionalHandle &cond = pc ? S->cond_pc : S->cond;
    SSG_CUDA_TRY(cudaGraphCreate(&graph, 0));
    SSG_CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, graph, 0u, cudaGraphCondAssignDefault));
    cudaStream_t cap;
    SSG_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    int rc = SSG_OK;
    cudaGraphNode_t init_node = nullptr, loop_node = nullptr;
    cudaGraph_t body = nullptr;
    cudaError_t e = capture_into(cap, graph, nullptr, 0, [&](cudaStream_t c) { return launch_init(S, c, 1, pc); }, &rc);
    if (e == cudaSuccess && rc == SSG_OK) e = last_node(graph, &init_node);
    if (e == cudaSuccess && rc == SSG_OK) e = add_while(graph, &init_node, cond, &loop_node, &body);
    if (e == cudaSuccess && rc == SSG_OK)
        e = capture_into(cap, body, nullptr, 0, [&](cudaStream_t c) {
                int r = SSG_OK;
                for (int u = 0; u < S->unroll && r == SSG_OK; ++u) r = launch_body(S, c, 1, pc);
                return r;
            }, &rc);
    if (e == cudaSuccess && rc == SSG_OK) e = cudaGraphInstantiate(&exec, graph, 0);
    cudaStreamDestroy(cap);
    if (rc != SSG_OK) return rc;
    if (e != cudaSuccess) {
        set_error(std::string("building the CG graph: ") + cudaGetErrorString(e));
        if (graph) cudaGraphDestroy(graph);
        graph = nullptr;
        exec = nullptr;
        return SSG_E_CUDA;
    }
    return SSG_OK;
}


// SSG_MIXED graph: init -> WHILE(outer) { inner_init -> WHILE(inner) { FP32
// SpMV, r update, d/p update } -> x += d -> FP64 SpMV -> residual + test }.
int build_graph_mixed(ssg_system *S, bool pc) {
    if (S->exec_m[pc]) return SSG_OK;
    cudaGraph_t &gm = S->graph_m[pc];
    SSG_CUDA_TRY(cudaGraphCreate(&gm, 0));
    SSG_CUDA_TRY(cudaGraphConditionalHandleCreate(&S->cond_out[pc], gm, 0u, cudaGraphCondAssignDefault));
    cudaStream_t cap;
    SSG_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    int rc = SSG_OK;
    cudaError_t e =
        capture_into(cap, gm, nullptr, 0, [&](cudaStream_t c) { return launch_mixed_init(S, c, 1, pc); }, &rc);
    cudaGraphNode_t n_init = nullptr, n_outer = nullptr, n_iinit = nullptr, n_inner = nullptr;
    cudaGraph_t body_out = nullptr, body_in = nullptr;
    if (e == cudaSuccess && rc == SSG_OK) e = last_node(gm, &n_init);
    if (e == cudaSuccess && rc == SSG_OK) e = add_while(gm, &n_init, S->cond_out[pc], &n_outer, &body_out);
    // the inner handle must exist before the kernels that set it are captured
    if (e == cudaSuccess && rc == SSG_OK)
        e = cudaGraphConditionalHandleCreate(&S->cond_in[pc], body_out, 0u, cudaGraphCondAssignDefault);
    if (e == cudaSuccess && rc == SSG_OK)
        e = capture_into(cap, body_out, nullptr, 0, [&](cudaStream_t c) { return launch_inner_init(S, c, 1, pc); },
                         &rc);
    if (e == cudaSuccess && rc == SSG_OK) e = last_node(body_out, &n_iinit);
    if (e == cudaSuccess && rc == SSG_OK) e = add_while(body_out, &n_iinit, S->cond_in[pc], &n_inner, &body_in);
    if (e == cudaSuccess && rc == SSG_OK)
        e = capture_into(cap, body_in, nullptr, 0, [&](cudaStream_t c) {
                int r = SSG_OK;
                for (int u = 0; u < S->unroll && r == SSG_OK; ++u) r = launch_inner_body(S, c, 1, pc);
                return r;
            },
                         &rc);
    if (e == cudaSuccess && rc == SSG_OK)
        e = capture_into(cap, body_out, &n_inner, 1,
                         [&](cudaStream_t c) { return launch_outer_tail(S, c, 1, pc); }, &rc);
    if (e == cudaSuccess && rc == SSG_OK) e = cudaGraphInstantiate(&S->exec_m[pc], gm, 0);
    cudaStreamDestroy(cap);
    if (rc != SSG_OK) return rc;
    if (e != cudaSuccess) {
        set_error(std::string("building the mixed-precision graph: ") + cudaGetErrorString(e));
        if (gm) cudaGraphDestroy(gm);
        gm = nullptr;
        S->exec_m[pc] = nullptr;
        return SSG_E_CUDA;
    }
    return SSG_OK;
}

int grid_for(int64_t n, int num_sms) {
    return std::max(1, std::min<int>(static_cast<int>((n + kBlock - 1) / kBlock), num_sms * 8));
}

int upload(ssg_system *S) {
    const HostMaps &M = S->maps;
    ssg_ctx *C = S->ctx;
    SSG_CUDA_TRY(cudaSetDevice(C->device));
    if (S->seg_sub.empty()) {
        S->seg_sub = {0, M.P};
        S->seg_node = {0, M.n};
        S->seg_nrhs = {1};
        S->seg_rhs_off = {0};
    }
    S->nseg = static_cast<int32_t>(S->seg_sub.size()) - 1;
    const int cl_ctas = S->nseg == 1 ? cluster_ctas_for(C) : 0;
    WorkPlan plan = make_plan(M, C->num_sms, S->seg_sub, C->slice_sort, cl_ctas);
    S->slice_slots = plan.slice_slots;
    S->slice_entries = plan.slice_entries;
    S->sorted_subdomains = plan.sorted_subdomains;
    S->max_window = plan.max_window;
    S->iface_slots = plan.iface_slots;
    S->group_slots = plan.group_slots;
    const int64_t N = M.nloc;
    // concatenated column ids
    std::vector<int32_t> gcol(static_cast<size_t>(M.nnz));
    for (int32_t s = 0; s < M.P; ++s)
        for (int64_t r = M.off[s]; r < M.off[s + 1]; ++r)
            for (int32_t k = M.lrowptr[r]; k < M.lrowptr[r + 1]; ++k) gcol[k] = M.off[s] + M.lcol[k];
    std::vector<uint8_t> mloc(static_cast<size_t>(N));
    for (int64_t k = 0; k < N; ++k) mloc[k] = static_cast<uint8_t>(M.mult[M.l2g[k]]);
    // owner-mask weight codes (ssg_set_weights): 1 on a node's owner copy
    // (every interior entry is one), 0 on its other copies
    std::vector<uint8_t> wown(static_cast<size_t>(N), 0);
    for (int32_t i = 0; i < M.n; ++i) wown[M.own[i]] = 1;
    // group flags: 1 when any of the 64 entries of a group is an interface copy
    std::vector<uint8_t> gflag(static_cast<size_t>((N + 63) / 64), 0);
    for (int64_t k = 0; k < N; ++k)
        if (mloc[k] > 1) gflag[k >> 6] = 1;
    std::vector<uint8_t> gflag128(static_cast<size_t>((N + 127) / 128), 0);
    for (int64_t k = 0; k < N; ++k)
        if (mloc[k] > 1) gflag128[k >> 7] = 1;
    std::vector<double> wtab(256, 0.0);
    std::vector<float> wtab32(256, 0.f);
    for (int m = 1; m < 256; ++m) {
        wtab[m] = 1.0 / static_cast<double>(m);
        wtab32[m] = static_cast<float>(wtab[m]);
    }

    for (int bps = 3; bps <= 6; ++bps) {
        S->grid_bps[bps] = plan.grid_bps[bps];
        S->grid_bps32[bps] = plan.grid_bps32[bps];
    }
    S->grid_spmv = plan.grid_bps[kSpmv64Variants[0].bps];
    S->grid_spmv32 = plan.grid_bps32[kSpmv32Variants[0].bps];
    S->grid_vec = std::max(1, std::min<int>(static_cast<int>((N / 2 + kBlock - 1) / kBlock), C->num_sms * kVecBlocksPerSM));
    int max_grid = S->grid_vec;
    for (int bps = 3; bps <= 6; ++bps) max_grid = std::max({max_grid, plan.grid_bps[bps], plan.grid_bps32[bps]});
    S->n_partials = 3 * max_grid;

    struct Piece {
        const void *src;
        size_t bytes;
        size_t off;
    };
    std::vector<Piece> pieces;
    size_t total = 0;
    // every piece starts 256-byte aligned and keeps >= 64 bytes of slack after
    // its end (the SpMV stages tiles with 16-byte copies that may overrun the
    // last nonzero by up to 12 bytes)
    auto add = [&](const void *src, size_t bytes) {
        pieces.push_back({src, bytes, total});
        total = align_up(total + bytes + 64, 256);
        return pieces.size() - 1;
    };
    size_t i_rowptr = add(M.lrowptr.data(), sizeof(int32_t) * (N + 1));
    size_t i_col = add(gcol.data(), sizeof(int32_t) * M.nnz);
    size_t i_val = add(M.lval.data(), sizeof(double) * M.nnz);
    size_t i_irp = add(plan.irp.data(), sizeof(int32_t) * plan.irp.size());
    size_t i_icol = add(plan.icol.data(), sizeof(int32_t) * plan.icol.size());
    size_t i_ival = add(plan.ival.data(), sizeof(double) * plan.ival.size());
    if (plan.sval.size() > static_cast<size_t>(INT32_MAX) || plan.gval.size() > static_cast<size_t>(INT32_MAX)) {
        set_error("sliced matrix larger than 2^31 entries");
        return SSG_E_INVALID;
    }
    std::vector<float> sval32(plan.sval.begin(), plan.sval.end());
    size_t i_sval = add(plan.sval.data(), sizeof(double) * plan.sval.size());
    size_t i_sval32 = add(sval32.data(), sizeof(float) * sval32.size());
    size_t i_scol = add(plan.scol.data(), sizeof(int32_t) * plan.scol.size());
    size_t i_sseg = add(plan.sseg.data(), sizeof(int32_t) * plan.sseg.size());
    size_t i_srow = add(plan.srow.data(), sizeof(int32_t) * plan.srow.size());
    size_t i_items = add(plan.items.data(), sizeof(WorkItem) * plan.items.size());
    size_t i_items_g = add(plan.items_g.data(), sizeof(WorkItem) * plan.items_g.size());
    size_t i_gcopy = add(plan.gcopy.data(), sizeof(int32_t) * plan.gcopy.size());
    size_t i_range_bps[7] = {0, 0, 0, 0, 0, 0, 0}, i_range_bps32[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int bps = 3; bps <= 6; ++bps)
        i_range_bps[bps] = add(plan.range_bps[bps].data(), sizeof(int2) * plan.range_bps[bps].size());
    for (int bps = 3; bps <= 6; ++bps)
        i_range_bps32[bps] = add(plan.range_bps32[bps].data(), sizeof(int2) * plan.range_bps32[bps].size());
    size_t i_brangeB = add(plan.warp_rangeB.data(), sizeof(int2) * plan.warp_rangeB.size());
    size_t i_rcluster = add(plan.range_cluster.data(), sizeof(int2) * plan.range_cluster.size());
    size_t i_blk_seg = add(plan.blk_seg.data(), sizeof(int32_t) * plan.blk_seg.size());
    size_t i_seg_blk = add(plan.seg_blk.data(), sizeof(int32_t) * plan.seg_blk.size());
    size_t i_chunk = add(plan.chunk.data(), sizeof(int4) * plan.chunk.size());
    size_t i_seg_chunk = add(plan.seg_chunk.data(), sizeof(int32_t) * plan.seg_chunk.size());
    size_t i_node_off = add(S->seg_node.data(), sizeof(int32_t) * S->seg_node.size());
    size_t i_rhs_off = add(S->seg_rhs_off.data(), sizeof(int64_t) * S->seg_rhs_off.size());
    size_t i_nrhs = add(S->seg_nrhs.data(), sizeof(int32_t) * S->seg_nrhs.size());
    size_t i_iptr = add(M.iptr.data(), sizeof(int32_t) * (M.ngamma + 1));
    size_t i_icopy = add(M.icopy.data(), sizeof(int32_t) * M.ncopies);
    size_t i_mult = add(mloc.data(), N);
    size_t i_wown = add(wown.data(), N);
    size_t i_wtab = add(wtab.data(), sizeof(double) * 256);
    size_t i_gflag = add(gflag.data(), gflag.size());
    size_t i_gflag128 = add(gflag128.data(), gflag128.size());
    size_t i_wtab32 = add(wtab32.data(), sizeof(float) * 256);
    size_t i_l2g = add(M.l2g.data(), sizeof(int32_t) * N);
    size_t i_own = add(M.own.data(), sizeof(int32_t) * M.n);
    std::vector<float> val32(M.lval.begin(), M.lval.end());
    std::vector<float> ival32(plan.ival.begin(), plan.ival.end());
    size_t i_val32 = add(val32.data(), sizeof(float) * val32.size());
    size_t i_ival32 = add(ival32.data(), sizeof(float) * ival32.size());
    size_t i_r32 = add(nullptr, sizeof(float) * N);
    size_t i_p32 = add(nullptr, sizeof(float) * N);
    size_t i_q32 = add(nullptr, sizeof(float) * N);
    size_t i_d32 = add(nullptr, sizeof(float) * N);
    size_t i_scal_in = add(nullptr, sizeof(Scal));
    // element sub-structures have no input-CSR entry per local entry (-1 maps)
    const bool from_csr = !M.lsrc.empty();
    std::vector<int32_t> vmap = from_csr ? M.lsrc : std::vector<int32_t>(static_cast<size_t>(M.nnz), -1);
    std::vector<int32_t> imap(plan.isrc.size()), smap(plan.ssrc.size());
    for (size_t i = 0; i < imap.size(); ++i) imap[i] = vmap[plan.isrc[i]];
    for (size_t i = 0; i < smap.size(); ++i) smap[i] = plan.ssrc[i] >= 0 ? vmap[plan.ssrc[i]] : -1;
    // local entry holding the diagonal of each local entry's node (in the
    // owner's local matrix), -1 if the matrix stores none
    std::vector<int32_t> diag_of_row(static_cast<size_t>(N), -1), dmap(static_cast<size_t>(N), -1);
    for (int32_t sd = 0; sd < M.P; ++sd)
        for (int64_t r = M.off[sd]; r < M.off[sd + 1]; ++r)
            for (int32_t e = M.lrowptr[r]; e < M.lrowptr[r + 1]; ++e)
                if (M.off[sd] + M.lcol[e] == r) diag_of_row[r] = e;
    for (int64_t k = 0; k < N; ++k) dmap[k] = diag_of_row[M.own[M.l2g[k]]];
    // element sub-structures: every copy holds a partial diagonal, so 1 / S_ii
    // comes from the assembled diagonal of the host maps
    std::vector<double> hdinv;
    std::vector<float> hdinv32;
    int hbad = 0;
    if (!from_csr) {
        hdinv.resize(static_cast<size_t>(N));
        hdinv32.resize(static_cast<size_t>(N));
        for (int64_t k = 0; k < N; ++k) {
            const double d = M.diag[M.l2g[k]];
            double v = 0.0;
            if (d > 0.0 && std::isfinite(d)) v = 1.0 / d;
            else hbad = 1;
            hdinv[k] = v;
            hdinv32[k] = static_cast<float>(v);
        }
        std::fill(dmap.begin(), dmap.end(), -1);
    }
    size_t i_dmap = add(dmap.data(), sizeof(int32_t) * N);
    size_t i_dinv = add(from_csr ? nullptr : hdinv.data(), sizeof(double) * N);
    size_t i_dinv32 = add(from_csr ? nullptr : hdinv32.data(), sizeof(float) * N);
    size_t i_diag_bad = add(from_csr ? nullptr : &hbad, sizeof(int));
    size_t i_vmap = add(vmap.data(), sizeof(int32_t) * M.nnz);
    size_t i_imap = add(imap.data(), sizeof(int32_t) * imap.size());
    size_t i_smap = add(smap.data(), sizeof(int32_t) * smap.size());
    size_t i_bl = add(nullptr, sizeof(double) * N);
    size_t i_xl = add(nullptr, sizeof(double) * N);
    size_t i_r = add(nullptr, sizeof(double) * N);
    size_t i_p = add(nullptr, sizeof(double) * N);
    size_t i_q = add(nullptr, sizeof(double) * N);
    size_t i_part = add(nullptr, sizeof(double) * S->n_partials);
    size_t i_scal = add(nullptr, sizeof(Scal));
    size_t i_scal2 = add(nullptr, sizeof(Scal));
    size_t i_xg = add(nullptr, sizeof(double) * M.n);
    size_t i_bg = add(nullptr, sizeof(double) * M.n);
    // the interface groups' sliced data (the small tables sit beside the
    // other item lists: every launch reads them first)
    std::vector<float> gval32(plan.gval.begin(), plan.gval.end());
    std::vector<int32_t> gmap(plan.gsrc.size());
    for (size_t i = 0; i < gmap.size(); ++i) gmap[i] = plan.gsrc[i] >= 0 ? vmap[plan.gsrc[i]] : -1;
    size_t i_gval = add(plan.gval.data(), sizeof(double) * plan.gval.size());
    size_t i_gval32 = add(gval32.data(), sizeof(float) * gval32.size());
    size_t i_gcol = add(plan.gcol.data(), sizeof(int32_t) * plan.gcol.size());
    size_t i_gmap = add(gmap.data(), sizeof(int32_t) * gmap.size());

    cudaError_t e = cudaMalloc(&S->arena, total);
    if (e != cudaSuccess) {
        set_error(std::string("device arena of ") + std::to_string(total) + " bytes: " + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SSG_E_OOM : SSG_E_CUDA;
    }
    S->arena_bytes = total;
    char *base = static_cast<char *>(S->arena);
    SSG_CUDA_TRY(cudaMemsetAsync(S->arena, 0, total, C->stream));  // slack bytes read by the tile copies
    for (const Piece &p : pieces)
        if (p.src && p.bytes) SSG_CUDA_TRY(cudaMemcpyAsync(base + p.off, p.src, p.bytes, cudaMemcpyHostToDevice, C->stream));
    auto at = [&](size_t i) { return static_cast<void *>(base + pieces[i].off); };
    S->op.rowptr = static_cast<const int32_t *>(at(i_rowptr));
    S->op.col = static_cast<const int32_t *>(at(i_col));
    S->op.val = static_cast<const double *>(at(i_val));
    S->op.val32 = static_cast<const float *>(at(i_val32));
    S->op.ival32 = static_cast<const float *>(at(i_ival32));
    S->d_r32 = static_cast<float *>(at(i_r32));
    S->d_p32 = static_cast<float *>(at(i_p32));
    S->d_q32 = static_cast<float *>(at(i_q32));
    S->d_d32 = static_cast<float *>(at(i_d32));
    S->d_scal_in = static_cast<Scal *>(at(i_scal_in));
    S->d_dmap = static_cast<int32_t *>(at(i_dmap));
    S->d_dinv = static_cast<double *>(at(i_dinv));
    S->d_dinv32 = static_cast<float *>(at(i_dinv32));
    S->d_diag_bad = static_cast<int *>(at(i_diag_bad));
    S->d_vmap = static_cast<int32_t *>(at(i_vmap));
    S->d_imap = static_cast<int32_t *>(at(i_imap));
    S->d_smap = static_cast<int32_t *>(at(i_smap));
    S->n_ival = static_cast<int64_t>(imap.size());
    S->n_sval = static_cast<int64_t>(smap.size());
    S->op.irp = static_cast<const int32_t *>(at(i_irp));
    S->op.icol = static_cast<const int32_t *>(at(i_icol));
    S->op.ival = static_cast<const double *>(at(i_ival));
    S->op.sval = static_cast<const double *>(at(i_sval));
    S->op.sval32 = static_cast<const float *>(at(i_sval32));
    S->op.scol = static_cast<const int32_t *>(at(i_scol));
    S->op.sseg = static_cast<const int32_t *>(at(i_sseg));
    S->op.srow = static_cast<const int32_t *>(at(i_srow));
    S->op.gcopy = static_cast<const int32_t *>(at(i_gcopy));
    S->op.gval = static_cast<const double *>(at(i_gval));
    S->op.gval32 = static_cast<const float *>(at(i_gval32));
    S->op.gcol = static_cast<const int32_t *>(at(i_gcol));
    S->d_gmap = static_cast<int32_t *>(at(i_gmap));
    S->n_gval = static_cast<int64_t>(gmap.size());
    // single-vector products: the list with interface groups when built;
    // the K-vector products and the one-cluster solve: the slices
    S->items_slices = static_cast<const WorkItem *>(at(i_items));
    S->op.items = plan.items_g.empty() ? S->items_slices : static_cast<const WorkItem *>(at(i_items_g));
    S->iface_groups = !plan.items_g.empty();
    for (int bps = 3; bps <= 6; ++bps) {
        S->range_bps[bps] = static_cast<const int2 *>(at(i_range_bps[bps]));
        S->range_bps32[bps] = static_cast<const int2 *>(at(i_range_bps32[bps]));
    }
    S->op.warp_range = S->range_bps[kSpmv64Variants[0].bps];
    S->op32 = S->op;  // filled below once the op is complete
    S->op.iptr = static_cast<const int32_t *>(at(i_iptr));
    S->op.icopy = static_cast<const int32_t *>(at(i_icopy));
    S->op.mult = static_cast<const uint8_t *>(at(i_mult));
    S->d_mult = S->op.mult;
    S->d_wown = static_cast<const uint8_t *>(at(i_wown));
    S->op.wtab = static_cast<const double *>(at(i_wtab));
    S->op.gflag = static_cast<const uint8_t *>(at(i_gflag));
    S->op.gflag128 = static_cast<const uint8_t *>(at(i_gflag128));
    S->op.wtab32 = static_cast<const float *>(at(i_wtab32));
    S->d_l2g = static_cast<int32_t *>(at(i_l2g));
    S->d_own = static_cast<int32_t *>(at(i_own));
    S->d_bl = static_cast<double *>(at(i_bl));
    S->d_xl = static_cast<double *>(at(i_xl));
    S->d_r = static_cast<double *>(at(i_r));
    S->d_p = static_cast<double *>(at(i_p));
    S->d_q = static_cast<double *>(at(i_q));
    S->d_partials = static_cast<double *>(at(i_part));
    S->d_scal = static_cast<Scal *>(at(i_scal));
    S->d_scal_op = static_cast<Scal *>(at(i_scal2));
    S->d_xg = static_cast<double *>(at(i_xg));
    S->d_bg = static_cast<double *>(at(i_bg));
    S->op32 = S->op;
    S->op32.items = S->items_slices;
    S->op32.warp_range = S->range_bps32[kSpmv32Variants[0].bps];
    S->opB64 = S->op;
    S->opB64.items = S->items_slices;
    S->opB64.warp_range = static_cast<const int2 *>(at(i_brangeB));
    S->opB32 = S->opB64;
    S->grid_spmmB = plan.gridB;
    if (!plan.range_cluster.empty()) {
        S->range_cluster = static_cast<const int2 *>(at(i_rcluster));
        S->cluster_ctas = cl_ctas;
        S->cluster_nranges = plan.cluster_nranges;
    }
    S->nchunks = static_cast<int32_t>(plan.chunk.size());
    S->tab.blk_seg = static_cast<const int32_t *>(at(i_blk_seg));
    S->tab.seg_blk = static_cast<const int32_t *>(at(i_seg_blk));
    S->tab.chunk = static_cast<const int4 *>(at(i_chunk));
    S->tab.seg_chunk = static_cast<const int32_t *>(at(i_seg_chunk));
    S->tab.node_off = static_cast<const int32_t *>(at(i_node_off));
    S->tab.rhs_off = static_cast<const int64_t *>(at(i_rhs_off));
    S->tab.nrhs = static_cast<const int32_t *>(at(i_nrhs));
    S->tab.nseg = S->nseg;
    SSG_CUDA_TRY(cudaMemsetAsync(S->d_scal, 0, sizeof(Scal), C->stream));
    SSG_CUDA_TRY(cudaMemsetAsync(S->d_scal_op, 0, sizeof(Scal), C->stream));
    if (from_csr)
        k_dinv<<<grid_for(N, C->num_sms), kBlock, 0, C->stream>>>(N, S->d_dmap, S->op.val, S->d_dinv, S->d_dinv32,
                                                                   S->d_diag_bad);
    SSG_CUDA_TRY(cudaGetLastError());
    SSG_CUDA_TRY(cudaEventCreate(&S->ev0));
    SSG_CUDA_TRY(cudaEventCreate(&S->ev1));
    // the host vectors above are freed when this function returns
    SSG_CUDA_TRY(cudaStreamSynchronize(C->stream));
    S->on_device = true;
    return SSG_OK;
}

int check_dev(const ssg_system *S) {
    if (!S) {
        set_error("null system");
        return SSG_E_INVALID;
    }
    if (!S->on_device) {
        set_error("system has host maps only (built without a context)");
        return SSG_E_INVALID;
    }
    return SSG_OK;
}

// One right-hand side: b_glob/x_glob are device pointers (length n).
int read_scal(ssg_system *S, const Scal *src, Scal *dst) {
    SSG_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(Scal), cudaMemcpyDeviceToHost, S->ctx->stream));
    SSG_CUDA_TRY(cudaStreamSynchronize(S->ctx->stream));
    return SSG_OK;
}

// Host-loop drivers (SSG_DRIVER_HOST): the same kernels, launched directly,
// the done flags read back every kHostChunk iterations.
int run_host_fp64(ssg_system *S, int64_t *launches, bool pc) {
    cudaStream_t s = S->ctx->stream;
    int rc = launch_init(S, s, 0, pc);
    if (rc != SSG_OK) return rc;
    *launches += 1;
    Scal h{};
    for (;;) {
        rc = read_scal(S, S->d_scal, &h);
        if (rc != SSG_OK) return rc;
        if (h.done) return SSG_OK;
        for (int i = 0; i < kHostChunk; ++i) {
            rc = launch_body(S, s, 0, pc);
            if (rc != SSG_OK) return rc;
        }
        *launches += 3 * kHostChunk;
    }
}

int run_host_mixed(ssg_system *S, int64_t *launches, bool pc) {
    cudaStream_t s = S->ctx->stream;
    int rc = launch_mixed_init(S, s, 0, pc);
    if (rc != SSG_OK) return rc;
    *launches += 1;
    Scal ho{}, hi{};
    for (;;) {
        rc = read_scal(S, S->d_scal, &ho);
        if (rc != SSG_OK) return rc;
        if (ho.done) return SSG_OK;
        rc = launch_inner_init(S, s, 0, pc);
        if (rc != SSG_OK) return rc;
        *launches += 1;
        for (;;) {
            rc = read_scal(S, S->d_scal_in, &hi);
            if (rc != SSG_OK) return rc;
            if (hi.done) break;
            for (int i = 0; i < kHostChunk; ++i) {
                rc = launch_inner_body(S, s, 0, pc);
                if (rc != SSG_OK) return rc;
            }
            *launches += 3 * kHostChunk;
        }
        rc = launch_outer_tail(S, s, 0, pc);
        if (rc != SSG_OK) return rc;
        *launches += 3;
    }
}

// The diagonal preconditioner needs every diagonal entry present and
// positive; k_dinv flags the first violation, read here once per set of values.
int check_diag(ssg_system *S) {
    if (S->diag_state < 0) {
        int bad = 0;
        SSG_CUDA_TRY(cudaMemcpyAsync(&bad, S->d_diag_bad, sizeof(int), cudaMemcpyDeviceToHost, S->ctx->stream));
        SSG_CUDA_TRY(cudaStreamSynchronize(S->ctx->stream));
        S->diag_state = bad ? 1 : 0;
    }
    if (S->diag_state) {
        set_error("SSG_FP64_JACOBI needs every diagonal entry present and positive");
        return SSG_E_INVALID;
    }
    return SSG_OK;
}

// The one-cluster solve's CTAs per cluster: the largest of 16, 8, 4 and 2
// for which the occupancy query places at least one cluster of both
// instances (16 is beyond the portable cluster size and must be allowed per
// kernel); 0 if none is placed or the query fails.
int pick_cluster_ctas(cudaStream_t st) {
    if (cudaFuncSetAttribute(k_cg_cluster<false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(k_cg_cluster<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    for (int nc = kClusterMaxCtas; nc >= 2; nc /= 2) {
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = nc;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(nc);
        cfg.blockDim = dim3(kClusterThreads);
        cfg.stream = st;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n0 = 0, n1 = 0;
        const bool ok = cudaOccupancyMaxActiveClusters(&n0, k_cg_cluster<false>, &cfg) == cudaSuccess &&
                        cudaOccupancyMaxActiveClusters(&n1, k_cg_cluster<true>, &cfg) == cudaSuccess;
        if (!ok) cudaGetLastError();
        if (ok && n0 > 0 && n1 > 0) return nc;
    }
    return 0;
}

// Whether a single-vector FP64 solve of S runs as the one-cluster kernel.
bool use_cluster(const ssg_system *S, bool mixed) {
    const ssg_ctx *C = S->ctx;
    return !mixed && C->driver == SSG_DRIVER_GRAPH && S->cluster_ctas > 0 && S->maps.nloc <= C->cluster_max_n &&
           S->nseg == 1;
}

int launch_cluster_cg(ssg_system *S, cudaStream_t st, bool pc) {
    const int nc = S->cluster_ctas;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = nc;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(nc);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    DevOp A = S->op;
    A.items = S->items_slices;
    A.warp_range = S->range_cluster;
    const int64_t N = S->maps.nloc;
    if (pc)
        SSG_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_cg_cluster<true>, A, N, S->cluster_nranges,
                                        static_cast<const double *>(S->d_bl), S->d_xl, S->d_r, S->d_p, S->d_q,
                                        static_cast<const double *>(S->d_dinv), S->d_scal));
    else
        SSG_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_cg_cluster<false>, A, N, S->cluster_nranges,
                                        static_cast<const double *>(S->d_bl), S->d_xl, S->d_r, S->d_p, S->d_q,
                                        static_cast<const double *>(S->d_dinv), S->d_scal));
    return SSG_OK;
}

// One right-hand side: b_glob/x_glob are device pointers (length n).
int solve_one(ssg_system *S, const double *b_glob, double *x_glob, int guess, double rtol, int32_t max_iter,
              int mode, ssg_stats *st) {
    const bool mixed = mode == SSG_MIXED || mode == SSG_MIXED_JACOBI;
    const bool pc = mode == SSG_FP64_JACOBI || mode == SSG_MIXED_JACOBI;
    if (pc) {
        int rc0 = check_diag(S);
        if (rc0 != SSG_OK) return rc0;
    }
    ssg_ctx *C = S->ctx;
    cudaStream_t s = C->stream;
    const int64_t N = S->maps.nloc;
    int64_t launches = 0;
    SSG_CUDA_TRY(cudaEventRecord(S->ev0, s));
    k_scatter<<<grid_for(N, C->num_sms), kBlock, 0, s>>>(N, S->d_l2g, b_glob, S->d_bl);
    ++launches;
    if (guess) {
        k_scatter<<<grid_for(N, C->num_sms), kBlock, 0, s>>>(N, S->d_l2g, x_glob, S->d_xl);
        v64(S)[S->var64].store<<<S->grid_spmv, kSpmvThreads, 0, s>>>(
            S->op, S->d_xl, S->d_q, S->d_partials, S->d_scal_op, nullptr, 0, 0);
        launches += 2;
    } else {
        SSG_CUDA_TRY(cudaMemsetAsync(S->d_xl, 0, sizeof(double) * N, s));
    }
    k_set_params<<<1, 32, 0, s>>>(S->d_scal, rtol, max_iter, guess);
    ++launches;
    if (mixed) {
        k_set_mixed<<<1, 32, 0, s>>>(S->d_scal, C->inner_rtol, C->max_outer);
        ++launches;
    }
    SSG_CUDA_TRY(cudaGetLastError());
    int rc = SSG_OK;
    const bool cluster = use_cluster(S, mixed);
    if (cluster) {
        rc = launch_cluster_cg(S, s, pc);
        if (rc != SSG_OK) return rc;
        ++launches;
    } else if (C->driver == SSG_DRIVER_GRAPH) {
        rc = mixed ? build_graph_mixed(S, pc) : build_graph(S, pc);
        if (rc != SSG_OK) return rc;
        SSG_CUDA_TRY(cudaGraphLaunch(mixed ? S->exec_m[pc] : pc ? S->exec_pc : S->exec, s));
    } else {
        rc = mixed ? run_host_mixed(S, &launches, pc) : run_host_fp64(S, &launches, pc);
        if (rc != SSG_OK) return rc;
    }
    k_gather<<<grid_for(S->maps.n, C->num_sms), kBlock, 0, s>>>(S->maps.n, S->d_own, S->d_xl, x_glob);
    // true residual ||b - S x||_w in FP64
    v64(S)[S->var64].store<<<S->grid_spmv, kSpmvThreads, 0, s>>>(
        S->op, S->d_xl, S->d_q, S->d_partials, S->d_scal_op, nullptr, 0, 0);
    k_wdot<true><<<S->grid_vec, kBlock, 0, s>>>(N, S->d_bl, S->d_q, S->op.mult, S->op.wtab, S->d_partials,
                                                S->d_scal_op, &S->d_scal->aux);
    launches += 3;
    SSG_CUDA_TRY(cudaGetLastError());
    SSG_CUDA_TRY(cudaEventRecord(S->ev1, s));
    Scal h{};
    rc = read_scal(S, S->d_scal, &h);
    if (rc != SSG_OK) return rc;
    float ms = 0.f;
    SSG_CUDA_TRY(cudaEventElapsedTime(&ms, S->ev0, S->ev1));
    if (C->driver == SSG_DRIVER_GRAPH && !cluster) {
        // every copy of an iteration in a loop pass launches all its kernels;
        // the device counts the residual-update launches (h.passes)
        if (mixed)  // init, per refinement: inner init + 3 tail kernels; 3 per inner copy
            launches += 1 + 4 * static_cast<int64_t>(h.iter) + 3 * int64_t(h.passes);
        else  // init, 3 per copy
            launches += 1 + 3 * static_cast<int64_t>(h.passes);
    }
    if (st) {
        st->status = h.status;
        st->iters = mixed ? h.total : h.iter;
        st->outer = mixed ? h.iter : 1;
        st->block = 1;
        st->relres = h.relres;
        st->true_relres = h.bnorm > 0.0 ? std::sqrt(h.aux) / h.bnorm : std::sqrt(h.aux);
        st->solve_ms = ms;
        st->kernel_launches = launches;
    }
    return h.status;
}

// ---------------------------------------------------------------------------
// Several right-hand sides, and several independent systems, together:
// K columns per launch, one state per segment (block.cuh).
// ---------------------------------------------------------------------------

int log2_of(int K) { return K == 2 ? 1 : K == 4 ? 2 : K == 8 ? 3 : 4; }

void destroy_block_graphs(ssg_system *S) {
    for (auto &by_k : S->blk.graph)
        for (ssg_system::BlockGraph &G : by_k) {
            if (G.exec) cudaGraphExecDestroy(G.exec);
            if (G.g) cudaGraphDestroy(G.g);
            G = ssg_system::BlockGraph{};
        }
}

void free_block(ssg_system *S) {
    destroy_block_graphs(S);
    if (S->blk.mem) {
        if (S->ctx && S->ctx->stream) cudaStreamSynchronize(S->ctx->stream);
        cudaFree(S->blk.mem);
    }
    S->blk = ssg_system::BlockState{};
}

// Device vectors for K columns (kept for later solves with K' <= K), the
// partials and one state per segment (+1 for the loop counters).
int ensure_block(ssg_system *S, int K) {
    if (S->blk.kcap >= K) return SSG_OK;
    free_block(S);
    const int64_t N = S->maps.nloc, n = S->maps.n;
    // part_a: the product's block partials, or up to three partial sets of the
    // setup kernels; part_b: (r, r)_w and, with the preconditioner, (r, z)_w
    const int64_t gmax = std::max<int64_t>(S->grid_spmmB, 3 * static_cast<int64_t>(S->nchunks));
    size_t total = 0;
    auto take = [&](size_t bytes) {
        const size_t o = total;
        total = align_up(total + bytes, 256);
        return o;
    };
    const size_t NK = static_cast<size_t>(N) * K;
    const size_t o_bl = take(8 * NK), o_xl = take(8 * NK), o_r = take(8 * NK), o_p = take(8 * NK),
                 o_q = take(8 * NK);
    const size_t o_r32 = take(4 * NK), o_p32 = take(4 * NK), o_q32 = take(4 * NK), o_d32 = take(4 * NK);
    const size_t o_pa = take(sizeof(double) * static_cast<size_t>(gmax) * kMaxRhs);
    const size_t o_pb = take(sizeof(double) * 2 * static_cast<size_t>(S->nchunks) * kMaxRhs);
    const size_t o_bg = take(8 * static_cast<size_t>(n) * K), o_xg = take(8 * static_cast<size_t>(n) * K);
    const size_t o_so = take(sizeof(ScalB) * (S->nseg + 1)), o_si = take(sizeof(ScalB) * (S->nseg + 1));
    void *mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, total);
    if (e != cudaSuccess) {
        set_error(std::string("block vectors of ") + std::to_string(total) + " bytes: " + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SSG_E_OOM : SSG_E_CUDA;
    }
    char *b = static_cast<char *>(mem);
    ssg_system::BlockState &B = S->blk;
    B.mem = mem;
    B.kcap = K;
    B.bl = reinterpret_cast<double *>(b + o_bl);
    B.xl = reinterpret_cast<double *>(b + o_xl);
    B.r = reinterpret_cast<double *>(b + o_r);
    B.p = reinterpret_cast<double *>(b + o_p);
    B.q = reinterpret_cast<double *>(b + o_q);
    B.r32 = reinterpret_cast<float *>(b + o_r32);
    B.p32 = reinterpret_cast<float *>(b + o_p32);
    B.q32 = reinterpret_cast<float *>(b + o_q32);
    B.d32 = reinterpret_cast<float *>(b + o_d32);
    B.part_a = reinterpret_cast<double *>(b + o_pa);
    B.part_b = reinterpret_cast<double *>(b + o_pb);
    B.bg = reinterpret_cast<double *>(b + o_bg);
    B.xg = reinterpret_cast<double *>(b + o_xg);
    B.so = reinterpret_cast<ScalB *>(b + o_so);
    B.si = reinterpret_cast<ScalB *>(b + o_si);
    SSG_CUDA_TRY(cudaMemsetAsync(mem, 0, total, S->ctx->stream));
    return SSG_OK;
}

// Partials: the K-vector product and the setup / residual / inner-setup
// kernels write part_a, the residual updates part_b.
template <int K, bool PC>
int launch_initB(ssg_system *S, cudaStream_t st, double *p, cudaGraphConditionalHandle h, int use_cond) {
    ssg_system::BlockState &B = S->blk;
    // q holds S x_1 when a guess was given, else zeros (set before the loop)
    k_residualB<K, PC><<<S->nchunks, kBlockV, 0, st>>>(B.bl, B.q, B.r, p, S->op.mult, S->op.wtab, B.part_a, S->tab, 1,
                                                      1, S->d_dinv);
    k_init_finB<K, PC><<<S->nseg, kBlock, 0, st>>>(B.part_a, S->nchunks, S->tab, B.so);
    k_seg_cond<<<1, kBlock, 0, st>>>(B.so, S->nseg, B.so + S->nseg, nullptr, 1, h, use_cond);
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

constexpr int log2_cols(int K) { return K == 2 ? 0 : K == 4 ? 1 : K == 8 ? 2 : 3; }

// The K-vector product of the solves with the chunk depth and L2 look-ahead
// chosen for (precision, K); segs given: frozen segments' blocks return.
template <typename T, int K, bool DOTS>
void spmm_seg(ssg_system *S, cudaStream_t st, const T *X, T *Y, double *part, const ScalB *segs) {
    const int pi = sizeof(T) == 8 ? 0 : 1, lk = log2_cols(K);
    DevOp A = pi == 0 ? S->opB64 : S->opB32;
    A.l2_ahead = S->spmm_ahead[pi][lk];
    if (S->spmm_nc[pi][lk] == 1)
        k_spmm_seg<T, K, DOTS, 1><<<S->grid_spmmB, kSpmvThreads, 0, st>>>(A, X, Y, part, S->tab, segs);
    else
        k_spmm_seg<T, K, DOTS, 2><<<S->grid_spmmB, kSpmvThreads, 0, st>>>(A, X, Y, part, S->tab, segs);
}

template <int K, bool PC>
int launch_bodyB64(ssg_system *S, cudaStream_t st, cudaGraphConditionalHandle h, int use_cond) {
    ssg_system::BlockState &B = S->blk;
    spmm_seg<double, K, true>(S, st, B.p, B.q, B.part_a, B.so);
    k_update_rB<K, PC><<<S->nchunks, kBlockV, 0, st>>>(B.q, B.r, S->op.mult, S->op.wtab, S->op.gflag, B.part_a,
                                                      B.part_b, S->tab, B.so, S->d_dinv);
    k_update_xpB<K, PC><<<S->nchunks, kBlockV, 0, st>>>(B.xl, B.p, B.r, B.part_b, S->tab, B.so, S->d_dinv);
    k_seg_cond<<<1, kBlock, 0, st>>>(B.so, S->nseg, B.so + S->nseg, nullptr, 0, h, use_cond);
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

template <int K, bool PC>
int launch_inner_initB(ssg_system *S, cudaStream_t st, cudaGraphConditionalHandle h, int use_cond) {
    ssg_system::BlockState &B = S->blk;
    k_inner_initB<K, PC><<<S->nchunks, kBlockV, 0, st>>>(B.r, B.r32, B.p32, B.d32, S->op.mult, S->op.wtab32, B.part_a,
                                                        S->tab, S->d_dinv32);
    k_inner_finB<K, PC><<<S->nseg, kBlock, 0, st>>>(B.part_a, S->nchunks, S->tab, B.si, B.so);
    k_seg_cond<<<1, kBlock, 0, st>>>(B.si, S->nseg, B.si + S->nseg, nullptr, 1, h, use_cond);
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

template <int K, bool PC>
int launch_inner_bodyB(ssg_system *S, cudaStream_t st, cudaGraphConditionalHandle h, int use_cond) {
    ssg_system::BlockState &B = S->blk;
    spmm_seg<float, K, true>(S, st, B.p32, B.q32, B.part_a, B.si);
    k_update_r32B<K, PC><<<S->nchunks, kBlockV, 0, st>>>(B.q32, B.r32, S->op.mult, S->op.wtab32, S->op.gflag128,
                                                        B.part_a, B.part_b, S->tab, B.si, S->d_dinv32);
    k_update_dp32B<K, PC><<<S->nchunks, kBlockV, 0, st>>>(B.d32, B.p32, B.r32, B.part_b, S->tab, B.si, B.so,
                                                         S->d_dinv32);
    k_seg_cond<<<1, kBlock, 0, st>>>(B.si, S->nseg, B.si + S->nseg, B.so + S->nseg, 0, h, use_cond);
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

template <int K>
int launch_outer_tailB(ssg_system *S, cudaStream_t st, cudaGraphConditionalHandle h, int use_cond) {
    ssg_system::BlockState &B = S->blk;
    const int64_t N = S->maps.nloc;
    k_ir_correct<<<grid_for(N * K, S->ctx->num_sms), kBlock, 0, st>>>(N * K, B.xl, B.d32);
    spmm_seg<double, K, false>(S, st, B.xl, B.q, nullptr, B.so);
    k_residualB<K><<<S->nchunks, kBlockV, 0, st>>>(B.bl, B.q, B.r, nullptr, S->op.mult, S->op.wtab, B.part_a, S->tab,
                                                  1, 0);
    k_outer_finB<K><<<S->nseg, kBlock, 0, st>>>(B.part_a, S->tab, B.so, B.si, 0);
    k_seg_cond<<<1, kBlock, 0, st>>>(B.so, S->nseg, B.so + S->nseg, nullptr, 0, h, use_cond);
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

// init -> WHILE(c_out) { body }
template <typename FI, typename FB>
int build_loop_graph(ssg_system::BlockGraph &G, FI init, FB body) {
    SSG_CUDA_TRY(cudaGraphCreate(&G.g, 0));
    SSG_CUDA_TRY(cudaGraphConditionalHandleCreate(&G.c_out, G.g, 0u, cudaGraphCondAssignDefault));
    cudaStream_t cap;
    SSG_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    int rc = SSG_OK;
    cudaGraphNode_t n_init = nullptr, n_loop = nullptr;
    cudaGraph_t g_body = nullptr;
    cudaError_t e = capture_into(cap, G.g, nullptr, 0, [&](cudaStream_t c) { return init(c, G.c_out); }, &rc);
    if (e == cudaSuccess && rc == SSG_OK) e = last_node(G.g, &n_init);
    if (e == cudaSuccess && rc == SSG_OK) e = add_while(G.g, &n_init, G.c_out, &n_loop, &g_body);
    if (e == cudaSuccess && rc == SSG_OK)
        e = capture_into(cap, g_body, nullptr, 0, [&](cudaStream_t c) { return body(c, G.c_out); }, &rc);
    if (e == cudaSuccess && rc == SSG_OK) e = cudaGraphInstantiate(&G.exec, G.g, 0);
    cudaStreamDestroy(cap);
    if (rc == SSG_OK && e != cudaSuccess) {
        set_error(std::string("building the block CG graph: ") + cudaGetErrorString(e));
        rc = SSG_E_CUDA;
    }
    if (rc != SSG_OK) {
        if (G.g) cudaGraphDestroy(G.g);
        G = ssg_system::BlockGraph{};
    }
    return rc;
}

// init -> WHILE(c_out) { inner init -> WHILE(c_in) { inner body } -> tail }
template <typename FI, typename FII, typename FIB, typename FT>
int build_nested_graph(ssg_system::BlockGraph &G, FI init, FII iinit, FIB ibody, FT tail) {
    SSG_CUDA_TRY(cudaGraphCreate(&G.g, 0));
    SSG_CUDA_TRY(cudaGraphConditionalHandleCreate(&G.c_out, G.g, 0u, cudaGraphCondAssignDefault));
    cudaStream_t cap;
    SSG_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    int rc = SSG_OK;
    cudaGraphNode_t n_init = nullptr, n_outer = nullptr, n_iinit = nullptr, n_inner = nullptr;
    cudaGraph_t body_out = nullptr, body_in = nullptr;
    cudaError_t e = capture_into(cap, G.g, nullptr, 0, [&](cudaStream_t c) { return init(c, G.c_out); }, &rc);
    if (e == cudaSuccess && rc == SSG_OK) e = last_node(G.g, &n_init);
    if (e == cudaSuccess && rc == SSG_OK) e = add_while(G.g, &n_init, G.c_out, &n_outer, &body_out);
    if (e == cudaSuccess && rc == SSG_OK)
        e = cudaGraphConditionalHandleCreate(&G.c_in, body_out, 0u, cudaGraphCondAssignDefault);
    if (e == cudaSuccess && rc == SSG_OK)
        e = capture_into(cap, body_out, nullptr, 0, [&](cudaStream_t c) { return iinit(c, G.c_in); }, &rc);
    if (e == cudaSuccess && rc == SSG_OK) e = last_node(body_out, &n_iinit);
    if (e == cudaSuccess && rc == SSG_OK) e = add_while(body_out, &n_iinit, G.c_in, &n_inner, &body_in);
    if (e == cudaSuccess && rc == SSG_OK)
        e = capture_into(cap, body_in, nullptr, 0, [&](cudaStream_t c) { return ibody(c, G.c_in); }, &rc);
    if (e == cudaSuccess && rc == SSG_OK)
        e = capture_into(cap, body_out, &n_inner, 1, [&](cudaStream_t c) { return tail(c, G.c_out); }, &rc);
    if (e == cudaSuccess && rc == SSG_OK) e = cudaGraphInstantiate(&G.exec, G.g, 0);
    cudaStreamDestroy(cap);
    if (rc == SSG_OK && e != cudaSuccess) {
        set_error(std::string("building the block mixed-precision graph: ") + cudaGetErrorString(e));
        rc = SSG_E_CUDA;
    }
    if (rc != SSG_OK) {
        if (G.g) cudaGraphDestroy(G.g);
        G = ssg_system::BlockGraph{};
    }
    return rc;
}

int read_glob(ssg_system *S, const ScalB *src, ScalB *dst) {
    SSG_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(ScalB), cudaMemcpyDeviceToHost, S->ctx->stream));
    SSG_CUDA_TRY(cudaStreamSynchronize(S->ctx->stream));
    return SSG_OK;
}

template <int K, bool PC>
int run_blockB_pc(ssg_system *S, int mode, int64_t *launches) {
    ssg_ctx *C = S->ctx;
    cudaStream_t s = C->stream;
    ssg_system::BlockState &B = S->blk;
    const bool mixed = mode == SSG_MIXED || mode == SSG_MIXED_JACOBI;
    int rc = SSG_OK;
    if (C->driver == SSG_DRIVER_GRAPH) {
        ssg_system::BlockGraph &G = B.graph[mode][log2_of(K)];
        if (!G.exec) {
            if (mixed)
                rc = build_nested_graph(
                    G,
                    [&](cudaStream_t c, cudaGraphConditionalHandle h) {
                        return launch_initB<K, false>(S, c, nullptr, h, 1);
                    },
                    [&](cudaStream_t c, cudaGraphConditionalHandle h) { return launch_inner_initB<K, PC>(S, c, h, 1); },
                    [&](cudaStream_t c, cudaGraphConditionalHandle h) { return launch_inner_bodyB<K, PC>(S, c, h, 1); },
                    [&](cudaStream_t c, cudaGraphConditionalHandle h) { return launch_outer_tailB<K>(S, c, h, 1); });
            else
                rc = build_loop_graph(
                    G, [&](cudaStream_t c, cudaGraphConditionalHandle h) { return launch_initB<K, PC>(S, c, B.p, h, 1); },
                    [&](cudaStream_t c, cudaGraphConditionalHandle h) { return launch_bodyB64<K, PC>(S, c, h, 1); });
            if (rc != SSG_OK) return rc;
        }
        SSG_CUDA_TRY(cudaGraphLaunch(G.exec, s));
        return SSG_OK;
    }
    ScalB ho{}, hi{};
    const ScalB *go = B.so + S->nseg, *gi = B.si + S->nseg;
    if (!mixed) {
        rc = launch_initB<K, PC>(S, s, B.p, 0, 0);
        *launches += 3;
        for (; rc == SSG_OK;) {
            rc = read_glob(S, go, &ho);
            if (rc != SSG_OK || ho.done) break;
            for (int i = 0; i < kHostChunk && rc == SSG_OK; ++i) rc = launch_bodyB64<K, PC>(S, s, 0, 0);
            *launches += 4 * kHostChunk;
        }
        return rc;
    }
    rc = launch_initB<K, false>(S, s, nullptr, 0, 0);
    *launches += 3;
    for (; rc == SSG_OK;) {
        rc = read_glob(S, go, &ho);
        if (rc != SSG_OK || ho.done) break;
        rc = launch_inner_initB<K, PC>(S, s, 0, 0);
        *launches += 3;
        for (; rc == SSG_OK;) {
            rc = read_glob(S, gi, &hi);
            if (rc != SSG_OK || hi.done) break;
            for (int i = 0; i < kHostChunk && rc == SSG_OK; ++i) rc = launch_inner_bodyB<K, PC>(S, s, 0, 0);
            *launches += 4 * kHostChunk;
        }
        if (rc == SSG_OK) rc = launch_outer_tailB<K>(S, s, 0, 0);
        *launches += 5;
    }
    return rc;
}

template <int K>
int run_blockB(ssg_system *S, int mode, int64_t *launches) {
    return mode == SSG_FP64_JACOBI || mode == SSG_MIXED_JACOBI ? run_blockB_pc<K, true>(S, mode, launches)
                                                               : run_blockB_pc<K, false>(S, mode, launches);
}

// All segments' right-hand sides at b_glob / x_glob (device; segment sg's
// right-hand side j at seg_rhs_off[sg] + j * n_sg); nr_single > 0 for a
// one-segment solve of nr_single right-hand sides; st receives one entry per
// (segment, right-hand side) in that order.
// The parts of a block solve around its loop, on stream s: before it the
// parameters, b scattered to the local copies, x and q set (x = 0, or the
// guess and q = S x); after it x gathered, the true residuals, and the
// states copied to pinned host memory for solve_block_finish.
template <int K>
int block_pre(ssg_system *S, int nr_single, const double *b_glob, double *x_glob, int guess, double rtol,
              int32_t max_iter, int mode, cudaStream_t s, int64_t *launches_out) {
    int rc = SSG_OK;
    if (mode == SSG_FP64_JACOBI || mode == SSG_MIXED_JACOBI) {
        rc = check_diag(S);
        if (rc != SSG_OK) return rc;
    }
    rc = ensure_block(S, K);
    if (rc != SSG_OK) return rc;
    ssg_ctx *C = S->ctx;
    ssg_system::BlockState &B = S->blk;
    const int64_t N = S->maps.nloc;
    int64_t launches = 0;
    SSG_CUDA_TRY(cudaEventRecord(S->ev0, s));
    k_set_paramsB<<<1, kBlock, 0, s>>>(B.so, S->nseg, rtol, max_iter, guess, C->inner_rtol, C->max_outer,
                                       const_cast<int32_t *>(S->tab.nrhs), nr_single);
    k_scatterB<K><<<S->nchunks, kBlockV, 0, s>>>(S->d_l2g, b_glob, B.bl, S->tab);
    launches += 2;
    if (guess) {
        k_scatterB<K><<<S->nchunks, kBlockV, 0, s>>>(S->d_l2g, x_glob, B.xl, S->tab);
        spmm_seg<double, K, false>(S, s, B.xl, B.q, nullptr, nullptr);
        launches += 2;
    } else {
        SSG_CUDA_TRY(cudaMemsetAsync(B.xl, 0, sizeof(double) * N * K, s));
        SSG_CUDA_TRY(cudaMemsetAsync(B.q, 0, sizeof(double) * N * K, s));
    }
    SSG_CUDA_TRY(cudaGetLastError());
    *launches_out += launches;
    return SSG_OK;
}

template <int K>
int block_post(ssg_system *S, int nr_single, double *x_glob, int mode, cudaStream_t s, int64_t launches) {
    ssg_system::BlockState &B = S->blk;
    k_gatherB<K><<<S->nchunks, kBlockV, 0, s>>>(S->d_l2g, S->d_own, B.xl, x_glob, S->tab);
    // true residuals ||b_j - S x_j||_w in FP64
    spmm_seg<double, K, false>(S, s, B.xl, B.q, nullptr, nullptr);
    k_residualB<K><<<S->nchunks, kBlockV, 0, s>>>(B.bl, B.q, nullptr, nullptr, S->op.mult, S->op.wtab, B.part_a,
                                                 S->tab, 1, 0);
    k_outer_finB<K><<<S->nseg, kBlock, 0, s>>>(B.part_a, S->tab, B.so, B.si, 1);
    launches += 4;
    SSG_CUDA_TRY(cudaGetLastError());
    SSG_CUDA_TRY(cudaEventRecord(S->ev1, s));
    if (!S->h_states) SSG_CUDA_TRY(cudaHostAlloc(&S->h_states, sizeof(ScalB) * (S->nseg + 1), cudaHostAllocDefault));
    SSG_CUDA_TRY(cudaMemcpyAsync(S->h_states, B.so, sizeof(ScalB) * (S->nseg + 1), cudaMemcpyDeviceToHost, s));
    S->pending_launches = launches;
    S->pending_k = K;
    S->pending_mode = mode;
    S->pending_nr = nr_single;
    return SSG_OK;
}

template <int K>
int solve_block_enqueue(ssg_system *S, int nr_single, const double *b_glob, double *x_glob, int guess, double rtol,
                        int32_t max_iter, int mode) {
    cudaStream_t s = S->ctx->stream;
    int64_t launches = 0;
    int rc = block_pre<K>(S, nr_single, b_glob, x_glob, guess, rtol, max_iter, mode, s, &launches);
    if (rc != SSG_OK) return rc;
    rc = run_blockB<K>(S, mode, &launches);
    if (rc != SSG_OK) return rc;
    return block_post<K>(S, nr_single, x_glob, mode, s, launches);
}

// Waits for the block solve enqueued on S and fills st (one entry per
// (segment, right-hand side)); returns SSG_OK or the first column's bad status.
int solve_block_finish(ssg_system *S, ssg_stats *st) {
    ssg_ctx *C = S->ctx;
    SSG_CUDA_TRY(cudaStreamSynchronize(C->stream));
    float ms = 0.f;
    SSG_CUDA_TRY(cudaEventElapsedTime(&ms, S->ev0, S->ev1));
    const ScalB *h = S->h_states;
    const ScalB &g = h[S->nseg];
    const int mode = S->pending_mode, K = S->pending_k, nr_single = S->pending_nr;
    const bool mixed = mode == SSG_MIXED || mode == SSG_MIXED_JACOBI;
    int64_t launches = S->pending_launches;
    if (C->driver == SSG_DRIVER_GRAPH) {
        if (mixed)  // init 3; per refinement inner init 3 + tail 5; 4 per inner loop iteration
            launches += 3 + 8 * static_cast<int64_t>(g.iter) + 4 * static_cast<int64_t>(g.loops);
        else
            launches += 3 + 4 * static_cast<int64_t>(g.iter);
    }
    int first_bad = SSG_OK;
    size_t o = 0;
    for (int sg = 0; sg < S->nseg; ++sg) {
        const ScalB &hs = h[sg];
        const int nr = nr_single > 0 ? nr_single : S->seg_nrhs[sg];
        for (int j = 0; j < nr; ++j, ++o) {
            if (hs.status[j] != SSG_OK && first_bad == SSG_OK) first_bad = hs.status[j];
            if (!st) continue;
            ssg_stats &t = st[o];
            t.status = hs.status[j];
            t.iters = hs.iters[j];
            t.outer = mixed ? hs.outer[j] : 1;
            t.block = K;
            t.relres = hs.relres[j];
            t.true_relres = hs.bnorm[j] > 0.0 ? std::sqrt(hs.aux[j]) / hs.bnorm[j] : std::sqrt(hs.aux[j]);
            t.solve_ms = ms;
            t.kernel_launches = launches;
        }
    }
    return first_bad;
}

template <int K>
int solve_block(ssg_system *S, int nr_single, const double *b_glob, double *x_glob, int guess, double rtol,
                int32_t max_iter, int mode, ssg_stats *st) {
    const int rc = solve_block_enqueue<K>(S, nr_single, b_glob, x_glob, guess, rtol, max_iter, mode);
    if (rc != SSG_OK) return rc;
    return solve_block_finish(S, st);
}

int solve_block_k(ssg_system *S, int nr, const double *b, double *x, int guess, double rtol, int32_t max_iter,
                  int mode, ssg_stats *st) {
    if (S->nseg != 1) {
        set_error("a batch of systems is solved with ssg_solve_batch");
        return SSG_E_INVALID;
    }
    if (nr <= 2) return solve_block<2>(S, nr, b, x, guess, rtol, max_iter, mode, st);
    if (nr <= 4) return solve_block<4>(S, nr, b, x, guess, rtol, max_iter, mode, st);
    if (nr <= 8) return solve_block<8>(S, nr, b, x, guess, rtol, max_iter, mode, st);
    return solve_block<16>(S, nr, b, x, guess, rtol, max_iter, mode, st);
}

int enqueue_batch_k(ssg_system *S, const double *b, double *x, int guess, double rtol, int32_t max_iter, int mode) {
    const int k = S->batch_k;
    if (k <= 2) return solve_block_enqueue<2>(S, 0, b, x, guess, rtol, max_iter, mode);
    if (k <= 4) return solve_block_enqueue<4>(S, 0, b, x, guess, rtol, max_iter, mode);
    if (k <= 8) return solve_block_enqueue<8>(S, 0, b, x, guess, rtol, max_iter, mode);
    return solve_block_enqueue<16>(S, 0, b, x, guess, rtol, max_iter, mode);
}

int solve_batch_k(ssg_system *S, const double *b, double *x, int guess, double rtol, int32_t max_iter, int mode,
                  ssg_stats *st) {
    const int k = S->batch_k;
    if (k <= 2) return solve_block<2>(S, 0, b, x, guess, rtol, max_iter, mode, st);
    if (k <= 4) return solve_block<4>(S, 0, b, x, guess, rtol, max_iter, mode, st);
    if (k <= 8) return solve_block<8>(S, 0, b, x, guess, rtol, max_iter, mode, st);
    return solve_block<16>(S, 0, b, x, guess, rtol, max_iter, mode, st);
}

template <typename T>
int spmm_checked(ssg_system *S, int32_t k, const T *x_loc, T *y_loc) {
    int rc = check_dev(S);
    if (rc != SSG_OK) return rc;
    if (!(k == 2 || k == 4 || k == 8 || k == 16)) {
        set_error("k must be 2, 4, 8 or 16");
        return SSG_E_INVALID;
    }
    const uintptr_t need = std::min<uintptr_t>(16, sizeof(T) * k);
    if (!x_loc || !y_loc || x_loc == y_loc || reinterpret_cast<uintptr_t>(x_loc) % need ||
        reinterpret_cast<uintptr_t>(y_loc) % need) {
        set_error("x_loc and y_loc must be distinct device blocks aligned to min(16, k * element size) bytes");
        return SSG_E_INVALID;
    }
    const DevOp &A = sizeof(T) == 8 ? S->opB64 : S->opB32;
    const int grid = S->grid_spmmB;
    cudaStream_t st = S->ctx->stream;
    switch (k) {
        case 2: k_spmm_asm<T, 2><<<grid, kSpmvThreads, 0, st>>>(A, x_loc, y_loc); break;
        case 4: k_spmm_asm<T, 4><<<grid, kSpmvThreads, 0, st>>>(A, x_loc, y_loc); break;
        case 8: k_spmm_asm<T, 8><<<grid, kSpmvThreads, 0, st>>>(A, x_loc, y_loc); break;
        default: k_spmm_asm<T, 16><<<grid, kSpmvThreads, 0, st>>>(A, x_loc, y_loc); break;
    }
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

// The system's input matrix must have the 7-point pattern of an nx x ny x nz
// grid (rows in cell order, columns ascending) before the grid kernels may
// index it: checked once on the host from the entry map, then the row
// pointers go to the device.
int check_fv7(ssg_system *S, int nx, int ny, int nz) {
    if (S->d_growptr && S->fv7_dims[0] == nx && S->fv7_dims[1] == ny && S->fv7_dims[2] == nz) return SSG_OK;
    const HostMaps &M = S->maps;
    if (M.lsrc.empty() || nx < 1 || ny < 1 || nz < 1 || static_cast<int64_t>(nx) * ny * nz != M.n) {
        set_error("grid size does not match the system");
        return SSG_E_INVALID;
    }
    const int64_t n = M.n;
    std::vector<int32_t> rp(static_cast<size_t>(n) + 1, 0), cols;
    cols.reserve(static_cast<size_t>(M.nnz));
    const int64_t sxy = static_cast<int64_t>(nx) * ny;
    for (int64_t i = 0; i < n; ++i) {
        const int ix = static_cast<int>(i % nx), iy = static_cast<int>((i / nx) % ny), iz = static_cast<int>(i / sxy);
        if (iz > 0) cols.push_back(static_cast<int32_t>(i - sxy));
        if (iy > 0) cols.push_back(static_cast<int32_t>(i - nx));
        if (ix > 0) cols.push_back(static_cast<int32_t>(i - 1));
        cols.push_back(static_cast<int32_t>(i));
        if (ix < nx - 1) cols.push_back(static_cast<int32_t>(i + 1));
        if (iy < ny - 1) cols.push_back(static_cast<int32_t>(i + nx));
        if (iz < nz - 1) cols.push_back(static_cast<int32_t>(i + sxy));
        rp[i + 1] = static_cast<int32_t>(cols.size());
    }
    if (static_cast<int64_t>(cols.size()) != M.nnz) {
        set_error("the system's matrix does not have the 7-point pattern of this grid");
        return SSG_E_INVALID;
    }
    // every local entry (row l2g[r], column l2g[off + lcol]) must sit at the
    // input position the pattern gives it
    for (int32_t s = 0; s < M.P; ++s)
        for (int64_t r = M.off[s]; r < M.off[s + 1]; ++r) {
            const int64_t gi = M.l2g[r];
            for (int32_t e = M.lrowptr[r]; e < M.lrowptr[r + 1]; ++e) {
                const int32_t k = M.lsrc[e];
                const int32_t gj = M.l2g[M.off[s] + M.lcol[e]];
                if (k < rp[gi] || k >= rp[gi + 1] || cols[k] != gj) {
                    set_error("the system's matrix does not have the 7-point pattern of this grid");
                    return SSG_E_INVALID;
                }
            }
        }
    if (S->d_growptr) cudaFree(S->d_growptr);
    S->d_growptr = nullptr;
    SSG_CUDA_TRY(cudaMalloc(&S->d_growptr, sizeof(int32_t) * rp.size()));
    SSG_CUDA_TRY(cudaMemcpyAsync(S->d_growptr, rp.data(), sizeof(int32_t) * rp.size(), cudaMemcpyHostToDevice,
                                 S->ctx->stream));
    SSG_CUDA_TRY(cudaStreamSynchronize(S->ctx->stream));
    S->fv7_dims[0] = nx;
    S->fv7_dims[1] = ny;
    S->fv7_dims[2] = nz;
    return SSG_OK;
}

}  // namespace

extern "C" {

const char *ssg_error_string(int status) {
    switch (status) {
        case SSG_OK: return "ok";
        case SSG_E_INVALID: return "invalid argument";
        case SSG_E_OOM: return "out of memory";
        case SSG_E_CUDA: return "CUDA error";
        case SSG_E_BREAKDOWN: return "CG breakdown: (Sp, p) <= 0 or not finite (matrix not SPD)";
        case SSG_E_NOT_CONVERGED: return "not converged within max_iter";
        case SSG_E_TIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

const char *ssg_last_error(void) { return g_last_error.c_str(); }

int ssg_create(ssg_ctx **ctx, int device, void *stream) {
    if (!ctx) {
        set_error("ctx is null");
        return SSG_E_INVALID;
    }
    *ctx = nullptr;
    int ndev = 0;
    SSG_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) {
        set_error("device " + std::to_string(device) + " out of range");
        return SSG_E_INVALID;
    }
    SSG_CUDA_TRY(cudaSetDevice(device));
    ssg_ctx *c = new (std::nothrow) ssg_ctx();
    if (!c) return SSG_E_OOM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        delete c;
        set_error(std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
        return SSG_E_CUDA;
    }
    c->cluster_ctas = pick_cluster_ctas(c->stream);
    *ctx = c;
    return SSG_OK;
}

int ssg_set_stream(ssg_ctx *ctx, void *stream) {
    if (!ctx) return SSG_E_INVALID;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return SSG_OK;
}

int ssg_set_driver(ssg_ctx *ctx, int driver) {
    if (!ctx || (driver != SSG_DRIVER_GRAPH && driver != SSG_DRIVER_HOST)) {
        set_error("bad context or driver");
        return SSG_E_INVALID;
    }
    ctx->driver = driver;
    return SSG_OK;
}

int ssg_set_slice_sort(ssg_ctx *ctx, int32_t window) {
    if (!ctx || window < -1) {
        set_error("ssg_set_slice_sort: null context, or window < -1");
        return SSG_E_INVALID;
    }
    ctx->slice_sort = window;
    return SSG_OK;
}

int ssg_set_cluster_solve(ssg_ctx *ctx, int64_t max_nloc, int32_t ctas) {
    if (!ctx || max_nloc < 0 || (ctas != 0 && ctas != 2 && ctas != 4 && ctas != 8 && ctas != 16)) {
        set_error("ssg_set_cluster_solve: null context, max_nloc < 0, or ctas not 0, 2, 4, 8 or 16");
        return SSG_E_INVALID;
    }
    ctx->cluster_max_n = max_nloc;
    ctx->cluster_ctas_set = ctas;
    return SSG_OK;
}

int ssg_get_cluster_solve(const ssg_ctx *ctx, int64_t *max_nloc, int32_t *ctas) {
    if (!ctx) {
        set_error("ssg_get_cluster_solve: null context");
        return SSG_E_INVALID;
    }
    if (max_nloc) *max_nloc = ctx->cluster_max_n;
    if (ctas) *ctas = ctx->cluster_ctas;
    return SSG_OK;
}

int ssg_set_unroll(ssg_ctx *ctx, int32_t iters) {
    if (!ctx || iters < 1 || iters > 8) {
        set_error("ssg_set_unroll: null context, or iterations per loop pass not in 1..8");
        return SSG_E_INVALID;
    }
    ctx->unroll = iters;
    return SSG_OK;
}

int ssg_set_mixed(ssg_ctx *ctx, double inner_rtol, int32_t max_outer) {
    if (!ctx || !(inner_rtol > 0.0 && inner_rtol < 1.0) || max_outer < 1) {
        set_error("ssg_set_mixed: need 0 < inner_rtol < 1 and max_outer >= 1");
        return SSG_E_INVALID;
    }
    ctx->inner_rtol = inner_rtol;
    ctx->max_outer = max_outer;
    return SSG_OK;
}

int ssg_set_rhs_block(ssg_ctx *ctx, int32_t kmax) {
    if (!ctx || !(kmax == 1 || kmax == 2 || kmax == 4 || kmax == 8 || kmax == 16)) {
        set_error("ssg_set_rhs_block: kmax must be 1, 2, 4, 8 or 16");
        return SSG_E_INVALID;
    }
    ctx->rhs_block = kmax;
    return SSG_OK;
}

int ssg_destroy(ssg_ctx *ctx) {
    if (!ctx) return SSG_OK;
    if (ctx->live_systems > 0) {
        set_error("context still has " + std::to_string(ctx->live_systems) + " live system(s); destroy them first");
        return SSG_E_INVALID;
    }
    delete ctx;
    return SSG_OK;
}

int ssg_partition(ssg_ctx *ctx, int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                  const int32_t *part, int32_t P, ssg_system **sys) {
    if (!sys) {
        set_error("sys is null");
        return SSG_E_INVALID;
    }
    *sys = nullptr;
    ssg_system *S = new (std::nothrow) ssg_system();
    if (!S) return SSG_E_OOM;
    std::string err;
    int rc = build_host_maps(n, rowptr, colidx, val, part, P, S->maps, &err);
    if (rc != SSG_OK) {
        set_error(err);
        delete S;
        return rc;
    }
    S->ctx = ctx;
    if (ctx) {
        ctx->live_systems++;
        S->unroll = ctx->unroll;
        rc = upload(S);
        if (rc != SSG_OK) {
            ssg_system_destroy(S);
            return rc;
        }
    } else {
        // host only: the interior slice layout the row-length rule gives
        // (ssg_get_layout), without a device
        const WorkPlan plan = make_plan(S->maps, 1, {0, S->maps.P}, 0, 0);
        S->slice_slots = plan.slice_slots;
        S->slice_entries = plan.slice_entries;
        S->sorted_subdomains = plan.sorted_subdomains;
        S->max_window = plan.max_window;
        S->iface_slots = plan.iface_slots;
        S->group_slots = plan.group_slots;
        S->iface_groups = !plan.items_g.empty();
    }
    *sys = S;
    return SSG_OK;
}

int ssg_partition_fe(ssg_ctx *ctx, int32_t n, int32_t ne, int32_t nv, const int32_t *elem, const double *kel,
                     const int32_t *epart, int32_t P, ssg_system **sys) {
    if (!sys) {
        set_error("sys is null");
        return SSG_E_INVALID;
    }
    *sys = nullptr;
    ssg_system *S = new (std::nothrow) ssg_system();
    if (!S) return SSG_E_OOM;
    std::string err;
    int rc = build_host_maps_fe(n, ne, nv, elem, kel, epart, P, S->maps, &err);
    if (rc != SSG_OK) {
        set_error(err);
        delete S;
        return rc;
    }
    S->ctx = ctx;
    if (ctx) {
        ctx->live_systems++;
        S->unroll = ctx->unroll;
        rc = upload(S);
        if (rc != SSG_OK) {
            ssg_system_destroy(S);
            return rc;
        }
    }
    *sys = S;
    return SSG_OK;
}

namespace {

int pow2_columns(int32_t nrhs) { return nrhs <= 2 ? 2 : nrhs <= 4 ? 4 : nrhs <= 8 ? 8 : 16; }

// A segmented system for a (validated) batch; rhs_off (may be null: packed in
// system order) gives each system's first value in the caller's b and x.
int make_batch(ssg_ctx *ctx, int32_t nsys, const int32_t *sys_node_off, const int32_t *sys_sub_off,
               const int32_t *sys_nrhs, const int64_t *rhs_off, const int32_t *rowptr, const int32_t *colidx,
               const double *val, const int32_t *part, ssg_system **out) {
    const int32_t n = sys_node_off[nsys], P = sys_sub_off[nsys];
    ssg_system *S = new (std::nothrow) ssg_system();
    if (!S) return SSG_E_OOM;
    std::string err;
    int rc = build_host_maps(n, rowptr, colidx, val, part, P, S->maps, &err);
    if (rc != SSG_OK) {
        set_error(err);
        delete S;
        return rc;
    }
    S->seg_sub.assign(sys_sub_off, sys_sub_off + nsys + 1);
    S->seg_node.assign(sys_node_off, sys_node_off + nsys + 1);
    S->seg_nrhs.assign(sys_nrhs, sys_nrhs + nsys);
    S->seg_rhs_off.assign(static_cast<size_t>(nsys), 0);
    int64_t o = 0;
    for (int32_t s = 0; s < nsys; ++s) {
        S->seg_rhs_off[s] = rhs_off ? rhs_off[s] : o;
        o += static_cast<int64_t>(sys_nrhs[s]) * (sys_node_off[s + 1] - sys_node_off[s]);
        S->batch_k = std::max(S->batch_k, sys_nrhs[s]);
    }
    S->ctx = ctx;
    ctx->live_systems++;
    S->unroll = ctx->unroll;
    rc = upload(S);
    if (rc != SSG_OK) {
        ssg_system_destroy(S);
        return rc;
    }
    *out = S;
    return SSG_OK;
}

// The K classes of a batch (see ssg_system::kclass): each class's systems
// cut out of the union, renumbered from 0 in the original order, with their
// original offsets in b and x.
int make_batch_classes(ssg_system *S, const int32_t *rowptr, const int32_t *colidx, const double *val,
                       const int32_t *part) {
    const int32_t nsys = S->nseg;
    std::vector<int32_t> cls(static_cast<size_t>(nsys));
    int kinds = 0;
    for (int32_t s = 0; s < nsys; ++s) {
        cls[s] = log2_of(pow2_columns(S->seg_nrhs[s]));
        kinds |= 1 << cls[s];
    }
    if ((kinds & (kinds - 1)) == 0) return SSG_OK;  // one class: the union is it
    for (int c = 1; c <= 4; ++c) {
        if (!((kinds >> c) & 1)) continue;
        std::vector<int32_t> ids, node_off{0}, sub_off{0}, nrhs, rp{0}, ci, pa;
        std::vector<int64_t> roff;
        std::vector<double> va;
        for (int32_t s = 0; s < nsys; ++s) {
            if (cls[s] != c) continue;
            ids.push_back(s);
            const int32_t n0 = S->seg_node[s], n1 = S->seg_node[s + 1];
            const int32_t shift_n = node_off.back() - n0, shift_p = sub_off.back() - S->seg_sub[s];
            for (int32_t i = n0; i < n1; ++i) {
                for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
                    ci.push_back(colidx[k] + shift_n);
                    va.push_back(val[k]);
                }
                rp.push_back(static_cast<int32_t>(ci.size()));
                pa.push_back(part[i] + shift_p);
            }
            node_off.push_back(node_off.back() + (n1 - n0));
            sub_off.push_back(sub_off.back() + (S->seg_sub[s + 1] - S->seg_sub[s]));
            nrhs.push_back(S->seg_nrhs[s]);
            roff.push_back(S->seg_rhs_off[s]);
        }
        // each class has a context of its own (a copy of the batch's, with
        // its own stream) so that the classes' solves can overlap
        ssg_ctx *cc = new (std::nothrow) ssg_ctx(*S->ctx);
        if (!cc) return SSG_E_OOM;
        cc->live_systems = 0;
        cudaError_t e = cudaStreamCreateWithFlags(&cc->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete cc;
            set_error(std::string("cudaStreamCreateWithFlags: ") + cudaGetErrorString(e));
            return SSG_E_CUDA;
        }
        ssg_system *C = nullptr;
        const int rc = make_batch(cc, static_cast<int32_t>(ids.size()), node_off.data(), sub_off.data(),
                                  nrhs.data(), roff.data(), rp.data(), ci.data(), va.data(), pa.data(), &C);
        if (rc != SSG_OK) {
            cudaStreamDestroy(cc->stream);
            delete cc;
            return rc;
        }
        C->own_ctx = cc;
        S->kclass.push_back(C);
        S->kclass_sys.push_back(std::move(ids));
    }
    return SSG_OK;
}

}  // namespace

int ssg_partition_batch(ssg_ctx *ctx, int32_t nsys, const int32_t *sys_node_off, const int32_t *sys_sub_off,
                        const int32_t *sys_nrhs, const int32_t *rowptr, const int32_t *colidx, const double *val,
                        const int32_t *part, ssg_system **sys) {
    if (!sys) {
        set_error("sys is null");
        return SSG_E_INVALID;
    }
    *sys = nullptr;
    if (!ctx || nsys < 1 || !sys_node_off || !sys_sub_off || !sys_nrhs) {
        set_error("batch: need a context, nsys >= 1 and the per-system tables");
        return SSG_E_INVALID;
    }
    if (sys_node_off[0] != 0 || sys_sub_off[0] != 0) {
        set_error("batch: node and subdomain offsets must start at 0");
        return SSG_E_INVALID;
    }
    for (int32_t s = 0; s < nsys; ++s)
        if (sys_node_off[s + 1] <= sys_node_off[s] || sys_sub_off[s + 1] <= sys_sub_off[s] || sys_nrhs[s] < 1 ||
            sys_nrhs[s] > kMaxRhs) {
            set_error("batch: every system needs >= 1 node, >= 1 subdomain and 1..16 right-hand sides");
            return SSG_E_INVALID;
        }
    const int32_t n = sys_node_off[nsys], P = sys_sub_off[nsys];
    {
        // the union's CSR is validated by the partitioner below; here only
        // what indexing it for the checks needs
        if (!rowptr || !colidx || !val || !part || n < 1 || P < 1 || rowptr[0] != 0) {
            set_error("batch: null or empty CSR / partition arrays");
            return SSG_E_INVALID;
        }
        for (int32_t i = 0; i < n; ++i)
            if (rowptr[i + 1] < rowptr[i]) {
                set_error("batch: row pointers decrease");
                return SSG_E_INVALID;
            }
    }
    int rc = SSG_OK;
    // the union must be block diagonal and every system's subdomains its own
    for (int32_t s = 0; s < nsys && rc == SSG_OK; ++s)
        for (int32_t i = sys_node_off[s]; i < sys_node_off[s + 1] && rc == SSG_OK; ++i) {
            if (part[i] < sys_sub_off[s] || part[i] >= sys_sub_off[s + 1]) rc = SSG_E_INVALID;
            for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
                if (colidx[k] < sys_node_off[s] || colidx[k] >= sys_node_off[s + 1]) rc = SSG_E_INVALID;
        }
    if (rc != SSG_OK) {
        set_error("batch: a node's subdomain lies outside its system's range, or an entry couples two systems");
        return rc;
    }
    ssg_system *S = nullptr;
    rc = make_batch(ctx, nsys, sys_node_off, sys_sub_off, sys_nrhs, nullptr, rowptr, colidx, val, part, &S);
    if (rc != SSG_OK) return rc;
    rc = make_batch_classes(S, rowptr, colidx, val, part);
    if (rc != SSG_OK) {
        ssg_system_destroy(S);
        return rc;
    }
    *sys = S;
    return SSG_OK;
}

}  // extern "C"

namespace {

// capture_into that also returns the node the captured work ends in.
template <typename F>
cudaError_t capture_branch(cudaStream_t cap, cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, F fn, int *rc,
                           cudaGraphNode_t *last) {
    cudaError_t e = cudaStreamBeginCaptureToGraph(cap, g, deps, nullptr, ndeps, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    *rc = fn(cap);
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t *d = nullptr;
    size_t nd = 0;
    cudaError_t e1 = cudaStreamGetCaptureInfo(cap, &st, nullptr, nullptr, &d, nullptr, &nd);
    if (e1 == cudaSuccess) {
        if (nd == 1) *last = d[0];
        else e1 = cudaErrorInvalidValue;
    }
    cudaGraph_t out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &out);
    return e1 != cudaSuccess ? e1 : e2;
}

// One column group's loop as a branch of G (no dependencies): its setup
// kernels and WHILE node, the mixed modes' inner WHILE nested in the outer
// body, each loop with a condition handle of its own (the structure
// build_loop_graph and build_nested_graph give one system).
template <int K, bool PC>
int class_branch(ssg_system *C, cudaGraph_t G, cudaStream_t cap, bool mixed) {
    cudaGraphConditionalHandle h_out;
    SSG_CUDA_TRY(cudaGraphConditionalHandleCreate(&h_out, G, 0u, cudaGraphCondAssignDefault));
    ssg_system::BlockState &B = C->blk;
    int rc = SSG_OK;
    cudaGraphNode_t n_init = nullptr, n_loop = nullptr;
    cudaGraph_t body = nullptr;
    cudaError_t e = capture_branch(
        cap, G, nullptr, 0,
        [&](cudaStream_t c) {
            return mixed ? launch_initB<K, false>(C, c, nullptr, h_out, 1) : launch_initB<K, PC>(C, c, B.p, h_out, 1);
        },
        &rc, &n_init);
    if (e == cudaSuccess && rc == SSG_OK) e = add_while(G, &n_init, h_out, &n_loop, &body);
    if (!mixed) {
        if (e == cudaSuccess && rc == SSG_OK)
            e = capture_into(cap, body, nullptr, 0,
                             [&](cudaStream_t c) { return launch_bodyB64<K, PC>(C, c, h_out, 1); }, &rc);
    } else {
        cudaGraphConditionalHandle h_in;
        cudaGraphNode_t n_iinit = nullptr, n_inner = nullptr;
        cudaGraph_t body_in = nullptr;
        if (e == cudaSuccess && rc == SSG_OK) e = cudaGraphConditionalHandleCreate(&h_in, body, 0u, cudaGraphCondAssignDefault);
        if (e == cudaSuccess && rc == SSG_OK)
            e = capture_branch(cap, body, nullptr, 0,
                               [&](cudaStream_t c) { return launch_inner_initB<K, PC>(C, c, h_in, 1); }, &rc, &n_iinit);
        if (e == cudaSuccess && rc == SSG_OK) e = add_while(body, &n_iinit, h_in, &n_inner, &body_in);
        if (e == cudaSuccess && rc == SSG_OK)
            e = capture_into(cap, body_in, nullptr, 0,
                             [&](cudaStream_t c) { return launch_inner_bodyB<K, PC>(C, c, h_in, 1); }, &rc);
        if (e == cudaSuccess && rc == SSG_OK)
            e = capture_into(cap, body, &n_inner, 1, [&](cudaStream_t c) { return launch_outer_tailB<K>(C, c, h_out, 1); },
                             &rc);
    }
    if (rc == SSG_OK && e != cudaSuccess) {
        set_error(std::string("building a column group's loop: ") + cudaGetErrorString(e));
        rc = SSG_E_CUDA;
    }
    return rc;
}

int class_branch_k(ssg_system *C, cudaGraph_t G, cudaStream_t cap, int mode) {
    const bool mixed = mode == SSG_MIXED || mode == SSG_MIXED_JACOBI;
    const bool pc = mode == SSG_FP64_JACOBI || mode == SSG_MIXED_JACOBI;
    switch (pow2_columns(C->batch_k)) {
        case 2: return pc ? class_branch<2, true>(C, G, cap, mixed) : class_branch<2, false>(C, G, cap, mixed);
        case 4: return pc ? class_branch<4, true>(C, G, cap, mixed) : class_branch<4, false>(C, G, cap, mixed);
        case 8: return pc ? class_branch<8, true>(C, G, cap, mixed) : class_branch<8, false>(C, G, cap, mixed);
        default: return pc ? class_branch<16, true>(C, G, cap, mixed) : class_branch<16, false>(C, G, cap, mixed);
    }
}

int block_pre_k(ssg_system *C, const double *b, double *x, int guess, double rtol, int32_t max_iter, int mode,
                cudaStream_t s, int64_t *launches) {
    switch (pow2_columns(C->batch_k)) {
        case 2: return block_pre<2>(C, 0, b, x, guess, rtol, max_iter, mode, s, launches);
        case 4: return block_pre<4>(C, 0, b, x, guess, rtol, max_iter, mode, s, launches);
        case 8: return block_pre<8>(C, 0, b, x, guess, rtol, max_iter, mode, s, launches);
        default: return block_pre<16>(C, 0, b, x, guess, rtol, max_iter, mode, s, launches);
    }
}

int block_post_k(ssg_system *C, double *x, int mode, cudaStream_t s, int64_t launches) {
    switch (pow2_columns(C->batch_k)) {
        case 2: return block_post<2>(C, 0, x, mode, s, launches);
        case 4: return block_post<4>(C, 0, x, mode, s, launches);
        case 8: return block_post<8>(C, 0, x, mode, s, launches);
        default: return block_post<16>(C, 0, x, mode, s, launches);
    }
}

// The graph of all column groups' loops for one mode (built at its first use,
// after the groups' vectors exist).
int classes_graph(ssg_system *S, int mode) {
    ssg_system::BlockGraph &G = S->classes_graph[mode];
    if (G.exec) return SSG_OK;
    SSG_CUDA_TRY(cudaGraphCreate(&G.g, 0));
    cudaStream_t cap;
    SSG_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    int rc = SSG_OK;
    for (size_t c = 0; c < S->kclass.size() && rc == SSG_OK; ++c) rc = class_branch_k(S->kclass[c], G.g, cap, mode);
    cudaStreamDestroy(cap);
    if (rc == SSG_OK) {
        cudaError_t e = cudaGraphInstantiate(&G.exec, G.g, 0);
        if (e != cudaSuccess) {
            set_error(std::string("instantiating the column groups' graph: ") + cudaGetErrorString(e));
            rc = SSG_E_CUDA;
        }
    }
    if (rc != SSG_OK) {
        if (G.g) cudaGraphDestroy(G.g);
        G = ssg_system::BlockGraph{};
    }
    return rc;
}

// Settings copied to the groups' contexts, their vectors allocated (and
// zeroed on their own streams, waited for), and the one-graph form built for
// this mode.  A failure to build the graph marks the mode: its solves then
// run the groups on their own streams.
int batch_classes_ready(ssg_system *S, int mode) {
    for (ssg_system *C : S->kclass) {
        C->ctx->driver = S->ctx->driver;
        C->ctx->inner_rtol = S->ctx->inner_rtol;
        C->ctx->max_outer = S->ctx->max_outer;
        int rc = ensure_block(C, pow2_columns(C->batch_k));
        if (rc != SSG_OK) return rc;
        SSG_CUDA_TRY(cudaStreamSynchronize(C->ctx->stream));
    }
    if (classes_graph(S, mode) != SSG_OK) {
        // the solve falls back to streams; the failed capture or
        // instantiation left its (non-sticky) error behind, which the next
        // launch check would otherwise report (the message stays set)
        S->classes_graph_refused[mode] = true;
        cudaGetLastError();
        return SSG_E_CUDA;
    }
    return SSG_OK;
}

// K-vector product candidates of ssg_autotune_block: entries loaded at once
// (1 or 2) x slices ahead prefetched into L2 (0, 1, 2).
constexpr int kBlockTuneCands = SSG_TUNE_BLOCK_CANDIDATES;
const int kCandNc[kBlockTuneCands] = {1, 1, 1, 2, 2, 2};
const int kCandAhead[kBlockTuneCands] = {0, 1, 2, 0, 1, 2};

// Times every candidate as the solves launch the product (with the block
// partials of (x, S x)_w, every segment active) and keeps the fastest.
template <typename T, int K>
int tune_spmm(ssg_system *S, int reps, double *us, int32_t *choice) {
    ssg_system::BlockState &B = S->blk;
    const int pi = sizeof(T) == 8 ? 0 : 1, lk = log2_cols(K);
    const T *X;
    T *Y;
    if constexpr (sizeof(T) == 8) {
        X = B.p;
        Y = B.q;
    } else {
        X = B.p32;
        Y = B.q32;
    }
    cudaStream_t st = S->ctx->stream;
    double best = 1e30;
    for (int c = 0; c < kBlockTuneCands; ++c) {
        S->spmm_nc[pi][lk] = static_cast<int8_t>(kCandNc[c]);
        S->spmm_ahead[pi][lk] = static_cast<int8_t>(kCandAhead[c]);
        for (int i = 0; i < 3; ++i) spmm_seg<T, K, true>(S, st, X, Y, B.part_a, nullptr);
        SSG_CUDA_TRY(cudaEventRecord(S->ev0, st));
        for (int i = 0; i < reps; ++i) spmm_seg<T, K, true>(S, st, X, Y, B.part_a, nullptr);
        SSG_CUDA_TRY(cudaEventRecord(S->ev1, st));
        SSG_CUDA_TRY(cudaGetLastError());
        SSG_CUDA_TRY(cudaEventSynchronize(S->ev1));
        float ms = 0.f;
        SSG_CUDA_TRY(cudaEventElapsedTime(&ms, S->ev0, S->ev1));
        us[c] = 1e3 * ms / reps;
        if (us[c] < best) {
            best = us[c];
            *choice = c;
        }
    }
    S->spmm_nc[pi][lk] = static_cast<int8_t>(kCandNc[*choice]);
    S->spmm_ahead[pi][lk] = static_cast<int8_t>(kCandAhead[*choice]);
    return SSG_OK;
}

// Tune one (non-batch, or one column group's) system for K columns; its block
// graphs, which hold the previous launches, are rebuilt on demand.
int tune_block_system(ssg_system *S, int K, int reps, ssg_tune_block *t) {
    int rc = ensure_block(S, K);
    if (rc != SSG_OK) return rc;
    t->k = K;
    for (int c = 0; c < kBlockTuneCands; ++c) {
        t->nc[c] = kCandNc[c];
        t->l2_ahead[c] = kCandAhead[c];
    }
    switch (K) {
        case 2: rc = tune_spmm<double, 2>(S, reps, t->fp64_us, &t->fp64_choice); break;
        case 4: rc = tune_spmm<double, 4>(S, reps, t->fp64_us, &t->fp64_choice); break;
        case 8: rc = tune_spmm<double, 8>(S, reps, t->fp64_us, &t->fp64_choice); break;
        default: rc = tune_spmm<double, 16>(S, reps, t->fp64_us, &t->fp64_choice); break;
    }
    if (rc != SSG_OK) return rc;
    switch (K) {
        case 2: rc = tune_spmm<float, 2>(S, reps, t->fp32_us, &t->fp32_choice); break;
        case 4: rc = tune_spmm<float, 4>(S, reps, t->fp32_us, &t->fp32_choice); break;
        case 8: rc = tune_spmm<float, 8>(S, reps, t->fp32_us, &t->fp32_choice); break;
        default: rc = tune_spmm<float, 16>(S, reps, t->fp32_us, &t->fp32_choice); break;
    }
    if (rc != SSG_OK) return rc;
    SSG_CUDA_TRY(cudaStreamSynchronize(S->ctx->stream));
    destroy_block_graphs(S);
    return SSG_OK;
}

// Single-vector loop graphs hold the operators by value: dropped here, built
// again by the next solve.
void destroy_single_graphs(ssg_system *S) {
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->graph) cudaGraphDestroy(S->graph);
    if (S->exec_pc) cudaGraphExecDestroy(S->exec_pc);
    if (S->graph_pc) cudaGraphDestroy(S->graph_pc);
    S->exec = nullptr;
    S->graph = nullptr;
    S->exec_pc = nullptr;
    S->graph_pc = nullptr;
    for (int i = 0; i < 2; ++i) {
        if (S->exec_m[i]) cudaGraphExecDestroy(S->exec_m[i]);
        if (S->graph_m[i]) cudaGraphDestroy(S->graph_m[i]);
        S->exec_m[i] = nullptr;
        S->graph_m[i] = nullptr;
    }
}

// Point every operator of S (and of its column classes) at the weight codes
// of `mode`; every graph holding the previous operators is dropped.
int apply_weights(ssg_system *S, int mode) {
    SSG_CUDA_TRY(cudaStreamSynchronize(S->ctx->stream));
    const uint8_t *codes = mode == SSG_WEIGHT_OWNER ? S->d_wown : S->d_mult;
    const uint8_t *wsel = mode == SSG_WEIGHT_OWNER ? S->d_wown : nullptr;
    for (DevOp *A : {&S->op, &S->op32, &S->opB64, &S->opB32}) {
        A->mult = codes;
        A->wsel = wsel;
    }
    S->weight_mode = mode;
    destroy_single_graphs(S);
    destroy_block_graphs(S);
    for (ssg_system *C : S->kclass) {
        const int rc = apply_weights(C, mode);
        if (rc != SSG_OK) return rc;
    }
    for (ssg_system::BlockGraph &G : S->classes_graph) {
        if (G.exec) cudaGraphExecDestroy(G.exec);
        if (G.g) cudaGraphDestroy(G.g);
        G = ssg_system::BlockGraph{};
    }
    return SSG_OK;
}

}  // namespace

extern "C" {

int ssg_autotune_block(ssg_system *S, int32_t k, int32_t reps, ssg_tune_block *out) {
    int rc = check_dev(S);
    if (rc != SSG_OK) return rc;
    if (reps <= 0) reps = 20;
    ssg_tune_block t{};
    if (S->kclass.empty()) {
        if (!(k == 2 || k == 4 || k == 8 || k == 16)) {
            set_error("ssg_autotune_block: k must be 2, 4, 8 or 16");
            return SSG_E_INVALID;
        }
        rc = tune_block_system(S, k, reps, &t);
        if (rc != SSG_OK) return rc;
    } else {
        // a batch: every column group for its own K; the group with the most
        // columns is reported
        for (ssg_system *C : S->kclass) {
            ssg_tune_block tc{};
            rc = tune_block_system(C, pow2_columns(C->batch_k), reps, &tc);
            if (rc != SSG_OK) return rc;
            if (tc.k >= t.k) t = tc;
        }
        for (ssg_system::BlockGraph &G : S->classes_graph) {
            if (G.exec) cudaGraphExecDestroy(G.exec);
            if (G.g) cudaGraphDestroy(G.g);
            G = ssg_system::BlockGraph{};
        }
    }
    if (out) *out = t;
    return SSG_OK;
}

int ssg_set_batch_graph(ssg_system *S, int32_t one_graph) {
    if (!S) {
        set_error("null system");
        return SSG_E_INVALID;
    }
    for (bool &r : S->classes_graph_refused) r = one_graph == 0;
    return SSG_OK;
}

int ssg_solve_batch(ssg_system *S, const double *b, double *x, int32_t x_is_guess, double rtol, int32_t max_iter,
                    int32_t mode, ssg_stats *stats) {
    int rc = check_dev(S);
    if (rc != SSG_OK) return rc;
    if (S->batch_k < 1) {
        set_error("not a batch of systems (use ssg_partition_batch)");
        return SSG_E_INVALID;
    }
    if (!b || !x || !(rtol >= 0.0) ||
        (mode != SSG_FP64 && mode != SSG_MIXED && mode != SSG_FP64_JACOBI && mode != SSG_MIXED_JACOBI)) {
        set_error("null b/x, negative rtol, or mode not SSG_FP64 / SSG_MIXED / SSG_FP64_JACOBI / SSG_MIXED_JACOBI");
        return SSG_E_INVALID;
    }
    int32_t nmax = 0;
    for (int32_t s = 0; s < S->nseg; ++s) nmax = std::max(nmax, S->seg_node[s + 1] - S->seg_node[s]);
    if (max_iter <= 0) max_iter = nmax;
    SSG_CUDA_TRY(cudaSetDevice(S->ctx->device));
    if (S->kclass.empty()) {
        rc = solve_batch_k(S, b, x, x_is_guess, rtol, max_iter, mode, stats);
    } else if (S->ctx->driver == SSG_DRIVER_GRAPH && !S->classes_graph_refused[mode] &&
               batch_classes_ready(S, mode) == SSG_OK) {
        // every column group's loop is a branch of one graph, launched once
        // on the context's stream; each group's setup before it and its end
        // after it on the same stream; statistics in (system, right-hand
        // side) order
        std::vector<int64_t> first(static_cast<size_t>(S->nseg) + 1, 0);
        for (int32_t sg = 0; sg < S->nseg; ++sg) first[sg + 1] = first[sg] + S->seg_nrhs[sg];
        cudaStream_t ps = S->ctx->stream;
        std::vector<int64_t> launches(S->kclass.size(), 0);
        for (size_t c = 0; c < S->kclass.size(); ++c) {
            rc = block_pre_k(S->kclass[c], b, x, x_is_guess, rtol, max_iter, mode, ps, &launches[c]);
            if (rc != SSG_OK) return rc;
        }
        SSG_CUDA_TRY(cudaGraphLaunch(S->classes_graph[mode].exec, ps));
        for (size_t c = 0; c < S->kclass.size(); ++c) {
            rc = block_post_k(S->kclass[c], x, mode, ps, launches[c]);
            if (rc != SSG_OK) return rc;
        }
        SSG_CUDA_TRY(cudaStreamSynchronize(ps));
        rc = SSG_OK;
        int64_t all_launches = 0;
        double ms = 0.0;
        for (size_t c = 0; c < S->kclass.size(); ++c) {
            ssg_system *C = S->kclass[c];
            int64_t nst = 0;
            for (int32_t sg : S->kclass_sys[c]) nst += S->seg_nrhs[sg];
            std::vector<ssg_stats> st(static_cast<size_t>(nst));
            const int rc_c = solve_block_finish(C, st.data());
            if (rc_c == SSG_E_CUDA || rc_c == SSG_E_OOM || rc_c == SSG_E_INVALID) return rc_c;
            if (rc_c != SSG_OK && rc == SSG_OK) rc = rc_c;
            if (!st.empty()) {
                all_launches += st[0].kernel_launches;
                ms = std::max(ms, st[0].solve_ms);
            }
            if (stats) {
                size_t o = 0;
                for (int32_t sg : S->kclass_sys[c])
                    for (int32_t j = 0; j < S->seg_nrhs[sg]; ++j) stats[first[sg] + j] = st[o++];
            }
        }
        if (stats)
            for (int64_t t = 0; t < first[S->nseg]; ++t) {
                stats[t].kernel_launches = all_launches;
                stats[t].solve_ms = ms;
            }
    } else {
        // host-loop driver (or a graph driver whose one-graph form could not
        // be built): one solve per column group, each on its own stream, side
        // by side after the work already on the context's stream, which then
        // waits for all of them
        std::vector<int64_t> first(static_cast<size_t>(S->nseg) + 1, 0);
        for (int32_t sg = 0; sg < S->nseg; ++sg) first[sg + 1] = first[sg] + S->seg_nrhs[sg];
        cudaStream_t ps = S->ctx->stream;
        cudaEvent_t fork = nullptr;
        SSG_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        std::vector<cudaEvent_t> join(S->kclass.size(), nullptr);
        cudaError_t e = cudaEventRecord(fork, ps);
        size_t enq = 0;
        int rc_enq = e == cudaSuccess ? SSG_OK : SSG_E_CUDA;
        for (; enq < S->kclass.size() && rc_enq == SSG_OK; ++enq) {
            ssg_system *C = S->kclass[enq];
            ssg_ctx *cc = C->ctx;
            cc->driver = S->ctx->driver;
            cc->inner_rtol = S->ctx->inner_rtol;
            cc->max_outer = S->ctx->max_outer;
            if (cudaStreamWaitEvent(cc->stream, fork, 0) != cudaSuccess ||
                cudaEventCreateWithFlags(&join[enq], cudaEventDisableTiming) != cudaSuccess) {
                rc_enq = SSG_E_CUDA;
                break;
            }
            rc_enq = enqueue_batch_k(C, b, x, x_is_guess, rtol, max_iter, mode);
            if (rc_enq != SSG_OK) break;
        }
        // every class enqueued so far is joined and finished, whatever happened after it
        rc = SSG_OK;
        for (size_t c = 0; c < enq; ++c) {
            ssg_system *C = S->kclass[c];
            if (cudaEventRecord(join[c], C->ctx->stream) != cudaSuccess || cudaStreamWaitEvent(ps, join[c], 0) != cudaSuccess)
                rc_enq = rc_enq == SSG_OK ? SSG_E_CUDA : rc_enq;
        }
        for (size_t c = 0; c < enq; ++c) {
            ssg_system *C = S->kclass[c];
            int64_t nst = 0;
            for (int32_t sg : S->kclass_sys[c]) nst += S->seg_nrhs[sg];
            std::vector<ssg_stats> st(static_cast<size_t>(nst));
            const int rc_c = solve_block_finish(C, st.data());
            if (rc_c == SSG_E_CUDA || rc_c == SSG_E_OOM || rc_c == SSG_E_INVALID) {
                if (rc_enq == SSG_OK) rc_enq = rc_c;
                continue;
            }
            if (rc_c != SSG_OK && rc == SSG_OK) rc = rc_c;
            if (stats) {
                size_t o = 0;
                for (int32_t sg : S->kclass_sys[c])
                    for (int32_t j = 0; j < S->seg_nrhs[sg]; ++j) stats[first[sg] + j] = st[o++];
            }
        }
        for (cudaEvent_t ev : join)
            if (ev) cudaEventDestroy(ev);
        cudaEventDestroy(fork);
        if (rc_enq != SSG_OK) return rc_enq;
        if (stats) {
            // every entry reports the whole batch solve: launches summed over
            // the classes, the duration of the longest class (they overlap)
            int64_t launches = 0;
            double ms = 0.0;
            size_t o = 0;
            for (size_t c = 0; c < S->kclass.size(); ++c) {
                const int32_t sg = S->kclass_sys[c][0];
                launches += stats[first[sg]].kernel_launches;
                ms = std::max(ms, stats[first[sg]].solve_ms);
                for (int32_t t : S->kclass_sys[c]) o += S->seg_nrhs[t];
            }
            for (size_t t = 0; t < o; ++t) {
                stats[t].kernel_launches = launches;
                stats[t].solve_ms = ms;
            }
        }
    }
    if (rc != SSG_OK && rc != SSG_E_CUDA && rc != SSG_E_OOM && rc != SSG_E_INVALID) set_error(ssg_error_string(rc));
    return rc;
}

int ssg_get_layout(const ssg_system *S, int64_t *out) {
    if (!S || !out) {
        set_error("null argument");
        return SSG_E_INVALID;
    }
    out[0] = S->slice_slots;
    out[1] = S->slice_entries;
    out[2] = S->sorted_subdomains;
    out[3] = S->max_window;
    return SSG_OK;
}

int ssg_get_iface_layout(const ssg_system *S, int64_t *out) {
    if (!S || !out) {
        set_error("null argument");
        return SSG_E_INVALID;
    }
    out[0] = S->iface_slots;
    out[1] = S->group_slots;
    out[2] = S->iface_groups ? 1 : 0;
    return SSG_OK;
}

int ssg_get_sizes(const ssg_system *S, ssg_sizes *o) {
    if (!S || !o) {
        set_error("null argument");
        return SSG_E_INVALID;
    }
    o->n = S->maps.n;
    o->P = S->maps.P;
    o->nnz = S->maps.nnz;
    o->nloc = S->maps.nloc;
    o->ngamma = S->maps.ngamma;
    o->max_mult = S->maps.max_mult;
    o->ncopies = S->maps.ncopies;
    return SSG_OK;
}

int ssg_copy_maps(const ssg_system *S, int32_t *off, int32_t *nint, int32_t *l2g, int32_t *mult, int32_t *lrowptr,
                  int32_t *lcol, double *lval, int32_t *gamma, int32_t *iptr, int32_t *icopy, int32_t *own) {
    if (!S) {
        set_error("null system");
        return SSG_E_INVALID;
    }
    const HostMaps &M = S->maps;
    auto cp = [](void *dst, const void *src, size_t bytes) {
        if (dst && bytes) memcpy(dst, src, bytes);
    };
    cp(off, M.off.data(), sizeof(int32_t) * (M.P + 1));
    cp(nint, M.nint.data(), sizeof(int32_t) * M.P);
    cp(l2g, M.l2g.data(), sizeof(int32_t) * M.nloc);
    cp(mult, M.mult.data(), sizeof(int32_t) * M.n);
    cp(lrowptr, M.lrowptr.data(), sizeof(int32_t) * (M.nloc + 1));
    cp(lcol, M.lcol.data(), sizeof(int32_t) * M.nnz);
    cp(lval, M.lval.data(), sizeof(double) * M.nnz);
    cp(gamma, M.gamma.data(), sizeof(int32_t) * M.ngamma);
    cp(iptr, M.iptr.data(), sizeof(int32_t) * (M.ngamma + 1));
    cp(icopy, M.icopy.data(), sizeof(int32_t) * M.ncopies);
    cp(own, M.own.data(), sizeof(int32_t) * M.n);
    return SSG_OK;
}

int ssg_scatter(ssg_system *S, const double *x_glob, double *x_loc) {
    int rc = check_dev(S);
    if (rc != SSG_OK) return rc;
    if (!x_glob || !x_loc) {
        set_error("null vector");
        return SSG_E_INVALID;
    }
    k_scatter<<<grid_for(S->maps.nloc, S->ctx->num_sms), kBlock, 0, S->ctx->stream>>>(S->maps.nloc, S->d_l2g,
                                                                                       x_glob, x_loc);
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

int ssg_gather(ssg_system *S, const double *x_loc, double *x_glob) {
    int rc = check_dev(S);
    if (rc != SSG_OK) return rc;
    if (!x_glob || !x_loc) {
        set_error("null vector");
        return SSG_E_INVALID;
    }
    k_gather<<<grid_for(S->maps.n, S->ctx->num_sms), kBlock, 0, S->ctx->stream>>>(S->maps.n, S->d_own, x_loc,
                                                                                   x_glob);
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

int ssg_spmv_assembled(ssg_system *S, const double *x_loc, double *y_loc, double *xSx_dev) {
    int rc = check_dev(S);
    if (rc != SSG_OK) return rc;
    if (!x_loc || !y_loc || x_loc == y_loc) {
        set_error("x_loc and y_loc must be distinct non-null device vectors");
        return SSG_E_INVALID;
    }
    // without xSx the loop's instance (block partials only); with it the one
    // whose last block sums the partials (a ticket, a few microseconds more)
    if (xSx_dev)
        v64(S)[S->var64].store<<<S->grid_spmv, kSpmvThreads, 0, S->ctx->stream>>>(
            S->op, x_loc, y_loc, S->d_partials, S->d_scal_op, xSx_dev, 0, 0);
    else
        v64(S)[S->var64].part<<<S->grid_spmv, kSpmvThreads, 0, S->ctx->stream>>>(
            S->op, x_loc, y_loc, S->d_partials, S->d_scal_op, nullptr, 0, 0);
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

int ssg_spmv_assembled_f32(ssg_system *S, const float *x_loc, float *y_loc, double *xSx_dev) {
    int rc = check_dev(S);
    if (rc != SSG_OK) return rc;
    if (!x_loc || !y_loc || x_loc == y_loc) {
        set_error("x_loc and y_loc must be distinct non-null device vectors");
        return SSG_E_INVALID;
    }
    if (xSx_dev)
        kSpmv32Variants[S->var32].store<<<S->grid_spmv32, kSpmvThreads, 0, S->ctx->stream>>>(
            S->op32, x_loc, y_loc, S->d_partials, S->d_scal_op, xSx_dev, 0, 0);
    else
        kSpmv32Variants[S->var32].part<<<S->grid_spmv32, kSpmvThreads, 0, S->ctx->stream>>>(
            S->op32, x_loc, y_loc, S->d_partials, S->d_scal_op, nullptr, 0, 0);
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

int ssg_autotune(ssg_system *S, int32_t reps, ssg_tune *out) {
    int rc = check_dev(S);
    if (rc != SSG_OK) return rc;
    if (reps <= 0) reps = 20;
    cudaStream_t st = S->ctx->stream;
    ssg_tune t{};
    // FP64 instances on the solver's work vectors (zero-initialised, finite),
    // as the loop launches them (block partials, no last-block sum)
    double best = 1e30;
    for (int v = 0; v < kSpmvVariants; ++v) {
        const SpmvVariant<double> &V = v64(S)[v];
        DevOp A = S->op;
        A.warp_range = S->range_bps[V.bps];
        const int grid = S->grid_bps[V.bps];
        for (int i = 0; i < 3; ++i)
            V.part<<<grid, kSpmvThreads, 0, st>>>(A, S->d_p, S->d_q, S->d_partials, S->d_scal_op, nullptr, 0, 0);
        SSG_CUDA_TRY(cudaEventRecord(S->ev0, st));
        for (int i = 0; i < reps; ++i)
            V.part<<<grid, kSpmvThreads, 0, st>>>(A, S->d_p, S->d_q, S->d_partials, S->d_scal_op, nullptr, 0, 0);
        SSG_CUDA_TRY(cudaEventRecord(S->ev1, st));
        SSG_CUDA_TRY(cudaGetLastError());
        SSG_CUDA_TRY(cudaEventSynchronize(S->ev1));
        float ms = 0.f;
        SSG_CUDA_TRY(cudaEventElapsedTime(&ms, S->ev0, S->ev1));
        t.fp64_blocks_per_sm[v] = V.bps;
        t.fp64_l2_ahead[v] = V.ahead;
        t.fp64_us[v] = 1e3 * ms / reps;
        if (t.fp64_us[v] < best) {
            best = t.fp64_us[v];
            t.fp64_choice = v;
        }
    }
    best = 1e30;
    for (int v = 0; v < kSpmvVariants; ++v) {
        const SpmvVariant<float> &V = kSpmv32Variants[v];
        DevOp A = S->op32;
        A.warp_range = S->range_bps32[V.bps];
        const int grid = S->grid_bps32[V.bps];
        for (int i = 0; i < 3; ++i)
            V.part<<<grid, kSpmvThreads, 0, st>>>(A, S->d_p32, S->d_q32, S->d_partials, S->d_scal_op, nullptr, 0, 0);
        SSG_CUDA_TRY(cudaEventRecord(S->ev0, st));
        for (int i = 0; i < reps; ++i)
            V.part<<<grid, kSpmvThreads, 0, st>>>(A, S->d_p32, S->d_q32, S->d_partials, S->d_scal_op, nullptr, 0, 0);
        SSG_CUDA_TRY(cudaEventRecord(S->ev1, st));
        SSG_CUDA_TRY(cudaGetLastError());
        SSG_CUDA_TRY(cudaEventSynchronize(S->ev1));
        float ms = 0.f;
        SSG_CUDA_TRY(cudaEventElapsedTime(&ms, S->ev0, S->ev1));
        t.fp32_blocks_per_sm[v] = V.bps;
        t.fp32_l2_ahead[v] = V.ahead;
        t.fp32_us[v] = 1e3 * ms / reps;
        if (t.fp32_us[v] < best) {
            best = t.fp32_us[v];
            t.fp32_choice = v;
        }
    }
    // adopt the choices; graphs holding the previous instances are rebuilt on demand
    SSG_CUDA_TRY(cudaStreamSynchronize(st));
    S->var64 = t.fp64_choice;
    S->var32 = t.fp32_choice;
    S->op.warp_range = S->range_bps[kSpmv64Variants[S->var64].bps];
    S->grid_spmv = S->grid_bps[kSpmv64Variants[S->var64].bps];
    S->op32.warp_range = S->range_bps32[kSpmv32Variants[S->var32].bps];
    S->grid_spmv32 = S->grid_bps32[kSpmv32Variants[S->var32].bps];
    destroy_single_graphs(S);
    if (out) *out = t;
    return SSG_OK;
}

int ssg_set_weights(ssg_system *S, int32_t mode) {
    int rc = check_dev(S);
    if (rc != SSG_OK) return rc;
    if (mode != SSG_WEIGHT_INV_MULT && mode != SSG_WEIGHT_OWNER) {
        set_error("ssg_set_weights: mode must be SSG_WEIGHT_INV_MULT or SSG_WEIGHT_OWNER");
        return SSG_E_INVALID;
    }
    return apply_weights(S, mode);
}

int ssg_spmm_assembled(ssg_system *S, int32_t k, const double *x_loc, double *y_loc) {
    return spmm_checked<double>(S, k, x_loc, y_loc);
}

int ssg_spmm_assembled_f32(ssg_system *S, int32_t k, const float *x_loc, float *y_loc) {
    return spmm_checked<float>(S, k, x_loc, y_loc);
}

int ssg_wdot(ssg_system *S, const double *u, const double *v, double *result_dev) {
    int rc = check_dev(S);
    if (rc != SSG_OK) return rc;
    if (!u || !v || !result_dev) {
        set_error("null argument");
        return SSG_E_INVALID;
    }
    k_wdot<false><<<S->grid_vec, kBlock, 0, S->ctx->stream>>>(S->maps.nloc, u, v, S->op.mult, S->op.wtab,
                                                               S->d_partials, S->d_scal_op, result_dev);
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

int ssg_set_values(ssg_system *S, const double *val) {
    int rc = check_dev(S);
    if (rc != SSG_OK) return rc;
    if (!val) {
        set_error("null values");
        return SSG_E_INVALID;
    }
    if (S->maps.lsrc.empty()) {
        set_error("a system built from elements has no input-CSR values to replace");
        return SSG_E_INVALID;
    }
    if (!S->kclass.empty()) {
        set_error("a batch solved in several column classes takes its values at partition time only");
        return SSG_E_INVALID;
    }
    cudaStream_t st = S->ctx->stream;
    const int ns = S->ctx->num_sms;
    k_gather_vals<<<grid_for(S->maps.nnz, ns), kBlock, 0, st>>>(S->maps.nnz, S->d_vmap, val,
                                                                const_cast<double *>(S->op.val),
                                                                const_cast<float *>(S->op.val32));
    if (S->n_ival)
        k_gather_vals<<<grid_for(S->n_ival, ns), kBlock, 0, st>>>(S->n_ival, S->d_imap, val,
                                                                  const_cast<double *>(S->op.ival),
                                                                  const_cast<float *>(S->op.ival32));
    if (S->n_sval)
        k_gather_vals<<<grid_for(S->n_sval, ns), kBlock, 0, st>>>(S->n_sval, S->d_smap, val,
                                                                  const_cast<double *>(S->op.sval),
                                                                  const_cast<float *>(S->op.sval32));
    if (S->n_gval)
        k_gather_vals<<<grid_for(S->n_gval, ns), kBlock, 0, st>>>(S->n_gval, S->d_gmap, val,
                                                                  const_cast<double *>(S->op.gval),
                                                                  const_cast<float *>(S->op.gval32));
    SSG_CUDA_TRY(cudaMemsetAsync(S->d_diag_bad, 0, sizeof(int), st));
    k_dinv<<<grid_for(S->maps.nloc, ns), kBlock, 0, st>>>(S->maps.nloc, S->d_dmap, S->op.val, S->d_dinv, S->d_dinv32,
                                                           S->d_diag_bad);
    S->diag_state = -1;
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

int ssg_pattern_grad(ssg_system *S, int32_t k, const double *lam, const double *x, double *g) {
    int rc = check_dev(S);
    if (rc != SSG_OK) return rc;
    if (k < 1 || !lam || !x || !g) {
        set_error("bad k or null vector");
        return SSG_E_INVALID;
    }
    if (S->maps.lsrc.empty()) {
        set_error("a system built from elements has no input-CSR entries");
        return SSG_E_INVALID;
    }
    k_pattern_grad<<<grid_for(S->maps.nloc, S->ctx->num_sms), kBlock, 0, S->ctx->stream>>>(
        S->maps.nloc, S->maps.n, k, S->op.rowptr, S->op.col, S->d_l2g, S->d_vmap, lam, x, g);
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

int ssg_fv7_values(ssg_system *S, int32_t nx, int32_t ny, int32_t nz, const double *logk, double *val) {
    int rc = check_dev(S);
    if (rc != SSG_OK) return rc;
    if (!logk || !val) {
        set_error("null vector");
        return SSG_E_INVALID;
    }
    rc = check_fv7(S, nx, ny, nz);
    if (rc != SSG_OK) return rc;
    k_fv7_values<<<grid_for(S->maps.n, S->ctx->num_sms), kBlock, 0, S->ctx->stream>>>(Fv7Grid{nx, ny, nz}, logk,
                                                                                       S->d_growptr, val);
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

int ssg_fv7_adjoint(ssg_system *S, int32_t nx, int32_t ny, int32_t nz, const double *logk, const double *gval,
                    double *glogk) {
    int rc = check_dev(S);
    if (rc != SSG_OK) return rc;
    if (!logk || !gval || !glogk) {
        set_error("null vector");
        return SSG_E_INVALID;
    }
    rc = check_fv7(S, nx, ny, nz);
    if (rc != SSG_OK) return rc;
    k_fv7_adjoint<<<grid_for(S->maps.n, S->ctx->num_sms), kBlock, 0, S->ctx->stream>>>(Fv7Grid{nx, ny, nz}, logk,
                                                                                        S->d_growptr, gval, glogk);
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

int ssg_solve(ssg_system *S, int32_t k, const double *b, double *x, int32_t x_is_guess, double rtol,
              int32_t max_iter, int32_t mode, ssg_stats *stats) {
    int rc = check_dev(S);
    if (rc != SSG_OK) return rc;
    if (k <= 0 || !b || !x || !(rtol >= 0.0)) {
        set_error("bad k, null b/x, or negative rtol");
        return SSG_E_INVALID;
    }
    if (mode != SSG_FP64 && mode != SSG_MIXED && mode != SSG_FP64_JACOBI && mode != SSG_MIXED_JACOBI) {
        set_error("mode must be SSG_FP64, SSG_MIXED, SSG_FP64_JACOBI or SSG_MIXED_JACOBI");
        return SSG_E_INVALID;
    }
    if (max_iter <= 0) max_iter = S->maps.n;
    SSG_CUDA_TRY(cudaSetDevice(S->ctx->device));
    int first_bad = SSG_OK;
    const int kb = std::max(1, S->ctx->rhs_block);
    for (int32_t j = 0; j < k;) {
        const int nr = std::min<int>(k - j, kb);
        const size_t o = static_cast<size_t>(j) * S->maps.n;
        ssg_stats *sj = stats ? stats + j : nullptr;
        rc = nr == 1 ? solve_one(S, b + o, x + o, x_is_guess, rtol, max_iter, mode, sj)
                     : solve_block_k(S, nr, b + o, x + o, x_is_guess, rtol, max_iter, mode, sj);
        if (rc == SSG_E_CUDA || rc == SSG_E_OOM || rc == SSG_E_INVALID) return rc;
        if (rc != SSG_OK && first_bad == SSG_OK) first_bad = rc;
        j += nr;
    }
    if (first_bad != SSG_OK) set_error(ssg_error_string(first_bad));
    return first_bad;
}

int ssg_solve_host(ssg_system *S, int32_t k, const double *b_host, double *x_host, int32_t x_is_guess, double rtol,
                   int32_t max_iter, int32_t mode, ssg_stats *stats) {
    int rc = check_dev(S);
    if (rc != SSG_OK) return rc;
    if (k <= 0 || !b_host || !x_host) {
        set_error("bad k or null b/x");
        return SSG_E_INVALID;
    }
    if (!(rtol >= 0.0) || (mode != SSG_FP64 && mode != SSG_MIXED && mode != SSG_FP64_JACOBI &&
                           mode != SSG_MIXED_JACOBI)) {
        set_error("negative rtol or bad mode");
        return SSG_E_INVALID;
    }
    cudaStream_t s = S->ctx->stream;
    const int kb = std::max(1, S->ctx->rhs_block);
    int first_bad = SSG_OK;
    for (int32_t j = 0; j < k;) {
        const int nr = std::min<int>(k - j, kb);
        const size_t o = static_cast<size_t>(j) * S->maps.n;
        const size_t nb = sizeof(double) * S->maps.n * nr;
        double *bg = S->d_bg, *xg = S->d_xg;
        if (nr > 1) {
            rc = ensure_block(S, nr <= 2 ? 2 : nr <= 4 ? 4 : nr <= 8 ? 8 : 16);
            if (rc != SSG_OK) return rc;
            bg = S->blk.bg;
            xg = S->blk.xg;
        }
        SSG_CUDA_TRY(cudaMemcpyAsync(bg, b_host + o, nb, cudaMemcpyHostToDevice, s));
        if (x_is_guess) SSG_CUDA_TRY(cudaMemcpyAsync(xg, x_host + o, nb, cudaMemcpyHostToDevice, s));
        rc = ssg_solve(S, nr, bg, xg, x_is_guess, rtol, max_iter, mode, stats ? stats + j : nullptr);
        if (rc == SSG_E_CUDA || rc == SSG_E_OOM || rc == SSG_E_INVALID) return rc;
        if (rc != SSG_OK && first_bad == SSG_OK) first_bad = rc;
        SSG_CUDA_TRY(cudaMemcpyAsync(x_host + o, xg, nb, cudaMemcpyDeviceToHost, s));
        j += nr;
    }
    SSG_CUDA_TRY(cudaStreamSynchronize(s));
    return first_bad;
}

int ssg_system_destroy(ssg_system *S) {
    if (!S) return SSG_OK;
    for (ssg_system::BlockGraph &G : S->classes_graph) {
        if (G.exec) cudaGraphExecDestroy(G.exec);
        if (G.g) cudaGraphDestroy(G.g);
    }
    for (ssg_system *C : S->kclass) ssg_system_destroy(C);  // each frees its own context
    S->kclass.clear();
    if (S->ctx) cudaSetDevice(S->ctx->device);
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->graph) cudaGraphDestroy(S->graph);
    if (S->exec_pc) cudaGraphExecDestroy(S->exec_pc);
    if (S->graph_pc) cudaGraphDestroy(S->graph_pc);
    for (int i = 0; i < 2; ++i) {
        if (S->exec_m[i]) cudaGraphExecDestroy(S->exec_m[i]);
        if (S->graph_m[i]) cudaGraphDestroy(S->graph_m[i]);
    }
    if (S->ev0) cudaEventDestroy(S->ev0);
    if (S->ev1) cudaEventDestroy(S->ev1);
    free_block(S);
    if (S->d_growptr) cudaFree(S->d_growptr);
    if (S->arena) {
        if (S->ctx && S->ctx->stream) cudaStreamSynchronize(S->ctx->stream);
        cudaFree(S->arena);
    }
    if (S->h_states) cudaFreeHost(S->h_states);
    if (S->ctx) S->ctx->live_systems--;
    ssg_ctx *own = S->own_ctx;
    delete S;
    if (own) {
        cudaStreamSynchronize(own->stream);
        cudaStreamDestroy(own->stream);
        delete own;
    }
    return SSG_OK;
}

}  // extern "C"
