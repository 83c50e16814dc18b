// Band-row and band-column splittings (Sections 2.1 and 2.2, Algorithms 1 and
// 2) as comparison operators for the sub-structured product.
//
// On one GPU every band shares one memory, so the device keeps A once: the
// band-row bands are row ranges of A and the band-column bands are, in every
// row, the runs of entries whose columns fall in one band's column range
// (columns are sorted, so a band's entries of a row are contiguous).  One
// kernel computes all bands' products:
//   band-row:    y_i = sum_k A_ik x_k, the row summed left to right;
//   band-column: y_i = sum over bands p (ascending) of the band's partial sum
//                of row i (left to right inside the band).
// Three kernel shapes, picked by the mean row length (rule_for) or by
// measurement (ssg_band_autotune):
//   staged   a tile of whole rows (at most one per thread, at most kTileNnz
//            entries) is copied to shared memory by two bulk asynchronous
//            copies (values, column ids) while the previous tile is being
//            reduced; each thread then sums its row from shared memory.
//            Loads of A are whole contiguous ranges, the order is left to right.
//   1 lane   one thread per row reading A from global memory, left to right.
//   V lanes  V = 2..32 lanes per row take strided entries, then a fixed
//            shuffle tree adds the lanes' partial sums (band-row only).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "ssg_ctx.h"
#include "ssg_internal.h"

namespace ssg {
namespace {

constexpr int kBandBlock = 256;          // threads per block; a staged tile holds at most one row per thread
constexpr int kTileNnz = 2048;           // entries a staged tile holds
constexpr int kValBuf = (kTileNnz + 2) * 8;   // bytes: the tile's values, widened to 16-byte boundaries
constexpr int kColBuf = (kTileNnz + 8) * 4;   // bytes: the tile's column ids, widened likewise
constexpr int kStageBytes = kValBuf + kColBuf;
constexpr int kStagedSmem = 2 * kStageBytes;  // two stages
constexpr int kStagedBlocksPerSM = 4;
constexpr int kVecBlocksPerSM = 8;
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // bounded mbarrier wait: one second of global time
constexpr uint32_t kWaitMaxTries = 1u << 26;      // and a cap on the tries should the timer not advance
static_assert(kValBuf % 16 == 0 && kColBuf % 16 == 0, "stage buffers keep 16-byte alignment");

struct BandDev {
    int32_t n, nb, q;              // q = floor(n / nb): columns per band (band-column)
    const int32_t *rowptr;
    const int32_t *col;
    const double *val;
    const int32_t *tile;           // [ntiles + 1] first row of each staged tile
    int32_t ntiles;
    int *err;                      // host-mapped flag: set when a bounded wait ran out
};

// Band of column c and the end of its column range (band-column splitting).
// (An FP32 first guess corrected by 64-bit multiplies measured slower than
// this integer division: 61 us against 53 us on the 128^3 matrix.)
__device__ __forceinline__ int32_t band_end(const BandDev &A, int32_t c) {
    const int32_t p = min(c / A.q, A.nb - 1);
    return p == A.nb - 1 ? A.n : (p + 1) * A.q;
}

// Row sum left to right; with COLSEG the row is cut at band boundaries and the
// bands' partial sums are added in ascending band order.  Entries go in
// groups of kRowUnroll: the group's column ids, values and x gathers are all
// issued before its multiply-adds, which then run in entry order.
constexpr int kRowUnroll = 4;
template <bool COLSEG, typename ColAt, typename ValAt>
__device__ __forceinline__ double row_sum(const BandDev &A, int32_t k0, int32_t k1, const double *__restrict__ x,
                                          ColAt colat, ValAt valat) {
    double s = 0.0, yv = 0.0;
    int32_t bend = -1;
    auto add = [&](int32_t c, double v, double xv) {
        if (COLSEG && c >= bend) {
            yv += s;
            s = 0.0;
            bend = band_end(A, c);
        }
        s = fma(v, xv, s);
    };
    int32_t k = k0;
    for (; k + kRowUnroll <= k1; k += kRowUnroll) {
        int32_t c[kRowUnroll];
        double v[kRowUnroll], xv[kRowUnroll];
#pragma unroll
        for (int u = 0; u < kRowUnroll; ++u) {
            c[u] = colat(k + u);
            v[u] = valat(k + u);
        }
#pragma unroll
        for (int u = 0; u < kRowUnroll; ++u) xv[u] = __ldg(x + c[u]);
#pragma unroll
        for (int u = 0; u < kRowUnroll; ++u) add(c[u], v[u], xv[u]);
    }
    for (; k < k1; ++k) {
        const int32_t c = colat(k);
        add(c, valat(k), __ldg(x + c));
    }
    return COLSEG ? yv + s : s;
}

// ---------------------------------------------------------------- staged --
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase with the given parity; false when the limit (one second,
// or kWaitMaxTries tries) ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < kWaitMaxTries; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && global_ns() - t0 > kWaitLimitNs) return false;
    }
    return false;
}

// Entry range [e0, e1) of a tile widened to 16-byte boundaries: values from
// va (2 doubles), column ids from ca (4 ints); at least 16 bytes each.
struct Stage {
    int32_t e0, e1, va, ca;
    uint32_t vbytes, cbytes;
};
__device__ __forceinline__ Stage stage_of(const BandDev &A, int32_t t) {
    Stage g;
    g.e0 = A.rowptr[A.tile[t]];
    g.e1 = A.rowptr[A.tile[t + 1]];
    g.va = g.e0 & ~1;
    g.ca = g.e0 & ~3;
    const int32_t va1 = max((g.e1 + 1) & ~1, g.va + 2);
    const int32_t ca1 = max((g.e1 + 3) & ~3, g.ca + 4);
    g.vbytes = static_cast<uint32_t>(va1 - g.va) * 8u;
    g.cbytes = static_cast<uint32_t>(ca1 - g.ca) * 4u;
    return g;
}
__device__ __forceinline__ bool staged_tile(const Stage &g) { return g.e1 - g.e0 <= kTileNnz; }

template <bool COLSEG>
__global__ void __launch_bounds__(kBandBlock, kStagedBlocksPerSM)
    k_band_staged(BandDev A, const double *__restrict__ x, double *__restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase[2] = {0u, 0u};
    bool issued[2] = {false, false};
    auto issue = [&](int32_t t, int b) {
        const Stage g = stage_of(A, t);
        if (!staged_tile(g)) return false;
        if (threadIdx.x == 0) {
            unsigned char *buf = smem + b * kStageBytes;
            mbar_expect_tx(&bar[b], g.vbytes + g.cbytes);
            bulk_copy_g2s(buf, A.val + g.va, g.vbytes, &bar[b]);
            bulk_copy_g2s(buf + kValBuf, A.col + g.ca, g.cbytes, &bar[b]);
        }
        return true;
    };
    int b = 0;
    int32_t t = blockIdx.x;
    if (t < A.ntiles) issued[0] = issue(t, 0);
    while (t < A.ntiles) {
        const int32_t tn = t + gridDim.x;
        if (tn < A.ntiles) issued[b ^ 1] = issue(tn, b ^ 1);
        const Stage g = stage_of(A, t);
        const int32_t r0 = A.tile[t], r1 = A.tile[t + 1];
        if (issued[b]) {
            const bool ok = mbar_wait_bounded(&bar[b], phase[b]);
            phase[b] ^= 1u;
            issued[b] = false;
            if (__syncthreads_or(!ok)) {
                // give the copies in flight a last bounded wait, flag the error and leave
                mbar_wait_bounded(&bar[b], phase[b] ^ 1u);
                if (issued[b ^ 1]) mbar_wait_bounded(&bar[b ^ 1], phase[b ^ 1]);
                if (threadIdx.x == 0) atomicExch(A.err, 1);
                return;
            }
            const double *sv = reinterpret_cast<const double *>(smem + b * kStageBytes);
            const int32_t *sc = reinterpret_cast<const int32_t *>(smem + b * kStageBytes + kValBuf);
            const int32_t row = r0 + threadIdx.x;
            if (row < r1)
                y[row] = row_sum<COLSEG>(A, A.rowptr[row], A.rowptr[row + 1], x,
                                         [&](int32_t k) { return sc[k - g.ca]; },
                                         [&](int32_t k) { return sv[k - g.va]; });
        } else if (threadIdx.x == 0) {
            // a row longer than a tile: read from global memory, same order
            for (int32_t row = r0; row < r1; ++row)
                y[row] = row_sum<COLSEG>(A, A.rowptr[row], A.rowptr[row + 1], x,
                                         [&](int32_t k) { return __ldg(A.col + k); },
                                         [&](int32_t k) { return __ldg(A.val + k); });
        }
        __syncthreads();  // every thread is done with stage b before it is refilled
        t = tn;
        b ^= 1;
    }
}

// The bounded wait's failure path, on its own: an mbarrier phase that
// nothing completes (no arrival, no copy issued), waited for by one warp with
// the staged kernel's bound; the timeout raises the error flag.  Nothing is
// in flight, so the context stays usable.
__global__ void k_band_wait_probe(int *err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(err, 1);
}

// ---------------------------------------------------------------- lanes --
template <int V, bool COLSEG>
__global__ void __launch_bounds__(kBandBlock) k_band_lanes(BandDev A, const double *__restrict__ x,
                                                           double *__restrict__ y) {
    constexpr int kRowsPerWarp = 32 / V;
    const int lane32 = threadIdx.x & 31;
    const int sub = lane32 & (V - 1);
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * kBandBlock + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * kBandBlock) >> 5;
    for (int64_t w0 = warp * kRowsPerWarp; w0 < A.n; w0 += nwarps * kRowsPerWarp) {
        const int64_t row = w0 + lane32 / V;
        const bool valid = row < A.n;
        double s = 0.0;
        if constexpr (V == 1) {
            if (valid)
                y[row] = row_sum<COLSEG>(A, A.rowptr[row], A.rowptr[row + 1], x,
                                         [&](int32_t k) { return __ldg(A.col + k); },
                                         [&](int32_t k) { return __ldg(A.val + k); });
            continue;
        }
        if (valid) {
            const int32_t k1 = A.rowptr[row + 1];
            for (int32_t k = A.rowptr[row] + sub; k < k1; k += V) s = fma(__ldg(A.val + k), __ldg(x + __ldg(A.col + k)), s);
        }
#pragma unroll
        for (int o = V / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, V);
        if (valid && sub == 0) y[row] = s;
    }
}

}  // namespace
}  // namespace ssg

using namespace ssg;

struct ssg_band {
    ssg_ctx *ctx = nullptr;
    int32_t kind = 0, n = 0, nb = 0;
    int64_t nnz = 0;
    std::vector<int32_t> rowptr, colidx;  // host copy of A, for ssg_band_get
    std::vector<double> val;
    void *arena = nullptr;
    int *h_err = nullptr;                 // host-mapped error flag
    BandDev dev{};
    int32_t variant = 1;
    int32_t rule_variant = 1;
};

namespace {

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

bool variant_valid(const ssg_band *B, int32_t v) {
    if (v == SSG_BAND_STAGED || v == 1) return true;
    if (B->kind == SSG_BAND_COL) return false;
    return v == 2 || v == 4 || v == 8 || v == 16 || v == 32;
}

// The row-length rule: one thread per row for short rows (mean length <= 8;
// measured on the 128^3 matrix: 39 us against 57 us for the staged kernel,
// which holds two stages of whole rows in shared memory and so runs at half
// the occupancy, and 74 us for two lanes per row), else lanes per row = the
// power of two >= half the mean length (2..32).  Band-column: one thread per
// row.
int32_t rule_for(int32_t kind, int32_t n, int64_t nnz) {
    const double mean = n > 0 ? static_cast<double>(nnz) / n : 0.0;
    if (kind == SSG_BAND_COL || mean <= 8.0) return 1;
    int32_t v = 2;
    while (v < 32 && v < mean / 2.0) v *= 2;
    return v;
}

int launch_variant(ssg_band *B, int32_t v, const double *x, double *y) {
    cudaStream_t st = B->ctx->stream;
    const int sms = B->ctx->num_sms;
    const bool col = B->kind == SSG_BAND_COL;
    if (v == SSG_BAND_STAGED) {
        const int grid = std::max(1, std::min(B->dev.ntiles, sms * kStagedBlocksPerSM));
        if (col)
            k_band_staged<true><<<grid, kBandBlock, kStagedSmem, st>>>(B->dev, x, y);
        else
            k_band_staged<false><<<grid, kBandBlock, kStagedSmem, st>>>(B->dev, x, y);
    } else {
        const int64_t warps = (static_cast<int64_t>(B->n) * v + 31) / 32;
        const int64_t want = (warps * 32 + kBandBlock - 1) / kBandBlock;
        const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, sms * kVecBlocksPerSM)));
        switch (v) {
            case 1:
                if (col)
                    k_band_lanes<1, true><<<grid, kBandBlock, 0, st>>>(B->dev, x, y);
                else
                    k_band_lanes<1, false><<<grid, kBandBlock, 0, st>>>(B->dev, x, y);
                break;
            case 2: k_band_lanes<2, false><<<grid, kBandBlock, 0, st>>>(B->dev, x, y); break;
            case 4: k_band_lanes<4, false><<<grid, kBandBlock, 0, st>>>(B->dev, x, y); break;
            case 8: k_band_lanes<8, false><<<grid, kBandBlock, 0, st>>>(B->dev, x, y); break;
            case 16: k_band_lanes<16, false><<<grid, kBandBlock, 0, st>>>(B->dev, x, y); break;
            case 32: k_band_lanes<32, false><<<grid, kBandBlock, 0, st>>>(B->dev, x, y); break;
            default: set_error("unknown band kernel variant"); return SSG_E_INVALID;
        }
    }
    SSG_CUDA_TRY(cudaGetLastError());
    return SSG_OK;
}

int check_band(const ssg_band *B) {
    if (!B) {
        set_error("null band operator");
        return SSG_E_INVALID;
    }
    return SSG_OK;
}

int check_err_flag(const ssg_band *B) {
    if (*reinterpret_cast<volatile int *>(B->h_err)) {
        set_error("band product: a bounded wait for a staged tile ran out");
        return SSG_E_TIMEOUT;
    }
    return SSG_OK;
}

void free_band(ssg_band *B) {
    if (B->arena) cudaFree(B->arena);
    if (B->h_err) cudaFreeHost(B->h_err);
    B->arena = nullptr;
    B->h_err = nullptr;
}

int upload_band(ssg_band *B) {
    // tiles of whole rows: at most kBandBlock rows and kTileNnz entries, a
    // longer row alone in its tile
    std::vector<int32_t> tile{0};
    int32_t r = 0;
    while (r < B->n) {
        int32_t r1 = r;
        while (r1 < B->n && r1 - r < kBandBlock && B->rowptr[r1 + 1] - B->rowptr[r] <= kTileNnz) ++r1;
        if (r1 == r) r1 = r + 1;
        tile.push_back(r1);
        r = r1;
    }
    const int32_t ntiles = static_cast<int32_t>(tile.size()) - 1;
    // padding: a staged copy may read up to 2 values and 4 column ids past the last entry
    const size_t b_rp = up256(sizeof(int32_t) * (B->n + 1));
    const size_t b_col = up256(sizeof(int32_t) * (B->nnz + 8));
    const size_t b_val = up256(sizeof(double) * (B->nnz + 4));
    const size_t b_tile = up256(sizeof(int32_t) * tile.size());
    char *a = nullptr;
    SSG_CUDA_TRY(cudaMalloc(&a, b_rp + b_col + b_val + b_tile));
    B->arena = a;
    cudaStream_t st = B->ctx->stream;
    int32_t *d_rp = reinterpret_cast<int32_t *>(a);
    int32_t *d_col = reinterpret_cast<int32_t *>(a + b_rp);
    double *d_val = reinterpret_cast<double *>(a + b_rp + b_col);
    int32_t *d_tile = reinterpret_cast<int32_t *>(a + b_rp + b_col + b_val);
    SSG_CUDA_TRY(cudaMemsetAsync(a, 0, b_rp + b_col + b_val + b_tile, st));
    SSG_CUDA_TRY(cudaMemcpyAsync(d_rp, B->rowptr.data(), sizeof(int32_t) * (B->n + 1), cudaMemcpyHostToDevice, st));
    if (B->nnz > 0) {
        SSG_CUDA_TRY(cudaMemcpyAsync(d_col, B->colidx.data(), sizeof(int32_t) * B->nnz, cudaMemcpyHostToDevice, st));
        SSG_CUDA_TRY(cudaMemcpyAsync(d_val, B->val.data(), sizeof(double) * B->nnz, cudaMemcpyHostToDevice, st));
    }
    SSG_CUDA_TRY(cudaMemcpyAsync(d_tile, tile.data(), sizeof(int32_t) * tile.size(), cudaMemcpyHostToDevice, st));
    SSG_CUDA_TRY(cudaHostAlloc(&B->h_err, sizeof(int), cudaHostAllocMapped));
    *B->h_err = 0;
    int *d_err = nullptr;
    SSG_CUDA_TRY(cudaHostGetDevicePointer(&d_err, B->h_err, 0));
    SSG_CUDA_TRY(cudaFuncSetAttribute(k_band_staged<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStagedSmem));
    SSG_CUDA_TRY(cudaFuncSetAttribute(k_band_staged<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStagedSmem));
    B->dev = BandDev{B->n, B->nb, B->n / B->nb, d_rp, d_col, d_val, d_tile, ntiles, d_err};
    SSG_CUDA_TRY(cudaStreamSynchronize(st));
    return SSG_OK;
}

}  // namespace

extern "C" {

int ssg_band_split(ssg_ctx *ctx, int32_t kind, int32_t n, const int32_t *rowptr, const int32_t *colidx,
                   const double *val, int32_t nb, ssg_band **out) {
    if (!out) {
        set_error("ssg_band_split: null output pointer");
        return SSG_E_INVALID;
    }
    *out = nullptr;
    if (!ctx || !rowptr || (kind != SSG_BAND_ROW && kind != SSG_BAND_COL) || n <= 0 || nb <= 0 || nb > n) {
        set_error("ssg_band_split: need a context, kind SSG_BAND_ROW or SSG_BAND_COL, n > 0 and 1 <= nb <= n");
        return SSG_E_INVALID;
    }
    if (rowptr[0] != 0) {
        set_error("ssg_band_split: rowptr[0] must be 0");
        return SSG_E_INVALID;
    }
    for (int32_t i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i]) {
            set_error("ssg_band_split: rowptr decreases at row " + std::to_string(i));
            return SSG_E_INVALID;
        }
    }
    const int64_t nnz = rowptr[n];
    if (nnz > 0 && (!colidx || !val)) {
        set_error("ssg_band_split: null colidx or val");
        return SSG_E_INVALID;
    }
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            if (colidx[k] < 0 || colidx[k] >= n || (k > rowptr[i] && colidx[k] <= colidx[k - 1])) {
                set_error("ssg_band_split: columns of row " + std::to_string(i) +
                          " out of range, unsorted or repeated");
                return SSG_E_INVALID;
            }
        }
    }
    ssg_band *B = new (std::nothrow) ssg_band;
    if (!B) {
        set_error("ssg_band_split: out of host memory");
        return SSG_E_OOM;
    }
    B->ctx = ctx;
    B->kind = kind;
    B->n = n;
    B->nb = nb;
    B->nnz = nnz;
    try {
        B->rowptr.assign(rowptr, rowptr + n + 1);
        B->colidx.assign(colidx, colidx + nnz);
        B->val.assign(val, val + nnz);
    } catch (...) {
        delete B;
        set_error("ssg_band_split: out of host memory");
        return SSG_E_OOM;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) {
        delete B;
        set_error(std::string("cudaSetDevice: ") + cudaGetErrorString(e));
        return SSG_E_CUDA;
    }
    int rc = upload_band(B);
    if (rc != SSG_OK) {
        free_band(B);
        delete B;
        return rc;
    }
    B->rule_variant = rule_for(kind, n, nnz);
    B->variant = B->rule_variant;
    ctx->live_systems++;
    *out = B;
    return SSG_OK;
}

int ssg_band_get(const ssg_band *band, int32_t p, int64_t *sizes, int32_t *rowptr, int32_t *colidx, double *val) {
    int rc = check_band(band);
    if (rc != SSG_OK) return rc;
    if (!sizes || p < 0 || p >= band->nb) {
        set_error("ssg_band_get: null sizes or band index out of range");
        return SSG_E_INVALID;
    }
    const int32_t n = band->n, q = n / band->nb;
    const int32_t displ = p * q;
    const int32_t np = (p == band->nb - 1) ? n - displ : q;
    const int32_t *A_rp = band->rowptr.data();
    const int32_t *A_ci = band->colidx.data();
    const double *A_v = band->val.data();
    sizes[0] = np;
    sizes[1] = displ;
    if (band->kind == SSG_BAND_ROW) {
        const int32_t base = A_rp[displ];
        sizes[2] = A_rp[displ + np] - base;
        if (rowptr)
            for (int32_t i = 0; i <= np; ++i) rowptr[i] = A_rp[displ + i] - base;
        if (colidx && sizes[2] > 0) std::memcpy(colidx, A_ci + base, sizeof(int32_t) * sizes[2]);
        if (val && sizes[2] > 0) std::memcpy(val, A_v + base, sizeof(double) * sizes[2]);
        return SSG_OK;
    }
    int64_t c = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (rowptr) rowptr[i] = static_cast<int32_t>(c);
        // the row's entries in [displ, displ + np) form one run (columns sorted)
        const int32_t *lo = std::lower_bound(A_ci + A_rp[i], A_ci + A_rp[i + 1], displ);
        const int32_t *hi = std::lower_bound(lo, A_ci + A_rp[i + 1], displ + np);
        for (const int32_t *k = lo; k < hi; ++k, ++c) {
            if (colidx) colidx[c] = *k - displ;
            if (val) val[c] = A_v[k - A_ci];
        }
    }
    if (rowptr) rowptr[n] = static_cast<int32_t>(c);
    sizes[2] = c;
    return SSG_OK;
}

int ssg_band_spmv(ssg_band *band, const double *x, double *y) {
    int rc = check_band(band);
    if (rc != SSG_OK) return rc;
    if (!x || !y) {
        set_error("ssg_band_spmv: null vector");
        return SSG_E_INVALID;
    }
    rc = check_err_flag(band);
    if (rc != SSG_OK) return rc;
    return launch_variant(band, band->variant, x, y);
}

int ssg_band_set_variant(ssg_band *band, int32_t variant) {
    int rc = check_band(band);
    if (rc != SSG_OK) return rc;
    if (variant == SSG_BAND_AUTO) {
        band->variant = band->rule_variant;
        return SSG_OK;
    }
    if (!variant_valid(band, variant)) {
        set_error("ssg_band_set_variant: " + std::to_string(variant) + " is not a kernel of this splitting");
        return SSG_E_INVALID;
    }
    band->variant = variant;
    return SSG_OK;
}

int ssg_band_autotune(ssg_band *band, int32_t reps, ssg_band_tune *out) {
    int rc = check_band(band);
    if (rc != SSG_OK) return rc;
    if (reps <= 0 || !out) {
        set_error("ssg_band_autotune: reps must be positive and out not null");
        return SSG_E_INVALID;
    }
    const int32_t codes[7] = {SSG_BAND_STAGED, 1, 2, 4, 8, 16, 32};
    cudaStream_t st = band->ctx->stream;
    double *xy = nullptr;
    SSG_CUDA_TRY(cudaMalloc(&xy, sizeof(double) * 2 * static_cast<size_t>(band->n)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaMemsetAsync(xy, 0, sizeof(double) * 2 * static_cast<size_t>(band->n), st);
    std::memset(out, 0, sizeof(*out));
    float best = 0.0f;
    int32_t best_v = band->rule_variant;
    rc = SSG_OK;
    for (int i = 0; i < 7 && rc == SSG_OK; ++i) {
        out->code[i] = codes[i];
        if (!variant_valid(band, codes[i])) continue;
        rc = launch_variant(band, codes[i], xy, xy + band->n);  // warm-up
        if (rc != SSG_OK) break;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && rc == SSG_OK; ++r) rc = launch_variant(band, codes[i], xy, xy + band->n);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            set_error("ssg_band_autotune: timing failed");
            rc = SSG_E_CUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        out->us[i] = 1000.0f * ms / reps;
        if (best == 0.0f || out->us[i] < best) {
            best = out->us[i];
            best_v = codes[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(xy);
    if (rc == SSG_OK) rc = check_err_flag(band);
    if (rc != SSG_OK) return rc;
    band->variant = best_v;
    out->variant = best_v;
    out->rule_variant = band->rule_variant;
    return SSG_OK;
}

int ssg_band_check_timeout(ssg_band *band) {
    int rc = check_band(band);
    if (rc != SSG_OK) return rc;
    SSG_CUDA_TRY(cudaStreamSynchronize(band->ctx->stream));
    rc = check_err_flag(band);
    if (rc != SSG_OK) return rc;
    k_band_wait_probe<<<1, 32, 0, band->ctx->stream>>>(band->dev.err);
    SSG_CUDA_TRY(cudaGetLastError());
    SSG_CUDA_TRY(cudaStreamSynchronize(band->ctx->stream));
    rc = check_err_flag(band);
    *band->h_err = 0;  // the probe's flag is its result, not a fault of the operator
    return rc;
}

int ssg_band_destroy(ssg_band *band) {
    if (!band) return SSG_OK;
    cudaStreamSynchronize(band->ctx->stream);
    free_band(band);
    band->ctx->live_systems--;
    delete band;
    return SSG_OK;
}

}  // extern "C"
