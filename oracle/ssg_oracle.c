/*
 * Plain FP64 CPU oracle for the sub-structured Conjugate Gradient.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the CUDA path is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may build or call it.
 * It shares no code, header or table with the CUDA library, and it must be
 * compiled with -ffp-contract=off so that every a*b+c rounds twice, the same
 * way on x86-64 and aarch64.
 *
 * What it computes, by paper section:
 *   or_spmv          global CSR product y = A x, rows in order, each row summed
 *                    left to right (CSR storage, Section 1.2).
 *   or_cg            Algorithm 3 (Conjugate Gradient) with M = I on the global
 *                    CSR, x1 = x0, stopping on the recursive residual.
 *   or_partition     the sub-structure data of Section 2.4: local matrices S_i
 *                    (Eq. mat_subdomains) whose interface blocks sum to S_33
 *                    (Eq. interface_summation), local-to-global maps and the
 *                    per-node interface lists (Section 3.4.2), with the
 *                    entry-ownership reading for assembled matrices.
 *   or_sub_spmv      the two-step sub-structured SpMV of Section 3.4.1: local
 *                    products, then assembly of interface contributions
 *                    (Algorithms 4 and 5, every copy receives the same sum).
 *   or_wdot          the interface-weighted dot of Section 3.4.2, w = 1/m
 *                    (or the owner mask, or_set_weights).
 *   or_sub_cg        Algorithm 3 with the sub-structured SpMV and weighted dots.
 *   or_cholesky_solve  textbook dense Cholesky (second opinion on tiny systems).
 *   or_band_row, or_band_col  the band-row and band-column splittings of
 *                    Sections 2.1 and 2.2 (Algorithms 1 and 2), one band at a time.
 *   or_band_row_spmv, or_band_col_spmv  y = A x through either splitting: each
 *                    band's block of y, or the sum of the bands' partial products.
 *   or_sub_cg_omp    or_sub_cg with the subdomains shared among OpenMP threads
 *                    (the CPU baseline on all host cores).
 *
 * Readings where the paper is silent (no tolerance, no initial guess, no
 * weights, no rule for splitting an assembled S_33) are stated at each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_INVALID 1
#define OR_OOM 2
#define OR_BREAKDOWN 4
#define OR_NOT_CONVERGED 5

/* ------------------------------------------------------------------ */
/* Global CSR product (Section 1.2).                                   */
/* ------------------------------------------------------------------ */
void or_spmv(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val, const double *x,
             double *y) {
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += val[k] * x[colidx[k]];
        y[i] = s;
    }
}

static double dot_plain(int64_t n, const double *u, const double *v) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += u[i] * v[i];
    return s;
}

/*
 * Algorithm 3 with M = I (z_k = r_k), on the assembled matrix.
 * Reading: x1 = x (input, the initial guess); the loop stops after the first
 * iteration k whose recursive residual satisfies sqrt(rho_k) <= rtol*||b||, or
 * when max_iter iterations are done.  A zero right-hand side with x = 0 is
 * converged at iteration 0.  (S p_k, p_k) <= 0 or non-finite is a breakdown.
 * hist_alpha/hist_beta (may be NULL) receive alpha_k and beta_k per iteration
 * (length >= max_iter); hist_res (may be NULL) receives sqrt(rho)/||b|| after
 * each iteration.
 */
int or_cg(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val, const double *b, double *x,
          double rtol, int32_t max_iter, int32_t *iters_out, double *relres_out, double *hist_alpha,
          double *hist_beta, double *hist_res) {
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *p = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *q = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!r || !p || !q) {
        free(r); free(p); free(q);
        return OR_OOM;
    }
    int status = OR_NOT_CONVERGED;
    or_spmv(n, rowptr, colidx, val, x, q);
    for (int32_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    for (int32_t i = 0; i < n; ++i) p[i] = r[i];
    double rho = dot_plain(n, r, r);
    double bnorm = sqrt(dot_plain(n, b, b));
    int32_t k = 0;
    double relres = bnorm > 0.0 ? sqrt(rho) / bnorm : 0.0;
    if (sqrt(rho) <= rtol * bnorm) status = OR_OK;
    while (status == OR_NOT_CONVERGED && k < max_iter) {
        or_spmv(n, rowptr, colidx, val, p, q);
        double pq = dot_plain(n, q, p);
        if (!(pq > 0.0) || !isfinite(pq)) {
            status = OR_BREAKDOWN;
            break;
        }
        double alpha = rho / pq;
        for (int32_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
        for (int32_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
        double rho_new = dot_plain(n, r, r);
        double beta = rho_new / rho;
        for (int32_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        if (hist_alpha) hist_alpha[k] = alpha;
        if (hist_beta) hist_beta[k] = beta;
        rho = rho_new;
        ++k;
        relres = bnorm > 0.0 ? sqrt(rho) / bnorm : 0.0;
        if (hist_res) hist_res[k - 1] = relres;
        if (sqrt(rho) <= rtol * bnorm) status = OR_OK;
    }
    *iters_out = k;
    *relres_out = relres;
    free(r); free(p); free(q);
    return status;
}

/* ------------------------------------------------------------------ */
/* Sub-structure data (Section 2.4, Section 3.4).                      */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t n, P;
    int64_t nnz;
    int64_t nloc;    /* sum over s of |V_s| */
    int32_t ngamma;  /* number of interface nodes */
    int64_t ncopies; /* sum of multiplicities over interface nodes */
    int32_t *off;    /* [P+1] first concatenated local index of each subdomain */
    int32_t *nint;   /* [P] number of interior (m = 1) nodes of each subdomain */
    int32_t *l2g;    /* [nloc] global node of each concatenated local index */
    int32_t *mult;   /* [n] multiplicity m_i */
    int32_t *lrowptr;/* [nloc+1] concatenated local CSR row pointers */
    int32_t *lcol;   /* [nnz] local column index inside its subdomain */
    double *lval;    /* [nnz] values, copied unchanged from A */
    int32_t *gamma;  /* [ngamma] interface nodes, ascending global id */
    int32_t *iptr;   /* [ngamma+1] */
    int32_t *icopy;  /* [ncopies] concatenated local index of each copy, ascending s */
    int32_t *own;    /* [n] concatenated local index of the copy in subdomain part(i) */
    double *w;       /* [nloc] weight 1/m of each local entry */
} or_part;

static int find_col(const int32_t *colidx, int32_t lo, int32_t hi, int32_t c) {
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (colidx[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

void or_part_free(or_part *h) {
    if (!h) return;
    free(h->off); free(h->nint); free(h->l2g); free(h->mult); free(h->lrowptr); free(h->lcol);
    free(h->lval); free(h->gamma); free(h->iptr); free(h->icopy); free(h->own); free(h->w);
    free(h);
}

/* owner subdomain of stored entry (i, j): the diagonal goes to part(i), an
 * off-diagonal entry to min(part(i), part(j)) (reading for an assembled S). */
static int32_t owner_of(const int32_t *part, int32_t i, int32_t j) {
    if (i == j) return part[i];
    return part[i] < part[j] ? part[i] : part[j];
}

typedef struct { int32_t key; int32_t a; double v; } triple;
static int cmp_triple(const void *x, const void *y) {
    const triple *p = (const triple *)x, *q = (const triple *)y;
    return (p->key > q->key) - (p->key < q->key);
}
static int cmp_int(const void *x, const void *y) {
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/*
 * Build the sub-structures from a global CSR matrix and a node partition.
 * Returns NULL with *status set on invalid input.  Checks: shapes, sorted and
 * unique columns, part ids in [0, P), structural and value symmetry.
 *
 * V_s     = {i : part(i) = s}  U  {j : some i with part(i) = s < part(j) has A_ij stored}
 * m_j     = number of subdomains whose V_s holds j; interface = {j : m_j >= 2}
 * order   = in each V_s, nodes with m = 1 first, then interface nodes, each ascending by global id
 *           ("interior then interface" numbering of Eq. 2.4:eqn0)
 * A^(s)   = the stored entries owned by s, rows in local order, columns sorted by local id
 * copies  = for each interface node (ascending id), its local copies in ascending s
 */
or_part *or_partition(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                      const int32_t *part, int32_t P, int *status) {
    *status = OR_INVALID;
    if (n <= 0 || P <= 0 || rowptr[0] != 0) return NULL;
    for (int32_t i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i]) return NULL;
        if (part[i] < 0 || part[i] >= P) return NULL;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            if (colidx[k] < 0 || colidx[k] >= n) return NULL;
            if (k > rowptr[i] && colidx[k] <= colidx[k - 1]) return NULL;
        }
    }
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            int32_t j = colidx[k];
            int32_t t = find_col(colidx, rowptr[j], rowptr[j + 1], i);
            if (t >= rowptr[j + 1] || colidx[t] != i) return NULL;
            if (val[t] != val[k]) return NULL;
        }
    }
    *status = OR_OOM;
    or_part *h = (or_part *)calloc(1, sizeof(or_part));
    if (!h) return NULL;
    h->n = n;
    h->P = P;
    h->nnz = rowptr[n];

    /* membership: subdomain list of every node (sorted, unique) */
    int32_t *mem_ptr = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)(h->nnz + n));
    int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * (size_t)(h->nnz + n));
    if (!mem_ptr || !cand || !mem) goto oom;
    {
        int64_t w = 0;
        for (int32_t j = 0; j < n; ++j) {
            int64_t c0 = 0;
            cand[c0++] = part[j];
            for (int32_t k = rowptr[j]; k < rowptr[j + 1]; ++k) {
                int32_t i = colidx[k];
                if (part[i] < part[j]) cand[c0++] = part[i];
            }
            qsort(cand, (size_t)c0, sizeof(int32_t), cmp_int);
            for (int64_t t = 0; t < c0; ++t)
                if (t == 0 || cand[t] != cand[t - 1]) mem[w++] = cand[t];
            mem_ptr[j + 1] = (int32_t)w;
        }
    }
    h->mult = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!h->mult) goto oom;
    for (int32_t j = 0; j < n; ++j) h->mult[j] = mem_ptr[j + 1] - mem_ptr[j];

    /* sizes and local numbering */
    h->off = (int32_t *)calloc((size_t)P + 1, sizeof(int32_t));
    h->nint = (int32_t *)calloc((size_t)P, sizeof(int32_t));
    int32_t *cnt = (int32_t *)calloc((size_t)P, sizeof(int32_t));
    if (!h->off || !h->nint || !cnt) { free(cnt); goto oom; }
    for (int32_t j = 0; j < n; ++j)
        for (int32_t t = mem_ptr[j]; t < mem_ptr[j + 1]; ++t) {
            cnt[mem[t]]++;
            if (h->mult[j] == 1) h->nint[mem[t]]++;
        }
    for (int32_t s = 0; s < P; ++s) h->off[s + 1] = h->off[s] + cnt[s];
    h->nloc = h->off[P];
    /* local index of node j inside each subdomain of its membership list */
    int32_t *memloc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(mem_ptr[n] > 0 ? mem_ptr[n] : 1));
    h->l2g = (int32_t *)malloc(sizeof(int32_t) * (size_t)(h->nloc > 0 ? h->nloc : 1));
    if (!memloc || !h->l2g) { free(cnt); free(memloc); goto oom; }
    for (int32_t s = 0; s < P; ++s) cnt[s] = 0;
    for (int pass = 0; pass < 2; ++pass) {
        /* pass 0: interior nodes (m = 1), pass 1: interface nodes, each ascending by id */
        for (int32_t j = 0; j < n; ++j) {
            int is_iface = h->mult[j] >= 2;
            if (is_iface != pass) continue;
            for (int32_t t = mem_ptr[j]; t < mem_ptr[j + 1]; ++t) {
                int32_t s = mem[t];
                memloc[t] = cnt[s]++;
                h->l2g[h->off[s] + memloc[t]] = j;
            }
        }
    }
    free(cnt);

    /* owner copy */
    h->own = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!h->own) { free(memloc); goto oom; }
    for (int32_t j = 0; j < n; ++j)
        for (int32_t t = mem_ptr[j]; t < mem_ptr[j + 1]; ++t)
            if (mem[t] == part[j]) h->own[j] = h->off[part[j]] + memloc[t];

    /* local CSR */
    h->lrowptr = (int32_t *)calloc((size_t)h->nloc + 1, sizeof(int32_t));
    h->lcol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(h->nnz > 0 ? h->nnz : 1));
    h->lval = (double *)malloc(sizeof(double) * (size_t)(h->nnz > 0 ? h->nnz : 1));
    if (!h->lrowptr || !h->lcol || !h->lval) { free(memloc); goto oom; }
    {
        triple *row = (triple *)malloc(sizeof(triple) * (size_t)(n > 0 ? n : 1));
        if (!row) { free(memloc); goto oom; }
        int64_t wpos = 0;
        for (int32_t s = 0; s < P; ++s) {
            for (int32_t li = 0; li < h->off[s + 1] - h->off[s]; ++li) {
                int32_t i = h->l2g[h->off[s] + li];
                int32_t c = 0;
                for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
                    int32_t j = colidx[k];
                    if (owner_of(part, i, j) != s) continue;
                    /* local id of j in s */
                    int32_t lj = -1;
                    for (int32_t t = mem_ptr[j]; t < mem_ptr[j + 1]; ++t)
                        if (mem[t] == s) lj = memloc[t];
                    if (lj < 0) { free(row); free(memloc); *status = OR_INVALID; goto fail; }
                    row[c].key = lj;
                    row[c].v = val[k];
                    row[c].a = 0;
                    ++c;
                }
                qsort(row, (size_t)c, sizeof(triple), cmp_triple);
                for (int32_t t = 0; t < c; ++t) {
                    h->lcol[wpos] = row[t].key;
                    h->lval[wpos] = row[t].v;
                    ++wpos;
                }
                h->lrowptr[h->off[s] + li + 1] = (int32_t)wpos;
            }
        }
        free(row);
        if (wpos != h->nnz) { free(memloc); *status = OR_INVALID; goto fail; }
    }

    /* interface lists */
    h->ngamma = 0;
    h->ncopies = 0;
    for (int32_t j = 0; j < n; ++j)
        if (h->mult[j] >= 2) { h->ngamma++; h->ncopies += h->mult[j]; }
    h->gamma = (int32_t *)malloc(sizeof(int32_t) * (size_t)(h->ngamma > 0 ? h->ngamma : 1));
    h->iptr = (int32_t *)calloc((size_t)h->ngamma + 1, sizeof(int32_t));
    h->icopy = (int32_t *)malloc(sizeof(int32_t) * (size_t)(h->ncopies > 0 ? h->ncopies : 1));
    if (!h->gamma || !h->iptr || !h->icopy) { free(memloc); goto oom; }
    {
        int32_t g = 0;
        int64_t c = 0;
        for (int32_t j = 0; j < n; ++j) {
            if (h->mult[j] < 2) continue;
            h->gamma[g] = j;
            for (int32_t t = mem_ptr[j]; t < mem_ptr[j + 1]; ++t) h->icopy[c++] = h->off[mem[t]] + memloc[t];
            h->iptr[++g] = (int32_t)c;
        }
    }
    /* weights w = 1/m per local entry */
    h->w = (double *)malloc(sizeof(double) * (size_t)(h->nloc > 0 ? h->nloc : 1));
    if (!h->w) { free(memloc); goto oom; }
    for (int64_t k = 0; k < h->nloc; ++k) h->w[k] = 1.0 / (double)h->mult[h->l2g[k]];
    free(memloc);
    free(mem_ptr); free(cand); free(mem);
    *status = OR_OK;
    return h;
oom:
    *status = OR_OOM;
fail:
    free(mem_ptr); free(cand); free(mem);
    or_part_free(h);
    return NULL;
}

void or_part_sizes(const or_part *h, int64_t *out) {
    out[0] = h->n;
    out[1] = h->P;
    out[2] = h->nnz;
    out[3] = h->nloc;
    out[4] = h->ngamma;
    out[5] = h->ncopies;
}

void or_part_copy(const or_part *h, int32_t *off, int32_t *nint, int32_t *l2g, int32_t *mult, int32_t *lrowptr,
                  int32_t *lcol, double *lval, int32_t *gamma, int32_t *iptr, int32_t *icopy, int32_t *own,
                  double *w) {
    memcpy(off, h->off, sizeof(int32_t) * (size_t)(h->P + 1));
    memcpy(nint, h->nint, sizeof(int32_t) * (size_t)h->P);
    memcpy(l2g, h->l2g, sizeof(int32_t) * (size_t)h->nloc);
    memcpy(mult, h->mult, sizeof(int32_t) * (size_t)h->n);
    memcpy(lrowptr, h->lrowptr, sizeof(int32_t) * (size_t)(h->nloc + 1));
    memcpy(lcol, h->lcol, sizeof(int32_t) * (size_t)h->nnz);
    memcpy(lval, h->lval, sizeof(double) * (size_t)h->nnz);
    memcpy(gamma, h->gamma, sizeof(int32_t) * (size_t)h->ngamma);
    memcpy(iptr, h->iptr, sizeof(int32_t) * (size_t)(h->ngamma + 1));
    memcpy(icopy, h->icopy, sizeof(int32_t) * (size_t)h->ncopies);
    memcpy(own, h->own, sizeof(int32_t) * (size_t)h->n);
    memcpy(w, h->w, sizeof(double) * (size_t)h->nloc);
}

/* global -> local: every copy of node i receives x_glob[i] */
void or_scatter(const or_part *h, const double *xg, double *xl) {
    for (int64_t k = 0; k < h->nloc; ++k) xl[k] = xg[h->l2g[k]];
}

/* local -> global: node i takes the value of its copy in subdomain part(i) */
void or_gather(const or_part *h, const double *xl, double *xg) {
    for (int32_t i = 0; i < h->n; ++i) xg[i] = xl[h->own[i]];
}

/*
 * Section 3.4.1: y_s = A^(s) x_s for every subdomain (rows in local order,
 * each row summed left to right), then, for every interface node in ascending
 * global id, the sum of its copies' values taken in ascending s is written back
 * to every copy (the collect/send and receive/update of Algorithms 4 and 5 with
 * one fixed summation order).
 */
void or_sub_spmv(const or_part *h, const double *xl, double *yl) {
    for (int32_t s = 0; s < h->P; ++s) {
        const int32_t o = h->off[s];
        for (int32_t li = 0; li < h->off[s + 1] - o; ++li) {
            double acc = 0.0;
            for (int32_t k = h->lrowptr[o + li]; k < h->lrowptr[o + li + 1]; ++k)
                acc += h->lval[k] * xl[o + h->lcol[k]];
            yl[o + li] = acc;
        }
    }
    for (int32_t g = 0; g < h->ngamma; ++g) {
        double S = 0.0;
        for (int32_t c = h->iptr[g]; c < h->iptr[g + 1]; ++c) S += yl[h->icopy[c]];
        for (int32_t c = h->iptr[g]; c < h->iptr[g + 1]; ++c) yl[h->icopy[c]] = S;
    }
}

/* Section 3.4.2 weighted dot: sum over concatenated local entries of w*u*v,
 * w = 1/m (reading: the paper does not give the weights). */
double or_wdot(const or_part *h, const double *u, const double *v) {
    double s = 0.0;
    for (int64_t k = 0; k < h->nloc; ++k) s += h->w[k] * u[k] * v[k];
    return s;
}

/*
 * The weights of every weighted dot (Section 3.4.2 asks for a weighted
 * combination of the subdomains' sums without giving the weights).  mode 0:
 * w = 1/m on every copy of a node (the default set by or_partition); mode 1,
 * the owner mask: w = 1 on the node's owner copy own[i] (its copy in
 * subdomain part(i); for element sub-structures, in the lowest subdomain) and
 * w = 0 on its other copies.  Either set sums to 1 over the copies of each
 * node, so for a consistent vector both dots are the global dot in exact
 * arithmetic.  Returns OR_OK, or OR_INVALID for another mode.
 */
int or_set_weights(or_part *h, int mode) {
    if (mode == 0) {
        for (int64_t k = 0; k < h->nloc; ++k) h->w[k] = 1.0 / (double)h->mult[h->l2g[k]];
        return OR_OK;
    }
    if (mode == 1) {
        for (int64_t k = 0; k < h->nloc; ++k) h->w[k] = 0.0;
        for (int32_t i = 0; i < h->n; ++i) h->w[h->own[i]] = 1.0;
        return OR_OK;
    }
    return OR_INVALID;
}

/*
 * Algorithm 3 (M = I) with the sub-structured SpMV and weighted dots, on the
 * concatenated local vectors; b and x are global (length n).  x is the
 * initial guess on input.  Same stopping rule and outputs as or_cg.
 */
int or_sub_cg(const or_part *h, const double *b, double *x, double rtol, int32_t max_iter, int32_t *iters_out,
              double *relres_out, double *hist_alpha, double *hist_beta, double *hist_res) {
    size_t N = (size_t)(h->nloc > 0 ? h->nloc : 1);
    double *bl = (double *)malloc(sizeof(double) * N);
    double *xl = (double *)malloc(sizeof(double) * N);
    double *r = (double *)malloc(sizeof(double) * N);
    double *p = (double *)malloc(sizeof(double) * N);
    double *q = (double *)malloc(sizeof(double) * N);
    if (!bl || !xl || !r || !p || !q) {
        free(bl); free(xl); free(r); free(p); free(q);
        return OR_OOM;
    }
    const int64_t L = h->nloc;
    or_scatter(h, b, bl);
    or_scatter(h, x, xl);
    or_sub_spmv(h, xl, q);
    for (int64_t k = 0; k < L; ++k) r[k] = bl[k] - q[k];
    for (int64_t k = 0; k < L; ++k) p[k] = r[k];
    double rho = or_wdot(h, r, r);
    double bnorm = sqrt(or_wdot(h, bl, bl));
    int status = OR_NOT_CONVERGED;
    int32_t it = 0;
    double relres = bnorm > 0.0 ? sqrt(rho) / bnorm : 0.0;
    if (sqrt(rho) <= rtol * bnorm) status = OR_OK;
    while (status == OR_NOT_CONVERGED && it < max_iter) {
        or_sub_spmv(h, p, q);
        double pq = or_wdot(h, q, p);
        if (!(pq > 0.0) || !isfinite(pq)) {
            status = OR_BREAKDOWN;
            break;
        }
        double alpha = rho / pq;
        for (int64_t k = 0; k < L; ++k) xl[k] = xl[k] + alpha * p[k];
        for (int64_t k = 0; k < L; ++k) r[k] = r[k] - alpha * q[k];
        double rho_new = or_wdot(h, r, r);
        double beta = rho_new / rho;
        for (int64_t k = 0; k < L; ++k) p[k] = r[k] + beta * p[k];
        if (hist_alpha) hist_alpha[it] = alpha;
        if (hist_beta) hist_beta[it] = beta;
        rho = rho_new;
        ++it;
        relres = bnorm > 0.0 ? sqrt(rho) / bnorm : 0.0;
        if (hist_res) hist_res[it - 1] = relres;
        if (sqrt(rho) <= rtol * bnorm) status = OR_OK;
    }
    or_gather(h, xl, x);
    *iters_out = it;
    *relres_out = relres;
    free(bl); free(xl); free(r); free(p); free(q);
    return status;
}

/* Textbook dense Cholesky A = L L^T (row-major n x n), then two triangular
 * solves.  Returns OR_BREAKDOWN if a pivot is not positive. */
int or_cholesky_solve(int32_t n, const double *A, const double *b, double *x) {
    double *L = (double *)calloc((size_t)n * (size_t)n, sizeof(double));
    double *y = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!L || !y) { free(L); free(y); return OR_OOM; }
    for (int32_t j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int32_t k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(d > 0.0)) { free(L); free(y); return OR_BREAKDOWN; }
        double ljj = sqrt(d);
        L[(size_t)j * n + j] = ljj;
        for (int32_t i = j + 1; i < n; ++i) {
            double s = A[(size_t)i * n + j];
            for (int32_t k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = s / ljj;
        }
    }
    for (int32_t i = 0; i < n; ++i) {
        double s = b[i];
        for (int32_t k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * y[k];
        y[i] = s / L[(size_t)i * n + i];
    }
    for (int32_t i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int32_t k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * x[k];
        x[i] = s / L[(size_t)i * n + i];
    }
    free(L); free(y);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Mixed precision: FP32 inner CG inside FP64 iterative refinement.    */
/* ------------------------------------------------------------------ */
/*
 * Not a method of the paper (its experiments are FP64 only); the reading
 * this oracle fixes for the library's SSG_MIXED mode:
 *   outer (FP64): r = b - S x with the sub-structured SpMV of Section 3.4.1,
 *     stop when sqrt((r,r)_w) <= rtol * sqrt((b,b)_w), after max_outer
 *     refinements, or when the inner iterations reach max_iter;
 *   inner (FP32): Algorithm 3 (M = I) on S32 d = r32 with S32 = (float)S,
 *     r32 = (float)r, d = 0, every product, sum and update in float (the
 *     local row products and the interface sums included); the dot
 *     products multiply in float and accumulate in double; alpha and beta
 *     are the double ratios rounded to float; stop when
 *     sqrt(rho_k) <= tau * sqrt(rho_0), tau = max(inner_rtol,
 *     rtol * ||b|| / ||r||) (the last refinement is not over-solved);
 *   update: x += (double) d.
 */
static void sub_spmv32(const or_part *h, const float *val32, const float *xl, float *yl) {
    for (int32_t s = 0; s < h->P; ++s) {
        const int32_t o = h->off[s];
        for (int32_t li = 0; li < h->off[s + 1] - o; ++li) {
            float acc = 0.0f;
            for (int32_t k = h->lrowptr[o + li]; k < h->lrowptr[o + li + 1]; ++k) acc += val32[k] * xl[o + h->lcol[k]];
            yl[o + li] = acc;
        }
    }
    for (int32_t g = 0; g < h->ngamma; ++g) {
        float S = 0.0f;
        for (int32_t c = h->iptr[g]; c < h->iptr[g + 1]; ++c) S += yl[h->icopy[c]];
        for (int32_t c = h->iptr[g]; c < h->iptr[g + 1]; ++c) yl[h->icopy[c]] = S;
    }
}

/* sub_spmv32 with the FP32 value copy made here (for tests) */
void or_sub_spmv32(const or_part *h, const float *xl, float *yl) {
    float *val32 = (float *)malloc(sizeof(float) * (size_t)(h->nnz > 0 ? h->nnz : 1));
    if (!val32) return;
    for (int64_t k = 0; k < h->nnz; ++k) val32[k] = (float)h->lval[k];
    sub_spmv32(h, val32, xl, yl);
    free(val32);
}

static double wdot32(const or_part *h, const float *u, const float *v) {
    double s = 0.0;
    for (int64_t k = 0; k < h->nloc; ++k) s += (double)((float)h->w[k] * u[k] * v[k]);
    return s;
}

int or_sub_cg_mixed(const or_part *h, const double *b, double *x, double rtol, int32_t max_iter, double inner_rtol,
                    int32_t max_outer, int32_t *iters_out, int32_t *outer_out, double *relres_out) {
    size_t N = (size_t)(h->nloc > 0 ? h->nloc : 1);
    const int64_t L = h->nloc;
    double *bl = (double *)malloc(sizeof(double) * N);
    double *xl = (double *)malloc(sizeof(double) * N);
    double *r = (double *)malloc(sizeof(double) * N);
    double *q = (double *)malloc(sizeof(double) * N);
    float *val32 = (float *)malloc(sizeof(float) * (size_t)(h->nnz > 0 ? h->nnz : 1));
    float *r32 = (float *)malloc(sizeof(float) * N);
    float *p32 = (float *)malloc(sizeof(float) * N);
    float *q32 = (float *)malloc(sizeof(float) * N);
    float *d32 = (float *)malloc(sizeof(float) * N);
    if (!bl || !xl || !r || !q || !val32 || !r32 || !p32 || !q32 || !d32) {
        free(bl); free(xl); free(r); free(q); free(val32); free(r32); free(p32); free(q32); free(d32);
        return OR_OOM;
    }
    for (int64_t k = 0; k < h->nnz; ++k) val32[k] = (float)h->lval[k];
    or_scatter(h, b, bl);
    or_scatter(h, x, xl);
    or_sub_spmv(h, xl, q);
    for (int64_t k = 0; k < L; ++k) r[k] = bl[k] - q[k];
    double rho = or_wdot(h, r, r);
    const double bnorm = sqrt(or_wdot(h, bl, bl));
    int32_t outer = 0, total = 0;
    int status = OR_NOT_CONVERGED;
    if (sqrt(rho) <= rtol * bnorm) status = OR_OK;
    while (status == OR_NOT_CONVERGED && outer < max_outer && total < max_iter) {
        double tau = rtol * bnorm / sqrt(rho);
        if (tau < inner_rtol) tau = inner_rtol;
        for (int64_t k = 0; k < L; ++k) {
            r32[k] = (float)r[k];
            p32[k] = r32[k];
            d32[k] = 0.0f;
        }
        double rho32 = wdot32(h, r32, r32);
        const double rho0 = rho32;
        int broke = 0;
        while (sqrt(rho32) > tau * sqrt(rho0) && total < max_iter) {
            sub_spmv32(h, val32, p32, q32);
            const double pq = wdot32(h, p32, q32);
            if (!(pq > 0.0) || !isfinite(pq)) {
                broke = 1;
                break;
            }
            const float alpha = (float)(rho32 / pq);
            for (int64_t k = 0; k < L; ++k) d32[k] = d32[k] + alpha * p32[k];
            for (int64_t k = 0; k < L; ++k) r32[k] = r32[k] - alpha * q32[k];
            const double rho_new = wdot32(h, r32, r32);
            const float beta = (float)(rho_new / rho32);
            for (int64_t k = 0; k < L; ++k) p32[k] = r32[k] + beta * p32[k];
            rho32 = rho_new;
            ++total;
        }
        for (int64_t k = 0; k < L; ++k) xl[k] = xl[k] + (double)d32[k];
        or_sub_spmv(h, xl, q);
        for (int64_t k = 0; k < L; ++k) r[k] = bl[k] - q[k];
        rho = or_wdot(h, r, r);
        ++outer;
        if (sqrt(rho) <= rtol * bnorm) status = OR_OK;
        else if (broke) status = OR_BREAKDOWN;
    }
    or_gather(h, xl, x);
    *iters_out = total;
    *outer_out = outer;
    *relres_out = bnorm > 0.0 ? sqrt(rho) / bnorm : 0.0;
    free(bl); free(xl); free(r); free(q); free(val32); free(r32); free(p32); free(q32); free(d32);
    return status;
}

/* ------------------------------------------------------------------ */
/* Algorithm 3 with the diagonal preconditioner M = diag(S).           */
/* ------------------------------------------------------------------ */
/*
 * Algorithm 3 with the preconditioner the paper's experiments use, the
 * diagonal of the matrix (Section 3.1): z = M^{-1} r = r / diag(S),
 * alpha = (z, r) / (S p, p), beta = (r_{k+1}, z_{k+1}) / (r_k, z_k),
 * p = z + beta p.  Reading: the stopping test stays on the recursive residual
 * sqrt((r, r)) <= rtol ||b|| (the paper gives none), so both (r, z) and
 * (r, r) are formed each iteration.  A missing or non-positive diagonal
 * entry is invalid input.
 */
int or_pcg(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val, const double *b, double *x,
           double rtol, int32_t max_iter, int32_t *iters_out, double *relres_out) {
    size_t N = (size_t)(n > 0 ? n : 1);
    double *d = (double *)malloc(sizeof(double) * N), *r = (double *)malloc(sizeof(double) * N);
    double *z = (double *)malloc(sizeof(double) * N), *p = (double *)malloc(sizeof(double) * N);
    double *q = (double *)malloc(sizeof(double) * N);
    if (!d || !r || !z || !p || !q) {
        free(d); free(r); free(z); free(p); free(q);
        return OR_OOM;
    }
    int status = OR_NOT_CONVERGED;
    for (int32_t i = 0; i < n; ++i) {
        d[i] = 0.0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            if (colidx[k] == i) d[i] = val[k];
        if (!(d[i] > 0.0)) status = OR_INVALID;
    }
    if (status == OR_INVALID) {
        free(d); free(r); free(z); free(p); free(q);
        return OR_INVALID;
    }
    or_spmv(n, rowptr, colidx, val, x, q);
    for (int32_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    for (int32_t i = 0; i < n; ++i) z[i] = r[i] / d[i];
    for (int32_t i = 0; i < n; ++i) p[i] = z[i];
    double rz = dot_plain(n, r, z), rr = dot_plain(n, r, r);
    const double bnorm = sqrt(dot_plain(n, b, b));
    int32_t k = 0;
    if (sqrt(rr) <= rtol * bnorm) status = OR_OK;
    while (status == OR_NOT_CONVERGED && k < max_iter) {
        or_spmv(n, rowptr, colidx, val, p, q);
        const double pq = dot_plain(n, q, p);
        if (!(pq > 0.0) || !isfinite(pq)) {
            status = OR_BREAKDOWN;
            break;
        }
        const double alpha = rz / pq;
        for (int32_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
        for (int32_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
        for (int32_t i = 0; i < n; ++i) z[i] = r[i] / d[i];
        const double rz_new = dot_plain(n, r, z);
        rr = dot_plain(n, r, r);
        const double beta = rz_new / rz;
        for (int32_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        rz = rz_new;
        ++k;
        if (sqrt(rr) <= rtol * bnorm) status = OR_OK;
    }
    *iters_out = k;
    *relres_out = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
    free(d); free(r); free(z); free(p); free(q);
    return status;
}

/* The assembled diagonal of S at every local entry: d_i = sum over the copies
 * of node i (ascending s) of the diagonal entry of its local row, where one is
 * stored.  With entry ownership only the copy in part(i) stores one, so d_i
 * is the global S_ii; with element sub-structures every copy holds a partial
 * sum (Eq. interface_summation). */
static int local_diagonal(const or_part *h, double *dl) {
    double *dg = (double *)calloc((size_t)(h->n > 0 ? h->n : 1), sizeof(double));
    if (!dg) return OR_OOM;
    for (int32_t s = 0; s < h->P; ++s)
        for (int32_t k = h->off[s]; k < h->off[s + 1]; ++k)
            for (int32_t e = h->lrowptr[k]; e < h->lrowptr[k + 1]; ++e)
                if (h->lcol[e] == k - h->off[s]) dg[h->l2g[k]] = dg[h->l2g[k]] + h->lval[e];
    for (int32_t i = 0; i < h->n; ++i)
        if (!(dg[i] > 0.0)) {
            free(dg);
            return OR_INVALID;
        }
    for (int64_t k = 0; k < h->nloc; ++k) dl[k] = dg[h->l2g[k]];
    free(dg);
    return OR_OK;
}

/* or_pcg on the sub-structured operator with weighted dots (Section 3.4). */
int or_sub_pcg(const or_part *h, const double *b, double *x, double rtol, int32_t max_iter, int32_t *iters_out,
               double *relres_out) {
    size_t N = (size_t)(h->nloc > 0 ? h->nloc : 1);
    const int64_t L = h->nloc;
    double *dl = (double *)malloc(sizeof(double) * N), *bl = (double *)malloc(sizeof(double) * N);
    double *xl = (double *)malloc(sizeof(double) * N), *r = (double *)malloc(sizeof(double) * N);
    double *z = (double *)malloc(sizeof(double) * N), *p = (double *)malloc(sizeof(double) * N);
    double *q = (double *)malloc(sizeof(double) * N);
    if (!dl || !bl || !xl || !r || !z || !p || !q) {
        free(dl); free(bl); free(xl); free(r); free(z); free(p); free(q);
        return OR_OOM;
    }
    int status = local_diagonal(h, dl);
    if (status != OR_OK) {
        free(dl); free(bl); free(xl); free(r); free(z); free(p); free(q);
        return status;
    }
    status = OR_NOT_CONVERGED;
    or_scatter(h, b, bl);
    or_scatter(h, x, xl);
    or_sub_spmv(h, xl, q);
    for (int64_t k = 0; k < L; ++k) r[k] = bl[k] - q[k];
    for (int64_t k = 0; k < L; ++k) z[k] = r[k] / dl[k];
    for (int64_t k = 0; k < L; ++k) p[k] = z[k];
    double rz = or_wdot(h, r, z), rr = or_wdot(h, r, r);
    const double bnorm = sqrt(or_wdot(h, bl, bl));
    int32_t it = 0;
    if (sqrt(rr) <= rtol * bnorm) status = OR_OK;
    while (status == OR_NOT_CONVERGED && it < max_iter) {
        or_sub_spmv(h, p, q);
        const double pq = or_wdot(h, q, p);
        if (!(pq > 0.0) || !isfinite(pq)) {
            status = OR_BREAKDOWN;
            break;
        }
        const double alpha = rz / pq;
        for (int64_t k = 0; k < L; ++k) xl[k] = xl[k] + alpha * p[k];
        for (int64_t k = 0; k < L; ++k) r[k] = r[k] - alpha * q[k];
        for (int64_t k = 0; k < L; ++k) z[k] = r[k] / dl[k];
        const double rz_new = or_wdot(h, r, z);
        rr = or_wdot(h, r, r);
        const double beta = rz_new / rz;
        for (int64_t k = 0; k < L; ++k) p[k] = z[k] + beta * p[k];
        rz = rz_new;
        ++it;
        if (sqrt(rr) <= rtol * bnorm) status = OR_OK;
    }
    or_gather(h, xl, x);
    *iters_out = it;
    *relres_out = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
    free(dl); free(bl); free(xl); free(r); free(z); free(p); free(q);
    return status;
}

/* ------------------------------------------------------------------ */
/* Sub-structures by elements (Section 2.4, finite elements).          */
/* ------------------------------------------------------------------ */
typedef struct { int32_t s, r, c, e; double v; } fe_entry;
static int cmp_fe_entry(const void *x, const void *y) {
    const fe_entry *p = (const fe_entry *)x, *q = (const fe_entry *)y;
    if (p->s != q->s) return (p->s > q->s) - (p->s < q->s);
    if (p->r != q->r) return (p->r > q->r) - (p->r < q->r);
    if (p->c != q->c) return (p->c > q->c) - (p->c < q->c);
    return (p->e > q->e) - (p->e < q->e);
}
typedef struct { int32_t node, s; } fe_pair;
static int cmp_fe_pair(const void *x, const void *y) {
    const fe_pair *p = (const fe_pair *)x, *q = (const fe_pair *)y;
    if (p->node != q->node) return (p->node > q->node) - (p->node < q->node);
    return (p->s > q->s) - (p->s < q->s);
}

/*
 * Sub-structures from finite elements, as Section 2.4 builds them: subdomain s
 * owns the elements e with epart[e] = s, V_s is the set of free nodes of its
 * elements, and its local matrix is the sum of its own element matrices in
 * local numbering (S_s = sum over e in s of K_e), so the interface blocks of
 * the local matrices add up to the global interface block (Eq.
 * interface_summation) and every S_s is a Neumann matrix (positive
 * semi-definite).  Element e has nv nodes elem[e*nv + a] (-1: an eliminated
 * Dirichlet node) and the symmetric matrix kel[e*nv*nv + a*nv + b]; rows and
 * columns of eliminated nodes are dropped.  A local entry is the sum of its
 * element contributions in ascending element order.  Numbering, multiplicity,
 * interface lists and weights are those of or_partition; the owner copy of a
 * node is its copy in the lowest subdomain holding it.  Invalid: epart out of
 * range, a node index out of range, a free node in no element, a
 * non-symmetric element matrix.
 */
or_part *or_partition_fe(int32_t n, int32_t ne, int32_t nv, const int32_t *elem, const double *kel,
                         const int32_t *epart, int32_t P, int *status) {
    *status = OR_INVALID;
    if (n <= 0 || ne <= 0 || nv <= 0 || P <= 0) return NULL;
    for (int32_t e = 0; e < ne; ++e) {
        if (epart[e] < 0 || epart[e] >= P) return NULL;
        for (int32_t a = 0; a < nv; ++a) {
            if (elem[(int64_t)e * nv + a] < -1 || elem[(int64_t)e * nv + a] >= n) return NULL;
            for (int32_t b = 0; b < nv; ++b)
                if (kel[((int64_t)e * nv + a) * nv + b] != kel[((int64_t)e * nv + b) * nv + a]) return NULL;
        }
    }
    *status = OR_OOM;
    or_part *h = (or_part *)calloc(1, sizeof(or_part));
    const int64_t npair = (int64_t)ne * nv;
    fe_pair *pairs = (fe_pair *)malloc(sizeof(fe_pair) * (size_t)npair);
    int32_t *mem_ptr = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * (size_t)npair);
    int32_t *memloc = (int32_t *)malloc(sizeof(int32_t) * (size_t)npair);
    fe_entry *ent = (fe_entry *)malloc(sizeof(fe_entry) * (size_t)(npair * nv));
    int32_t *cnt = (int32_t *)calloc((size_t)P, sizeof(int32_t));
    if (!h || !pairs || !mem_ptr || !mem || !memloc || !ent || !cnt) goto fail;
    h->n = n;
    h->P = P;
    /* membership: sorted unique (node, subdomain) pairs */
    int64_t np = 0;
    for (int32_t e = 0; e < ne; ++e)
        for (int32_t a = 0; a < nv; ++a) {
            const int32_t i = elem[(int64_t)e * nv + a];
            if (i >= 0) { pairs[np].node = i; pairs[np].s = epart[e]; ++np; }
        }
    qsort(pairs, (size_t)np, sizeof(fe_pair), cmp_fe_pair);
    {
        int64_t w = 0;
        for (int64_t t = 0; t < np; ++t) {
            if (t > 0 && pairs[t].node == pairs[t - 1].node && pairs[t].s == pairs[t - 1].s) continue;
            mem[w] = pairs[t].s;
            mem_ptr[pairs[t].node + 1]++;
            ++w;
        }
        for (int32_t j = 0; j < n; ++j) mem_ptr[j + 1] += mem_ptr[j];
    }
    for (int32_t j = 0; j < n; ++j)
        if (mem_ptr[j + 1] == mem_ptr[j]) { *status = OR_INVALID; goto fail; }
    h->mult = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    h->off = (int32_t *)calloc((size_t)P + 1, sizeof(int32_t));
    h->nint = (int32_t *)calloc((size_t)P, sizeof(int32_t));
    if (!h->mult || !h->off || !h->nint) goto fail;
    for (int32_t j = 0; j < n; ++j) h->mult[j] = mem_ptr[j + 1] - mem_ptr[j];
    for (int32_t j = 0; j < n; ++j)
        for (int32_t t = mem_ptr[j]; t < mem_ptr[j + 1]; ++t) {
            cnt[mem[t]]++;
            if (h->mult[j] == 1) h->nint[mem[t]]++;
        }
    for (int32_t s = 0; s < P; ++s) h->off[s + 1] = h->off[s] + cnt[s];
    h->nloc = h->off[P];
    h->l2g = (int32_t *)malloc(sizeof(int32_t) * (size_t)h->nloc);
    if (!h->l2g) goto fail;
    for (int32_t s = 0; s < P; ++s) cnt[s] = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (int32_t j = 0; j < n; ++j) {
            if ((h->mult[j] >= 2) != pass) continue;
            for (int32_t t = mem_ptr[j]; t < mem_ptr[j + 1]; ++t) {
                const int32_t s = mem[t];
                memloc[t] = cnt[s]++;
                h->l2g[h->off[s] + memloc[t]] = j;
            }
        }
    h->own = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!h->own) goto fail;
    for (int32_t j = 0; j < n; ++j) h->own[j] = h->off[mem[mem_ptr[j]]] + memloc[mem_ptr[j]];
    /* local matrices: element contributions keyed by (s, local row, local column, e) */
    int64_t nent = 0;
    for (int32_t e = 0; e < ne; ++e) {
        const int32_t s = epart[e];
        for (int32_t a = 0; a < nv; ++a) {
            const int32_t i = elem[(int64_t)e * nv + a];
            if (i < 0) continue;
            int32_t li = -1;
            for (int32_t t = mem_ptr[i]; t < mem_ptr[i + 1]; ++t)
                if (mem[t] == s) li = memloc[t];
            for (int32_t b = 0; b < nv; ++b) {
                const int32_t j = elem[(int64_t)e * nv + b];
                if (j < 0) continue;
                int32_t lj = -1;
                for (int32_t t = mem_ptr[j]; t < mem_ptr[j + 1]; ++t)
                    if (mem[t] == s) lj = memloc[t];
                ent[nent].s = s;
                ent[nent].r = li;
                ent[nent].c = lj;
                ent[nent].e = e;
                ent[nent].v = kel[((int64_t)e * nv + a) * nv + b];
                ++nent;
            }
        }
    }
    qsort(ent, (size_t)nent, sizeof(fe_entry), cmp_fe_entry);
    h->lrowptr = (int32_t *)calloc((size_t)h->nloc + 1, sizeof(int32_t));
    h->lcol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nent > 0 ? nent : 1));
    h->lval = (double *)malloc(sizeof(double) * (size_t)(nent > 0 ? nent : 1));
    if (!h->lrowptr || !h->lcol || !h->lval) goto fail;
    {
        int64_t w = 0;
        for (int64_t t = 0; t < nent;) {
            int64_t u = t;
            double v = 0.0;
            while (u < nent && ent[u].s == ent[t].s && ent[u].r == ent[t].r && ent[u].c == ent[t].c) v = v + ent[u++].v;
            h->lcol[w] = ent[t].c;
            h->lval[w] = v;
            h->lrowptr[h->off[ent[t].s] + ent[t].r + 1]++;
            ++w;
            t = u;
        }
        for (int64_t k = 0; k < h->nloc; ++k) h->lrowptr[k + 1] += h->lrowptr[k];
        h->nnz = w;
    }
    /* interface lists and weights, as or_partition */
    h->ngamma = 0;
    h->ncopies = 0;
    for (int32_t j = 0; j < n; ++j)
        if (h->mult[j] >= 2) { h->ngamma++; h->ncopies += h->mult[j]; }
    h->gamma = (int32_t *)malloc(sizeof(int32_t) * (size_t)(h->ngamma > 0 ? h->ngamma : 1));
    h->iptr = (int32_t *)calloc((size_t)h->ngamma + 1, sizeof(int32_t));
    h->icopy = (int32_t *)malloc(sizeof(int32_t) * (size_t)(h->ncopies > 0 ? h->ncopies : 1));
    h->w = (double *)malloc(sizeof(double) * (size_t)h->nloc);
    if (!h->gamma || !h->iptr || !h->icopy || !h->w) goto fail;
    {
        int32_t g = 0;
        int64_t c = 0;
        for (int32_t j = 0; j < n; ++j) {
            if (h->mult[j] < 2) continue;
            h->gamma[g] = j;
            for (int32_t t = mem_ptr[j]; t < mem_ptr[j + 1]; ++t) h->icopy[c++] = h->off[mem[t]] + memloc[t];
            h->iptr[++g] = (int32_t)c;
        }
    }
    for (int64_t k = 0; k < h->nloc; ++k) h->w[k] = 1.0 / (double)h->mult[h->l2g[k]];
    free(pairs); free(mem_ptr); free(mem); free(memloc); free(ent); free(cnt);
    *status = OR_OK;
    return h;
fail:
    free(pairs); free(mem_ptr); free(mem); free(memloc); free(ent); free(cnt);
    or_part_free(h);
    return NULL;
}

/* ------------------------------------------------------------------ */
/* Mixed precision with the diagonal preconditioner.                   */
/* ------------------------------------------------------------------ */
/*
 * or_sub_cg_mixed with Algorithm 3's diagonal preconditioner in the inner
 * FP32 solves: z32 = r32 / (float) diag(S) (the assembled diagonal of
 * local_diagonal, rounded to FP32), alpha = (r32, z32)_w / (p32, S p32)_w,
 * beta = (r32, z32)_w(k+1) / (r32, z32)_w(k), p32 = z32 + beta p32; the inner
 * test stays on (r32, r32)_w: sqrt((r32, r32)_w) <= tau sqrt((r32, r32)_w at
 * the inner start).  The outer FP64 refinement is that of or_sub_cg_mixed.
 */
int or_sub_pcg_mixed(const or_part *h, const double *b, double *x, double rtol, int32_t max_iter,
                     double inner_rtol, int32_t max_outer, int32_t *iters_out, int32_t *outer_out,
                     double *relres_out) {
    size_t N = (size_t)(h->nloc > 0 ? h->nloc : 1);
    const int64_t L = h->nloc;
    double *bl = (double *)malloc(sizeof(double) * N), *xl = (double *)malloc(sizeof(double) * N);
    double *r = (double *)malloc(sizeof(double) * N), *q = (double *)malloc(sizeof(double) * N);
    double *dl = (double *)malloc(sizeof(double) * N);
    float *val32 = (float *)malloc(sizeof(float) * (size_t)(h->nnz > 0 ? h->nnz : 1));
    float *r32 = (float *)malloc(sizeof(float) * N), *z32 = (float *)malloc(sizeof(float) * N);
    float *p32 = (float *)malloc(sizeof(float) * N), *q32 = (float *)malloc(sizeof(float) * N);
    float *d32 = (float *)malloc(sizeof(float) * N), *g32 = (float *)malloc(sizeof(float) * N);
    int status = OR_OOM;
    if (!bl || !xl || !r || !q || !dl || !val32 || !r32 || !z32 || !p32 || !q32 || !d32 || !g32) goto done;
    status = local_diagonal(h, dl);
    if (status != OR_OK) goto done;
    for (int64_t k = 0; k < L; ++k) g32[k] = (float)dl[k];
    for (int64_t k = 0; k < h->nnz; ++k) val32[k] = (float)h->lval[k];
    or_scatter(h, b, bl);
    or_scatter(h, x, xl);
    or_sub_spmv(h, xl, q);
    for (int64_t k = 0; k < L; ++k) r[k] = bl[k] - q[k];
    double rho = or_wdot(h, r, r);
    const double bnorm = sqrt(or_wdot(h, bl, bl));
    int32_t outer = 0, total = 0;
    status = OR_NOT_CONVERGED;
    if (sqrt(rho) <= rtol * bnorm) status = OR_OK;
    while (status == OR_NOT_CONVERGED && outer < max_outer && total < max_iter) {
        double tau = rtol * bnorm / sqrt(rho);
        if (tau < inner_rtol) tau = inner_rtol;
        for (int64_t k = 0; k < L; ++k) {
            r32[k] = (float)r[k];
            z32[k] = r32[k] / g32[k];
            p32[k] = z32[k];
            d32[k] = 0.0f;
        }
        double rz = wdot32(h, r32, z32);
        double rr = wdot32(h, r32, r32);
        const double rr0 = rr;
        int broke = 0;
        while (sqrt(rr) > tau * sqrt(rr0) && total < max_iter) {
            sub_spmv32(h, val32, p32, q32);
            const double pq = wdot32(h, p32, q32);
            if (!(pq > 0.0) || !isfinite(pq)) {
                broke = 1;
                break;
            }
            const float alpha = (float)(rz / pq);
            for (int64_t k = 0; k < L; ++k) d32[k] = d32[k] + alpha * p32[k];
            for (int64_t k = 0; k < L; ++k) r32[k] = r32[k] - alpha * q32[k];
            for (int64_t k = 0; k < L; ++k) z32[k] = r32[k] / g32[k];
            const double rz_new = wdot32(h, r32, z32);
            rr = wdot32(h, r32, r32);
            const float beta = (float)(rz_new / rz);
            for (int64_t k = 0; k < L; ++k) p32[k] = z32[k] + beta * p32[k];
            rz = rz_new;
            ++total;
        }
        for (int64_t k = 0; k < L; ++k) xl[k] = xl[k] + (double)d32[k];
        or_sub_spmv(h, xl, q);
        for (int64_t k = 0; k < L; ++k) r[k] = bl[k] - q[k];
        rho = or_wdot(h, r, r);
        ++outer;
        if (sqrt(rho) <= rtol * bnorm) status = OR_OK;
        else if (broke) status = OR_BREAKDOWN;
    }
    or_gather(h, xl, x);
    *iters_out = total;
    *outer_out = outer;
    *relres_out = bnorm > 0.0 ? sqrt(rho) / bnorm : 0.0;
done:
    free(bl); free(xl); free(r); free(q); free(dl); free(val32); free(r32); free(z32); free(p32); free(q32);
    free(d32); free(g32);
    return status;
}

/* ------------------------------------------------------------------ */
/* Band splittings (Section 2.1 Algorithm 1, Section 2.2 Algorithm 2). */
/* ------------------------------------------------------------------ */

/*
 * Extent of band p of nb: q = floor(n / nb) rows (Algorithm 1) or columns
 * (Algorithm 2) per band, the last band taking the rest, n - (nb-1) q.
 * Reading: bands are numbered 0..nb-1 (the listing mixes 1- and 0-based
 * numbering); 0 < nb <= n.  Returns OR_INVALID otherwise.
 */
static int band_extent(int32_t n, int32_t nb, int32_t p, int32_t *np, int32_t *displ) {
    if (n <= 0 || nb <= 0 || nb > n || p < 0 || p >= nb) return OR_INVALID;
    const int32_t q = n / nb;
    *displ = p * q;
    *np = (p == nb - 1) ? n - p * q : q;
    return OR_OK;
}

/*
 * Algorithm 1, band-row splitting: band p holds rows [displ, displ + N_p) of
 * A as an N_p x n CSR matrix.  Its row pointers are A's, shifted so that the
 * band starts at 0; its column ids (global, 0..n-1) and values are A's
 * entries of those rows, copied in order.  sizes[0..2] = N_p, displ,
 * nnz_count.  brow (N_p + 1), bcol and bval (nnz_count) may be NULL to query
 * the sizes only.
 */
int or_band_row(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val, int32_t nb,
                int32_t p, int64_t *sizes, int32_t *brow, int32_t *bcol, double *bval) {
    int32_t np, displ;
    if (band_extent(n, nb, p, &np, &displ) != OR_OK) return OR_INVALID;
    const int32_t nnz_displ = rowptr[displ];
    const int32_t nnz_count = rowptr[displ + np] - nnz_displ;
    sizes[0] = np;
    sizes[1] = displ;
    sizes[2] = nnz_count;
    if (brow) {
        for (int32_t i = 0; i <= np; ++i) brow[i] = rowptr[displ + i] - nnz_displ;
        for (int32_t k = 0; k < nnz_count; ++k) {
            bcol[k] = colidx[nnz_displ + k];
            bval[k] = val[nnz_displ + k];
        }
    }
    return OR_OK;
}

/*
 * Algorithm 2, band-column splitting: band p holds columns [displ, displ +
 * N_p) of A as an n x N_p CSR matrix: every row of A, keeping (in order) the
 * entries whose column lies in the band, with the column id shifted by displ
 * (reading: the listing's column offset is the band's first column, and its
 * inner loop runs over row i of A).  sizes as for or_band_row; brow has n + 1
 * entries.
 */
int or_band_col(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val, int32_t nb,
                int32_t p, int64_t *sizes, int32_t *brow, int32_t *bcol, double *bval) {
    int32_t np, displ;
    if (band_extent(n, nb, p, &np, &displ) != OR_OK) return OR_INVALID;
    int64_t c = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (brow) brow[i] = (int32_t)c;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            if (displ <= colidx[k] && colidx[k] < displ + np) {
                if (brow) {
                    bcol[c] = colidx[k] - displ;
                    bval[c] = val[k];
                }
                ++c;
            }
        }
    }
    if (brow) brow[n] = (int32_t)c;
    sizes[0] = np;
    sizes[1] = displ;
    sizes[2] = c;
    return OR_OK;
}

/*
 * y = A x through the band-row splitting: every band multiplies its rows by
 * the whole of x (rows in order, each summed left to right) and writes its
 * block y[displ .. displ + N_p).
 */
int or_band_row_spmv(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val, int32_t nb,
                     const double *x, double *y) {
    for (int32_t p = 0; p < nb; ++p) {
        int64_t sz[3];
        if (or_band_row(n, rowptr, colidx, val, nb, p, sz, NULL, NULL, NULL) != OR_OK) return OR_INVALID;
        int32_t *br = (int32_t *)malloc(sizeof(int32_t) * (size_t)(sz[0] + 1));
        int32_t *bc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(sz[2] > 0 ? sz[2] : 1));
        double *bv = (double *)malloc(sizeof(double) * (size_t)(sz[2] > 0 ? sz[2] : 1));
        if (!br || !bc || !bv) {
            free(br); free(bc); free(bv);
            return OR_OOM;
        }
        or_band_row(n, rowptr, colidx, val, nb, p, sz, br, bc, bv);
        or_spmv((int32_t)sz[0], br, bc, bv, x, y + sz[1]);
        free(br); free(bc); free(bv);
    }
    return OR_OK;
}

/*
 * y = A x through the band-column splitting: band p forms the partial
 * product y_p = A_p x[displ .. displ + N_p) (n entries, each row summed left
 * to right), and y is the sum of the partials taken in ascending p, starting
 * from zero (reading: the paper does not give the order in which the bands'
 * contributions are summed; one fixed order makes the result reproducible).
 */
int or_band_col_spmv(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val, int32_t nb,
                     const double *x, double *y) {
    double *yp = (double *)malloc(sizeof(double) * (size_t)n);
    if (!yp) return OR_OOM;
    for (int32_t i = 0; i < n; ++i) y[i] = 0.0;
    for (int32_t p = 0; p < nb; ++p) {
        int64_t sz[3];
        if (or_band_col(n, rowptr, colidx, val, nb, p, sz, NULL, NULL, NULL) != OR_OK) {
            free(yp);
            return OR_INVALID;
        }
        int32_t *br = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
        int32_t *bc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(sz[2] > 0 ? sz[2] : 1));
        double *bv = (double *)malloc(sizeof(double) * (size_t)(sz[2] > 0 ? sz[2] : 1));
        if (!br || !bc || !bv) {
            free(br); free(bc); free(bv); free(yp);
            return OR_OOM;
        }
        or_band_col(n, rowptr, colidx, val, nb, p, sz, br, bc, bv);
        or_spmv(n, br, bc, bv, x + sz[1], yp);
        for (int32_t i = 0; i < n; ++i) y[i] += yp[i];
        free(br); free(bc); free(bv);
    }
    free(yp);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* The sub-structured CG with the subdomains shared among CPU threads. */
/* ------------------------------------------------------------------ */
/*
 * Baseline timing on all host cores (TEST INFRASTRUCTURE like the rest of
 * this file).  Section 3.4.2 gives each subdomain to its own process; here
 * threads stand in for the processes:
 *   - the local products run subdomain by subdomain in parallel, and the
 *     interface sums node by node in parallel (a node writes only its own
 *     copies), each entry computed exactly as in or_sub_spmv;
 *   - the vector updates run entry by entry in parallel, as in or_sub_cg;
 *   - every weighted dot is formed the way the paper's processes form it:
 *     each subdomain sums its own entries in order, then the subdomain sums
 *     are added in ascending s.
 * So the result does not depend on the number of threads, and it differs
 * from or_sub_cg only in how the dot sums are grouped (one running sum
 * there); with one subdomain the two compute the same bits.  nthreads <= 0
 * uses every thread OpenMP offers.  Built without OpenMP, it runs on one
 * thread with the same results.
 */
#ifdef _OPENMP
#include <omp.h>
#endif

int or_omp_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static void sub_spmv_par(const or_part *h, const double *xl, double *yl, int nt) {
#pragma omp parallel num_threads(nt)
    {
#pragma omp for schedule(dynamic, 1)
        for (int32_t s = 0; s < h->P; ++s) {
            const int32_t o = h->off[s];
            for (int32_t li = 0; li < h->off[s + 1] - o; ++li) {
                double acc = 0.0;
                for (int32_t k = h->lrowptr[o + li]; k < h->lrowptr[o + li + 1]; ++k)
                    acc = acc + h->lval[k] * xl[h->lcol[k] + o];
                yl[o + li] = acc;
            }
        }
#pragma omp for schedule(static)
        for (int32_t g = 0; g < h->ngamma; ++g) {
            double S = 0.0;
            for (int32_t c = h->iptr[g]; c < h->iptr[g + 1]; ++c) S += yl[h->icopy[c]];
            for (int32_t c = h->iptr[g]; c < h->iptr[g + 1]; ++c) yl[h->icopy[c]] = S;
        }
    }
}

static double wdot_by_subdomain(const or_part *h, const double *u, const double *v, double *part, int nt) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int32_t s = 0; s < h->P; ++s) {
        double acc = 0.0;
        for (int64_t k = h->off[s]; k < h->off[s + 1]; ++k) acc += h->w[k] * u[k] * v[k];
        part[s] = acc;
    }
    double t = 0.0;
    for (int32_t s = 0; s < h->P; ++s) t += part[s];
    return t;
}

int or_sub_cg_omp(const or_part *h, const double *b, double *x, double rtol, int32_t max_iter, int32_t nthreads,
                  int32_t *iters_out, double *relres_out) {
    const int nt = nthreads > 0 ? nthreads : or_omp_max_threads();
    size_t N = (size_t)(h->nloc > 0 ? h->nloc : 1);
    double *bl = (double *)malloc(sizeof(double) * N);
    double *xl = (double *)malloc(sizeof(double) * N);
    double *r = (double *)malloc(sizeof(double) * N);
    double *p = (double *)malloc(sizeof(double) * N);
    double *q = (double *)malloc(sizeof(double) * N);
    double *part = (double *)malloc(sizeof(double) * (size_t)(h->P > 0 ? h->P : 1));
    if (!bl || !xl || !r || !p || !q || !part) {
        free(bl); free(xl); free(r); free(p); free(q); free(part);
        return OR_OOM;
    }
    const int64_t L = h->nloc;
    or_scatter(h, b, bl);
    or_scatter(h, x, xl);
    sub_spmv_par(h, xl, q, nt);
#pragma omp parallel for schedule(static) num_threads(nt)
    for (int64_t k = 0; k < L; ++k) {
        r[k] = bl[k] - q[k];
        p[k] = r[k];
    }
    double rho = wdot_by_subdomain(h, r, r, part, nt);
    double bnorm = sqrt(wdot_by_subdomain(h, bl, bl, part, nt));
    int status = OR_NOT_CONVERGED;
    int32_t it = 0;
    double relres = bnorm > 0.0 ? sqrt(rho) / bnorm : 0.0;
    if (sqrt(rho) <= rtol * bnorm) status = OR_OK;
    while (status == OR_NOT_CONVERGED && it < max_iter) {
        sub_spmv_par(h, p, q, nt);
        double pq = wdot_by_subdomain(h, q, p, part, nt);
        if (!(pq > 0.0) || !isfinite(pq)) {
            status = OR_BREAKDOWN;
            break;
        }
        double alpha = rho / pq;
#pragma omp parallel for schedule(static) num_threads(nt)
        for (int64_t k = 0; k < L; ++k) {
            xl[k] = xl[k] + alpha * p[k];
            r[k] = r[k] - alpha * q[k];
        }
        double rho_new = wdot_by_subdomain(h, r, r, part, nt);
        double beta = rho_new / rho;
#pragma omp parallel for schedule(static) num_threads(nt)
        for (int64_t k = 0; k < L; ++k) p[k] = r[k] + beta * p[k];
        rho = rho_new;
        ++it;
        relres = bnorm > 0.0 ? sqrt(rho) / bnorm : 0.0;
        if (sqrt(rho) <= rtol * bnorm) status = OR_OK;
    }
    or_gather(h, xl, x);
    *iters_out = it;
    *relres_out = relres;
    free(bl); free(xl); free(r); free(p); free(q); free(part);
    return status;
}
