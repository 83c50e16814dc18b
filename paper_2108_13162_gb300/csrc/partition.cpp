// Host construction of the sub-structures (Section 2.4) for an assembled CSR
// matrix: subdomain node sets, multiplicities, interior-then-interface local
// numbering (Eq. 2.4:eqn0), local matrices whose interface blocks sum to the
// global one (Eq. mat_subdomains / interface_summation) and the interface
// lists of Section 3.4.2.  Integer work only; the values are copied.
//
// Rules (the paper only describes the split of S_33 through finite-element
// assembly; for an assembled matrix this library takes entry ownership):
//   diagonal (i,i)   -> subdomain part(i)
//   entry (i,j)      -> subdomain min(part(i), part(j))
//   V_s              -> nodes of s plus every node j with part(j) > s that
//                       shares a stored entry with a node of s
#include <algorithm>
#include <cstring>
#include <new>

#include "ssg_internal.h"

namespace ssg {

namespace {

bool validate(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val, const int32_t *part,
              int32_t P, std::string *err) {
    if (n <= 0) { *err = "n must be positive"; return false; }
    if (P <= 0 || P > 65535) { *err = "P must be in [1, 65535]"; return false; }
    if (!rowptr || !colidx || !val || !part) { *err = "null input array"; return false; }
    if (rowptr[0] != 0) { *err = "rowptr[0] must be 0"; return false; }
    for (int32_t i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i]) { *err = "rowptr not non-decreasing at row " + std::to_string(i); return false; }
        if (part[i] < 0 || part[i] >= P) { *err = "part id out of range at node " + std::to_string(i); return false; }
    }
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            int32_t j = colidx[k];
            if (j < 0 || j >= n) { *err = "column index out of range in row " + std::to_string(i); return false; }
            if (k > rowptr[i] && j <= colidx[k - 1]) {
                *err = "columns not sorted/unique in row " + std::to_string(i);
                return false;
            }
        }
    }
    // symmetric pattern and values
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            int32_t j = colidx[k];
            const int32_t *b = colidx + rowptr[j], *e = colidx + rowptr[j + 1];
            const int32_t *t = std::lower_bound(b, e, i);
            if (t == e || *t != i) {
                *err = "pattern not symmetric at (" + std::to_string(i) + "," + std::to_string(j) + ")";
                return false;
            }
            if (val[t - colidx] != val[k]) {
                *err = "values not symmetric at (" + std::to_string(i) + "," + std::to_string(j) + ")";
                return false;
            }
        }
    }
    return true;
}

}  // namespace

int build_host_maps(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                    const int32_t *part, int32_t P, HostMaps &M, std::string *err) {
    if (!validate(n, rowptr, colidx, val, part, P, err)) return SSG_E_INVALID;
    try {
        M = HostMaps();
        M.n = n;
        M.P = P;
        M.nnz = rowptr[n];
        // 1. membership lists: for node j the sorted subdomains holding it,
        //    part(j) plus the lower part ids of its neighbours.
        std::vector<int64_t> mptr(static_cast<size_t>(n) + 1, 0);
        std::vector<int32_t> mem;
        mem.reserve(static_cast<size_t>(n) + static_cast<size_t>(M.nnz) / 4);
        std::vector<int32_t> tmp;
        for (int32_t j = 0; j < n; ++j) {
            tmp.clear();
            const int32_t pj = part[j];
            tmp.push_back(pj);
            for (int32_t k = rowptr[j]; k < rowptr[j + 1]; ++k) {
                const int32_t pi = part[colidx[k]];
                if (pi < pj) tmp.push_back(pi);
            }
            std::sort(tmp.begin(), tmp.end());
            tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
            if (tmp.size() > 255) {
                *err = "node " + std::to_string(j) + " is shared by more than 255 subdomains";
                return SSG_E_INVALID;
            }
            mem.insert(mem.end(), tmp.begin(), tmp.end());
            mptr[j + 1] = static_cast<int64_t>(mem.size());
        }
        M.mult.resize(n);
        M.max_mult = 0;
        for (int32_t j = 0; j < n; ++j) {
            M.mult[j] = static_cast<int32_t>(mptr[j + 1] - mptr[j]);
            M.max_mult = std::max(M.max_mult, M.mult[j]);
        }
        // 2. sizes and local numbering (interior first, then interface, ascending ids)
        std::vector<int64_t> cnt(P, 0);
        M.nint.assign(P, 0);
        for (int32_t j = 0; j < n; ++j)
            for (int64_t t = mptr[j]; t < mptr[j + 1]; ++t) {
                cnt[mem[t]]++;
                if (M.mult[j] == 1) M.nint[mem[t]]++;
            }
        M.off.assign(static_cast<size_t>(P) + 1, 0);
        int64_t acc = 0;
        for (int32_t s = 0; s < P; ++s) {
            acc += cnt[s];
            if (acc > INT32_MAX - 1) { *err = "sum of subdomain sizes exceeds int32"; return SSG_E_INVALID; }
            M.off[s + 1] = static_cast<int32_t>(acc);
        }
        M.nloc = acc;
        std::vector<int32_t> loc(mem.size());  // local index of node j in mem[t]
        M.l2g.assign(static_cast<size_t>(M.nloc), 0);
        std::vector<int32_t> fill(P, 0);
        for (int pass = 0; pass < 2; ++pass)
            for (int32_t j = 0; j < n; ++j) {
                if ((M.mult[j] >= 2) != (pass == 1)) continue;
                for (int64_t t = mptr[j]; t < mptr[j + 1]; ++t) {
                    const int32_t s = mem[t];
                    loc[t] = fill[s]++;
                    M.l2g[static_cast<size_t>(M.off[s]) + loc[t]] = j;
                }
            }
        M.own.assign(n, 0);
        for (int32_t j = 0; j < n; ++j)
            for (int64_t t = mptr[j]; t < mptr[j + 1]; ++t)
                if (mem[t] == part[j]) M.own[j] = M.off[mem[t]] + loc[t];
        // 3. local matrices: row of node i in s keeps the entries owned by s,
        //    columns renumbered to s's local ids and sorted.
        M.lrowptr.assign(static_cast<size_t>(M.nloc) + 1, 0);
        M.lcol.resize(static_cast<size_t>(M.nnz));
        M.lval.resize(static_cast<size_t>(M.nnz));
        M.lsrc.resize(static_cast<size_t>(M.nnz));
        std::vector<std::pair<int32_t, int32_t>> row;  // (local column, entry of the input CSR)
        int64_t w = 0;
        for (int32_t s = 0; s < P; ++s) {
            const int32_t ns = M.off[s + 1] - M.off[s];
            for (int32_t li = 0; li < ns; ++li) {
                const int32_t i = M.l2g[static_cast<size_t>(M.off[s]) + li];
                const int32_t pi = part[i];
                row.clear();
                for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
                    const int32_t j = colidx[k];
                    const int32_t pj = part[j];
                    const int32_t owner = (i == j) ? pi : std::min(pi, pj);
                    if (owner != s) continue;
                    const int32_t *mb = mem.data() + mptr[j], *me = mem.data() + mptr[j + 1];
                    const int32_t *f = std::lower_bound(mb, me, s);
                    if (f == me || *f != s) { *err = "internal: column node missing from subdomain"; return SSG_E_INVALID; }
                    row.emplace_back(loc[f - mem.data()], k);
                }
                std::sort(row.begin(), row.end(),
                          [](const std::pair<int32_t, int32_t> &a, const std::pair<int32_t, int32_t> &b) {
                              return a.first < b.first;
                          });
                for (auto &e : row) {
                    M.lcol[w] = e.first;
                    M.lval[w] = val[e.second];
                    M.lsrc[w] = e.second;
                    ++w;
                }
                M.lrowptr[static_cast<size_t>(M.off[s]) + li + 1] = static_cast<int32_t>(w);
            }
        }
        if (w != M.nnz) { *err = "internal: entry ownership does not cover the matrix"; return SSG_E_INVALID; }
        // 4. interface lists: nodes with m >= 2 ascending, copies in ascending s
        M.ngamma = 0;
        M.ncopies = 0;
        for (int32_t j = 0; j < n; ++j)
            if (M.mult[j] >= 2) {
                M.ngamma++;
                M.ncopies += M.mult[j];
            }
        M.gamma.resize(M.ngamma);
        M.iptr.assign(static_cast<size_t>(M.ngamma) + 1, 0);
        M.icopy.resize(static_cast<size_t>(M.ncopies));
        int32_t g = 0;
        int64_t c = 0;
        for (int32_t j = 0; j < n; ++j) {
            if (M.mult[j] < 2) continue;
            M.gamma[g] = j;
            for (int64_t t = mptr[j]; t < mptr[j + 1]; ++t) M.icopy[c++] = M.off[mem[t]] + loc[t];
            M.iptr[++g] = static_cast<int32_t>(c);
        }
    } catch (const std::bad_alloc &) {
        *err = "host allocation failed while building the sub-structures";
        return SSG_E_OOM;
    }
    return SSG_OK;
}

}  // namespace ssg
