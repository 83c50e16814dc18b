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

// Sub-structures from finite elements (Section 2.4): subdomain s owns the
// elements with epart[e] = s, V_s is the set of free nodes of its elements and
// its local matrix is the sum of its own element matrices in local numbering,
// each local entry summed in ascending element order; interface blocks of the
// local matrices add up to the global one (Eq. interface_summation).  The
// numbering, multiplicities and interface lists follow the assembled-matrix
// rules; the owner copy of a node is its copy in the lowest subdomain.  Also
// returns, in M.diag, the assembled diagonal: per node the sum over its copies
// (ascending s) of the local diagonal entries.
int build_host_maps_fe(int32_t n, int32_t ne, int32_t nv, const int32_t *elem, const double *kel,
                       const int32_t *epart, int32_t P, HostMaps &M, std::string *err) {
    if (n <= 0 || ne <= 0 || nv <= 0 || nv > 64) { *err = "need n > 0, ne > 0, 1 <= nv <= 64"; return SSG_E_INVALID; }
    if (P <= 0 || P > 65535) { *err = "P must be in [1, 65535]"; return SSG_E_INVALID; }
    if (!elem || !kel || !epart) { *err = "null input array"; return SSG_E_INVALID; }
    for (int32_t e = 0; e < ne; ++e) {
        if (epart[e] < 0 || epart[e] >= P) { *err = "element part id out of range at " + std::to_string(e); return SSG_E_INVALID; }
        for (int32_t a = 0; a < nv; ++a) {
            const int32_t i = elem[static_cast<int64_t>(e) * nv + a];
            if (i < -1 || i >= n) { *err = "element node out of range at element " + std::to_string(e); return SSG_E_INVALID; }
            for (int32_t b = 0; b < nv; ++b)
                if (kel[(static_cast<int64_t>(e) * nv + a) * nv + b] != kel[(static_cast<int64_t>(e) * nv + b) * nv + a]) {
                    *err = "element matrix not symmetric at element " + std::to_string(e);
                    return SSG_E_INVALID;
                }
        }
    }
    try {
        M = HostMaps();
        M.n = n;
        M.P = P;
        // 1. membership: subdomains of the elements around each node
        std::vector<int64_t> mptr(static_cast<size_t>(n) + 1, 0);
        for (int64_t t = 0; t < static_cast<int64_t>(ne) * nv; ++t)
            if (elem[t] >= 0) mptr[elem[t] + 1]++;
        for (int32_t j = 0; j < n; ++j) mptr[j + 1] += mptr[j];
        std::vector<int32_t> raw(static_cast<size_t>(mptr[n]));
        {
            std::vector<int64_t> fill(mptr.begin(), mptr.end() - 1);
            for (int32_t e = 0; e < ne; ++e)
                for (int32_t a = 0; a < nv; ++a) {
                    const int32_t i = elem[static_cast<int64_t>(e) * nv + a];
                    if (i >= 0) raw[fill[i]++] = epart[e];
                }
        }
        std::vector<int64_t> mp2(static_cast<size_t>(n) + 1, 0);
        std::vector<int32_t> mem;
        mem.reserve(raw.size());
        for (int32_t j = 0; j < n; ++j) {
            if (mptr[j + 1] == mptr[j]) { *err = "node " + std::to_string(j) + " belongs to no element"; return SSG_E_INVALID; }
            std::sort(raw.begin() + mptr[j], raw.begin() + mptr[j + 1]);
            const size_t before = mem.size();
            for (int64_t t = mptr[j]; t < mptr[j + 1]; ++t)
                if (t == mptr[j] || raw[t] != raw[t - 1]) mem.push_back(raw[t]);
            if (mem.size() - before > 255) {
                *err = "node " + std::to_string(j) + " is shared by more than 255 subdomains";
                return SSG_E_INVALID;
            }
            mp2[j + 1] = static_cast<int64_t>(mem.size());
        }
        mptr.swap(mp2);
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
        std::vector<int32_t> loc(mem.size());
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
        for (int32_t j = 0; j < n; ++j) M.own[j] = M.off[mem[mptr[j]]] + loc[mptr[j]];
        auto local_of = [&](int32_t i, int32_t s) {
            const int32_t *b = mem.data() + mptr[i], *e = mem.data() + mptr[i + 1];
            return loc[std::lower_bound(b, e, s) - mem.data()];
        };
        // 3. local matrices: element contributions in ascending element order,
        //    then a stable sort by (row, column) keeps that order for the sums
        std::vector<int32_t> eptr(static_cast<size_t>(P) + 1, 0), eord(ne);
        for (int32_t e = 0; e < ne; ++e) eptr[epart[e] + 1]++;
        for (int32_t s = 0; s < P; ++s) eptr[s + 1] += eptr[s];
        {
            std::vector<int32_t> ef(eptr.begin(), eptr.end() - 1);
            for (int32_t e = 0; e < ne; ++e) eord[ef[epart[e]]++] = e;
        }
        struct Contrib {
            int32_t r, c;
            double v;
        };
        std::vector<Contrib> con;
        M.lrowptr.assign(static_cast<size_t>(M.nloc) + 1, 0);
        for (int32_t s = 0; s < P; ++s) {
            con.clear();
            for (int32_t q = eptr[s]; q < eptr[s + 1]; ++q) {
                const int32_t e = eord[q];
                for (int32_t a = 0; a < nv; ++a) {
                    const int32_t i = elem[static_cast<int64_t>(e) * nv + a];
                    if (i < 0) continue;
                    const int32_t li = local_of(i, s);
                    for (int32_t b = 0; b < nv; ++b) {
                        const int32_t j = elem[static_cast<int64_t>(e) * nv + b];
                        if (j < 0) continue;
                        con.push_back({li, local_of(j, s), kel[(static_cast<int64_t>(e) * nv + a) * nv + b]});
                    }
                }
            }
            std::stable_sort(con.begin(), con.end(), [](const Contrib &x, const Contrib &y) {
                return x.r != y.r ? x.r < y.r : x.c < y.c;
            });
            for (size_t t = 0; t < con.size();) {
                size_t u = t;
                double v = 0.0;
                while (u < con.size() && con[u].r == con[t].r && con[u].c == con[t].c) v = v + con[u++].v;
                M.lcol.push_back(con[t].c);
                M.lval.push_back(v);
                M.lrowptr[static_cast<size_t>(M.off[s]) + con[t].r + 1]++;
                t = u;
            }
        }
        for (int64_t k = 0; k < M.nloc; ++k) M.lrowptr[k + 1] += M.lrowptr[k];
        M.nnz = static_cast<int64_t>(M.lval.size());
        if (M.nnz > INT32_MAX - 1) { *err = "local matrices exceed int32 entries"; return SSG_E_INVALID; }
        // 4. assembled diagonal: sum over the copies (ascending s) of the local diagonal entries
        M.diag.assign(n, 0.0);
        for (int32_t s = 0; s < P; ++s)
            for (int64_t r = M.off[s]; r < M.off[s + 1]; ++r)
                for (int32_t e = M.lrowptr[r]; e < M.lrowptr[r + 1]; ++e)
                    if (M.off[s] + M.lcol[e] == r) M.diag[M.l2g[r]] = M.diag[M.l2g[r]] + M.lval[e];
        // 5. interface lists: nodes with m >= 2 ascending, copies in ascending s
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
