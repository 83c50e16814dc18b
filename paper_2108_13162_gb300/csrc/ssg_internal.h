// Internal definitions shared by the library's translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "ssg.h"

namespace ssg {

// Host-side sub-structure maps (Section 2.4 and Section 3.4.2), built by
// build_host_maps() in partition.cpp.
struct HostMaps {
    int32_t n = 0, P = 0;
    int64_t nnz = 0, nloc = 0;
    int32_t ngamma = 0, max_mult = 0;
    int64_t ncopies = 0;
    std::vector<int32_t> off, nint, l2g, mult, lrowptr, lcol, gamma, iptr, icopy, own;
    std::vector<double> lval;
    std::vector<int32_t> lsrc;  // entry of the input CSR each local entry copies (ownership is one-to-one);
                                // empty for element sub-structures (local entries are sums)
    std::vector<double> diag;   // element sub-structures: assembled diagonal per node
};

// Returns SSG_OK or SSG_E_INVALID / SSG_E_OOM with a message in *err.
int build_host_maps(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                    const int32_t *part, int32_t P, HostMaps &out, std::string *err);

int build_host_maps_fe(int32_t n, int32_t ne, int32_t nv, const int32_t *elem, const double *kel,
                       const int32_t *epart, int32_t P, HostMaps &out, std::string *err);

void set_error(const std::string &msg);

}  // namespace ssg
