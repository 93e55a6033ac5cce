// Storage plan of a batch of systems (host code, plain C++): how each
// system's Hamiltonian is held within a byte budget, 12 bytes per stored
// nonzero.  Systems are taken in ascending order of their connected pair
// count (ties by index).  When the upper triangles of all systems fit, every
// system is stored: as both triangles for as many systems as the rest of the
// budget takes (each costs 12 more bytes per pair), as its upper triangle for
// the others.  Otherwise upper triangles are stored in that order while they
// fit and the remaining systems are applied on the fly.  Every system's bytes
// buy about the same product time per byte in either form, so the order only
// decides how many systems get the faster form: small first gives the most.
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

#include "shci.h"

namespace shci {

inline std::vector<int> storage_plan(const std::vector<int64_t> &nnz_upper, double budget_bytes) {
    const size_t n = nnz_upper.size();
    std::vector<int> order(n), modes(n, SHCI_ON_THE_FLY);
    for (size_t s = 0; s < n; s++) order[s] = (int)s;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return nnz_upper[x] < nnz_upper[y]; });
    double all_upper = 0.0;
    for (int64_t v : nnz_upper) all_upper += 12.0 * (double)v;
    double left = budget_bytes;
    if (all_upper <= left) {
        left -= all_upper;
        for (int s : order) {
            const double extra = 12.0 * (double)nnz_upper[s];
            if (extra <= left) {
                modes[s] = SHCI_STORED;
                left -= extra;
            } else {
                modes[s] = SHCI_STORED_UPPER;
            }
        }
    } else {
        for (int s : order) {
            const double need = 12.0 * (double)nnz_upper[s];
            if (need > left) break;
            modes[s] = SHCI_STORED_UPPER;
            left -= need;
        }
    }
    return modes;
}

}  // namespace shci
