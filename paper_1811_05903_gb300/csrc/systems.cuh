// Lookup of the independent system (single simulation or ensemble member)
// that holds a stream-K unit or a tile, by binary search in the system table.
#pragma once

#include <stdint.h>

#include "steps_internal.h"

namespace steps {

// System holding stream-K unit u (last table entry whose unit_off <= u).
__device__ __forceinline__ int sim_of_unit(const SimDesc *__restrict__ sims, int nsims, int64_t u) {
    int lo = 0, hi = nsims;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (sims[mid].unit_off <= u) lo = mid; else hi = mid;
    }
    return lo;
}

// System holding global tile r.
__device__ __forceinline__ int sim_of_tile(const SimDesc *__restrict__ sims, int nsims, int64_t r) {
    int lo = 0, hi = nsims;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (sims[mid].tile_off <= r) lo = mid; else hi = mid;
    }
    return lo;
}

}  // namespace steps
