// The cardinality estimate of Sec. 5.2 from a vertex's (start, duration) density histogram,
// shared by the edge-map's access choice and the estimate entry point.
//
// Bucket i of a span [lo, lo + span) holds the integers [lo + ceil(i span / B), lo +
// ceil((i + 1) span / B) - 1] (possibly none) and its centre is the floor of the mean of those
// ends.  A predicate "departure in [a, b], arrival t + lam <= tw" counts every edge of a
// bucket (i, j) whose centres satisfy it: a <= centre_i <= b and centre_i + centre_j <= tw.
// Everything is exact integer arithmetic.
#pragma once
#include <stdint.h>

#include "common.cuh"

namespace kairos {

__host__ __device__ __forceinline__ uint64_t hist_first(uint64_t lo, uint64_t span, int i) {
    return lo + ((uint64_t)i * span + HIST_B - 1) / HIST_B;
}

__host__ __device__ __forceinline__ uint64_t hist_centre(uint64_t lo, uint64_t span, int i) {
    return (hist_first(lo, span, i) + hist_first(lo, span, i + 1) - 1) / 2;
}

// Edges of the histogram's vertex counted towards departure in [a, b] and arrival <= tw;
// cum = its HIST_B x HIST_B row-wise inclusive prefix sums.
__device__ __forceinline__ uint64_t hist_estimate(const HistHdr &h, const uint32_t *__restrict__ cum, uint64_t a,
                                                  uint64_t b, uint64_t tw) {
    uint64_t est = 0;
    const uint64_t dlast = hist_centre(h.lmin, h.D, HIST_B - 1);
    for (int i = 0; i < HIST_B; ++i) {
        const uint64_t s0 = hist_first(h.tmin, h.S, i), s1 = hist_first(h.tmin, h.S, i + 1) - 1;
        if (s0 > s1) continue;  // no integer start in this bucket
        const uint64_t sc = (s0 + s1) / 2;
        if (sc > b) break;  // centres only grow with i
        if (sc < a || sc > tw) continue;
        const uint64_t cap = tw - sc;
        int J;
        if (dlast <= cap) {
            J = HIST_B - 1;
        } else {  // the buckets whose centre is at most cap form a prefix
            int lo = 0, hi = HIST_B - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (hist_centre(h.lmin, h.D, mid) <= cap) lo = mid + 1; else hi = mid;
            }
            J = lo - 1;
        }
        if (J >= 0) est += __ldg(&cum[i * HIST_B + J]);
    }
    return est;
}

}  // namespace kairos
