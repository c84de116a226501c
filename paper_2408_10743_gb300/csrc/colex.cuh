// colex.cuh -- t-subsets of {0..n-1} in colexicographic order, for the
// isometry kernel (host and device).
//
// A subset c[0] < c[1] < ... < c[t-1] has rank sum_i C(c[i], i + 1) (the
// combinatorial number system); consecutive subsets mostly differ in c[0]
// alone, which runs from 0 to c[1] - 1 before a higher element moves.
#pragma once
#include "dist_types.h"

#if defined(__CUDACC__)
#define DIST_CX __host__ __device__ __forceinline__
#else
#define DIST_CX inline
#endif

namespace dist {

// B: binomial table, B[m * stride + k] = C(m, k) for m <= n, k <= t.
DIST_CX void colex_unrank(const unsigned long long* B, int stride, int n, unsigned long long R, int t,
                          uint8_t* c) {
    for (int i = t; i >= 1; --i) {
        int lo = i - 1, hi = n;  // C(lo, i) <= R < C(hi, i)
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (B[mid * stride + i] <= R) lo = mid;
            else hi = mid;
        }
        c[i - 1] = (uint8_t)lo;
        R -= B[lo * stride + i];
        n = lo;
    }
}

// Successor of a subset whose lowest element has reached c[1] - 1 (t >= 2):
// the smallest j >= 1 with c[j] + 1 below the next element (n past the last)
// moves up by one and c[0..j-1] restart at 0..j-1.  Returns j, or -1 after
// the last subset.
DIST_CX int colex_carry(uint8_t* c, int t, int n) {
    int j = 1;
    while (j < t && c[j] + 1 >= (j + 1 < t ? (int)c[j + 1] : n)) j++;
    if (j >= t) return -1;
    c[j]++;
    for (int i = 0; i < j; i++) c[i] = (uint8_t)i;
    return j;
}

}  // namespace dist
