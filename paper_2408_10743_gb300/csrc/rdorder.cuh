// rdorder.cuh -- the revolving-door successor with its move, for the
// isometry kernel (host and device).
#pragma once
#include "dist_types.h"

namespace dist {

// Successor in revolving-door order (Knuth's Algorithm R, steps R3-R5) of
// the ascending t-subset s of {0..n-1} -- the order of rd_next in walk.cuh --
// also reporting the element that left (*out) and the one that entered
// (*in): consecutive subsets of the order differ by exactly one of each (the
// isometry kernel moves one row out of its running sum and one in).  The
// caller never steps past the last subset.
DIST_HD void rd_next_delta(uint8_t* s, int t, int n, int* out, int* in) {
#define DIST_CJ(j) ((j) <= t ? (int)s[(j)-1] : n)
    int j;
    if (t & 1) {
        if (s[0] + 1 < DIST_CJ(2)) {
            *out = s[0];
            *in = s[0] + 1;
            s[0]++;
            return;
        }
        j = 2;
        goto r4;
    } else {
        if (s[0] > 0) {
            *out = s[0];
            *in = s[0] - 1;
            s[0]--;
            return;
        }
        j = 2;
        goto r5;
    }
r4:
    if (j > t) return;
    if (DIST_CJ(j) >= j) {  // s[j-1] leaves, j - 2 enters below s[j-2]
        *out = s[j - 1];
        *in = j - 2;
        s[j - 1] = s[j - 2];
        s[j - 2] = (uint8_t)(j - 2);
        return;
    }
    j++;
r5:
    if (j > t) return;
    if (DIST_CJ(j) + 1 < DIST_CJ(j + 1)) {  // s[j-2] leaves, s[j-1] + 1 enters
        *out = s[j - 2];
        *in = s[j - 1] + 1;
        s[j - 2] = s[j - 1];
        s[j - 1]++;
        return;
    }
    j++;
    goto r4;
#undef DIST_CJ
}

}  // namespace dist
