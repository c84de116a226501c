// packed.cuh -- a small ascending set packed into one register (host and
// device): element p of a set of at most 8 values below 256 in bits
// 8p..8p+7 of a 64-bit word.  Reading or replacing an element is a shift,
// where an array indexed at run time would live in local memory on the
// device.
#pragma once
#include "dist_types.h"

namespace dist {

DIST_HD int pk_get(uint64_t S, int p) { return (int)((S >> (8 * p)) & 0xFFu); }

DIST_HD uint64_t pk_put(uint64_t S, int p, int v) {
    return (S & ~(0xFFull << (8 * p))) | ((uint64_t)(unsigned)v << (8 * p));
}

}  // namespace dist
