// iso.h -- the isometry method (Algorithm 3, Saved_isometry) on the GPU:
// host-side planning shared by iso.cpp and iso.cu.
//
// The map (a, b) -> (a, b, a + b) sends F2^{2n} into F2^{3n} and multiplies
// every symplectic weight by two (wt_H(iso(c)) = 2 wt_s(c)).  The image code
// is searched with the plain binary Brouwer-Zimmermann algorithm: systematic
// generator matrices Gamma_1..Gamma_m on disjoint information sets (the last
// ones may have deficient rank), every r-subset of every matrix's rows for
// r = 1, 2, ..., and the bound L = sum_j max(0, r + 1 - f_j).  d = U / 2 once
// L >= U.
#pragma once
#include <stdint.h>

#include <vector>

#include "plan.h"

namespace dist {

constexpr int kIsoMaxWords = (3 * DIST_MAXN + 31) / 32;  // a row of 3n bits

// One systematic matrix of the image code.
struct IsoGamma {
    int k = 0;                       // rank on the columns it could use
    int f = 0;                       // rows without a pivot: K - k
    int words = 0;                   // u32 words of the columns outside its information set
    std::vector<uint32_t> rows;      // [K][words]: each row on those columns, packed
    std::vector<uint8_t> piv;        // [K]: 1 if the row has a pivot (it adds 1 on the set)
    std::vector<Coef> coef;          // [K]: coefficients over the plan's basis
};

struct IsoPlan {
    int K = 0;                       // F2 rows of the code (an F4 input counts twice)
    int n3 = 0;                      // 3n
    int words = 0;                   // max words over the matrices
    std::vector<IsoGamma> G;
    int u0 = 0;                      // lightest row (Hamming weight of the image), any matrix
    int u0_g = -1, u0_row = -1;      // where it is
};

// Builds the matrices of the image of plan p's code (outside S in exclusion
// mode, the seed is the lightest row outside S).  P_EZERO if the code is 0.
int iso_build(const Plan& p, IsoPlan* ip);

// Lower bound on the Hamming weight of the image once matrices 0..jpos have
// finished round r and the others round r - 1 (DIST_WINF if a matrix has
// been enumerated completely).
int iso_lower_bound(const IsoPlan& ip, int r, int jpos);

// Witness of Hamming weight wH from `count` rows of matrix g: checks it and
// writes the codeword (weight wH / 2) and its input-row coefficients.
int iso_decode(const Plan& p, const IsoPlan& ip, int g, const uint8_t* rows, int count, int wH,
               uint8_t* witness, uint8_t* coeffs);

}  // namespace dist
