// Device-side building blocks shared by the cascade kernels.
//
// Error-free transformations (Knuth's TwoSum, Dekker's FastTwoSum) and the
// FP64x2 additions used to add across bins (Sec. "Cascading vectors and dot
// products": bins 0-2 are added in FP64x2 or with quick-two-sum) and to
// accumulate rank-K_C updates into C (Sec. "Simple").  Every operation is an
// explicit round-to-nearest intrinsic, so the compiler can neither contract
// nor reassociate anything here.
#pragma once
#include <cstdint>

#include "ddgemm_internal.h"

namespace ddg {

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = __dadd_rn(a, b);
    double bv = __dsub_rn(s, a);
    double av = __dsub_rn(s, bv);
    e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}

// Requires |a| >= |b| (or a == 0).
__device__ __forceinline__ void fast_two_sum(double a, double b, double &s, double &e) {
    s = __dadd_rn(a, b);
    e = __dsub_rn(b, __dsub_rn(s, a));
}

// (h, l) += b for an FP64 b.
__device__ __forceinline__ void dd_add_d(double &h, double &l, double b) {
    double s, e;
    two_sum(h, b, s, e);
    e = __dadd_rn(e, l);
    fast_two_sum(s, e, h, l);
}

// (ah, al) + (bh, bl): two TwoSums and two renormalisations.
__device__ __forceinline__ void dd_add(double ah, double al, double bh, double bl,
                                       double &rh, double &rl) {
    double s, e, t, f;
    two_sum(ah, bh, s, e);
    two_sum(al, bl, t, f);
    e = __dadd_rn(e, t);
    fast_two_sum(s, e, s, e);
    e = __dadd_rn(e, f);
    fast_two_sum(s, e, rh, rl);
}

// Sum across bins for one k-block, from the likely lowest-order bin up
// (Sec. "Simple"): bin 3-6, bin 2, bin 1, bin 0.
__device__ __forceinline__ void assemble_bins(double b0, double b1, double b2, double b36,
                                              double &h, double &l) {
    two_sum(b2, b36, h, l);
    dd_add_d(h, l, b1);
    dd_add_d(h, l, b0);
}

// Tile order for L2 reuse: consecutive CTAs walk down `group` row tiles of
// one column, then the next column, so a wave of CTAs shares a few row
// panels of A and a few column panels of B.  bid in [0, tiles_m * tiles_n).
__device__ __forceinline__ void grouped_tile(unsigned bid, int tiles_m, int tiles_n, int group,
                                             int &tm, int &tn) {
    const unsigned per_group = (unsigned)group * (unsigned)tiles_n;
    const int g = (int)(bid / per_group);
    const int first = g * group;
    const int rows = min(group, tiles_m - first);
    const unsigned r = bid % per_group;
    tm = first + (int)(r % (unsigned)rows);
    tn = (int)(r / (unsigned)rows);
}

}  // namespace ddg
