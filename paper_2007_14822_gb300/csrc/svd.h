// Truncated SVD internals shared with the sweep driver.
#pragma once

#include "tnh_internal.h"

namespace tnh {

struct SvdResult;
struct SvdShape {
    std::vector<std::vector<int>> qn;   // charges of the kept link sectors (ascending)
    std::vector<int> dims;              // kept dimension of each sector
    double truncerr = 0.0;
};
// exact_side 0: U comes out orthonormal to float64 accuracy (a left-to-right
// move), 1: V does (right-to-left); the other factor carries S or not per
// the absorb argument of svd_fetch.
SvdResult* svd_run(Ctx* ctx, const Layout& T, int nrow, double cutoff, int maxdim, int mindim, int exact_side);
SvdShape svd_shape(const SvdResult* R);
// absorb: 0 none, 1 multiply S into U, 2 multiply S into V
void svd_fetch(SvdResult* R, const Layout& U, double* S, const Layout& V, int absorb);
void svd_delete(SvdResult* R);

}  // namespace tnh
