// Environment-update plan (three labelled contractions).
#pragma once

#include "tnh_internal.h"

namespace tnh {

struct EnvPlan {
    int dir = 1;
    double flops = 0.0;
    std::unique_ptr<ContractPlan> c1, c2, c3;
    DevBuf x, y;
    Workspace ws;
    ~EnvPlan();
};

std::unique_ptr<EnvPlan> make_env(Ctx* ctx, int dir, const Layout& E, const Layout& A, const Layout& W,
                                  const Layout& out);
void run_env(Ctx* ctx, EnvPlan& P, const double* E, const double* A, const double* W, double* out,
             tnh_precision prec);

}  // namespace tnh
