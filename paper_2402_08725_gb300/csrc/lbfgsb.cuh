// L-BFGS-B driver (lbfgsb.cu), internal.
#pragma once

#include <functional>
#include <vector>

#include "common.cuh"

namespace sr {

constexpr int kLbfgsMaxMemory = 10;

// One bound-constrained problem: n variables, lower bounds lo[i - r0] on the range [r0, r1)
// (no other bounds), and eval(x, g, &f) = the loss and its gradient at the device vector x.
struct LbfgsbProblem {
    long long n = 0, r0 = 0, r1 = 0;
    std::vector<float> lo;
    std::function<sr_status(const float *x, float *g, double *f)> eval;
};

// Minimise from x (device, n floats, overwritten with the last accepted iterate).
sr_status lbfgsb_run(const LbfgsbProblem &P, float *x, const sr_lbfgsb_cfg &cfg, double *f_hist,
                     sr_lbfgsb_info *info, cudaStream_t st);

}  // namespace sr
