// L-BFGS-B driver (lbfgsb.cu), internal.
#pragma once

#include <functional>
#include <vector>

#include "common.cuh"

namespace sr {

constexpr int kLbfgsMaxMemory = 10;

// One bound-constrained problem: n variables, lower bounds on the variables of `ranges` ([begin,
// end) index pairs, disjoint; lo holds their bounds in the order of the ranges), no other bounds,
// and eval(x, g, &f) = the loss and its gradient at the device vector x.
struct LbfgsbProblem {
    long long n = 0;
    std::vector<std::pair<long long, long long>> ranges;
    std::vector<float> lo;
    std::function<sr_status(const float *x, float *g, double *f)> eval;
};

// Minimise from x (device, n floats, overwritten with the last accepted iterate).
sr_status lbfgsb_run(const LbfgsbProblem &P, float *x, const sr_lbfgsb_cfg &cfg, double *f_hist,
                     sr_lbfgsb_info *info, cudaStream_t st);

}  // namespace sr
