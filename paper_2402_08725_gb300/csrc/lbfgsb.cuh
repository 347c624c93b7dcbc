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

// Independent problems on disjoint segments [off[f], off[f] + len[f]) of one packed vector (every
// index in one segment), each with its lower-bounded ranges (global indices) and their bounds;
// eval(x, g, losses_dev) evaluates every problem at once: the gradient into g and problem f's loss
// into losses_dev[f] (device).
struct LbfgsbFields {
    long long n = 0;
    std::vector<long long> off, len;
    std::vector<std::vector<std::pair<long long, long long>>> ranges;
    std::vector<std::vector<float>> lo;
    std::function<sr_status(const float *x, float *g, double *losses_dev)> eval;
};

// One L-BFGS-B run per problem, all advanced together: per iteration one direction for every
// active problem, then line-search rounds of one joint evaluation each until every problem has
// its step or has failed.  A problem's iterates do not depend on the others.  f_hist: NULL or
// [problems][max_iter + 1] (NaN past a problem's last iterate); info: NULL or one per problem;
// *rounds: joint evaluations after the first.
sr_status lbfgsb_fields_run(const LbfgsbFields &P, float *x, const sr_lbfgsb_cfg &cfg, double *f_hist,
                            sr_lbfgsb_info *info, int *rounds, cudaStream_t st);

// Minimise from x (device, n floats, overwritten with the last accepted iterate).
sr_status lbfgsb_run(const LbfgsbProblem &P, float *x, const sr_lbfgsb_cfg &cfg, double *f_hist,
                     sr_lbfgsb_info *info, cudaStream_t st);

}  // namespace sr
