// Host-side rules of the job server (pp_server.cu): the cost model that
// orders queued jobs, the choice of the job to admit, and the share of the
// GPU a layer of a running job takes.  Plain C++ with no CUDA, so the same
// code is compiled into the library and into a CPU test driver.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <utility>
#include <vector>

#include "../../include/pp.h"

namespace ppadm {

// Features of a job for the cost model: 1, log layers, log gates per layer,
// log 1/eps (eps = 0 counts as 1e-12), per-gate or per-layer noise, noise x
// log 1/eps, log n, and whether a group merges the strings.
constexpr int kFeat = 8;
inline void job_features(const pp_config& cfg, int n_layers, int n_gates, double* f) {
  const double eps = cfg.coeff_eps > 1e-12 ? cfg.coeff_eps : 1e-12;
  const double le = std::log(1.0 / eps);
  const double noise = cfg.noise_mode != PP_NOISE_NONE ? 1.0 : 0.0;
  f[0] = 1.0;
  f[1] = std::log((double)std::max(n_layers, 1));
  f[2] = std::log((double)std::max(n_gates, 1));
  f[3] = le;
  f[4] = noise;
  f[5] = noise * le;
  f[6] = std::log((double)std::max(cfg.n_qubits, 1));
  f[7] = cfg.symmetry != PP_SYM_NONE ? 1.0 : 0.0;
}

// Prior coefficients: the fit of log(run ms) on the features over the first
// 300 jobs of the full-size serving stream run in arrival order.
constexpr double kPrior[kFeat] = {-7.845, 0.887, 1.444, 0.703, 0.519, -0.438, -1.080, -0.338};
constexpr double kRidge = 1.0;

// Predicted log run time of a job, learned from the jobs the server has
// finished: ridge regression of log(run ms) on the features, pulled towards
// the prior (minimises |F beta - y|^2 + kRidge |beta - kPrior|^2).  Refitted
// after every finished job (an 8 x 8 solve).
struct CostModel {
  double A[kFeat][kFeat] = {};  // sum of f f^T
  double b[kFeat] = {};         // sum of f y
  double beta[kFeat];
  int n_obs = 0;

  CostModel() { std::copy(kPrior, kPrior + kFeat, beta); }

  double predict(const double* f) const {
    double v = 0.0;
    for (int i = 0; i < kFeat; ++i) v += beta[i] * f[i];
    return v;
  }

  void add(const double* f, double y) {
    for (int i = 0; i < kFeat; ++i) {
      b[i] += f[i] * y;
      for (int k = 0; k < kFeat; ++k) A[i][k] += f[i] * f[k];
    }
    ++n_obs;
    // (A + kRidge I) beta = b + kRidge kPrior, by Gaussian elimination with
    // partial pivoting; the prior keeps the system well posed
    double M[kFeat][kFeat + 1];
    for (int i = 0; i < kFeat; ++i) {
      for (int k = 0; k < kFeat; ++k) M[i][k] = A[i][k] + (i == k ? kRidge : 0.0);
      M[i][kFeat] = b[i] + kRidge * kPrior[i];
    }
    for (int c = 0; c < kFeat; ++c) {
      int piv = c;
      for (int r = c + 1; r < kFeat; ++r)
        if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
      if (std::fabs(M[piv][c]) < 1e-12) return;  // keep the previous fit
      if (piv != c)
        for (int k = 0; k <= kFeat; ++k) std::swap(M[c][k], M[piv][k]);
      for (int r = 0; r < kFeat; ++r) {
        if (r == c) continue;
        const double m = M[r][c] / M[c][c];
        for (int k = c; k <= kFeat; ++k) M[r][k] -= m * M[c][k];
      }
    }
    for (int i = 0; i < kFeat; ++i) beta[i] = M[i][kFeat] / M[i][i];
  }
};

// A queued job passed this many times by jobs after it in admission order
// is passed no more.
constexpr int kMaxBypass = 8;
// A job's admission key drops by one (natural-log) unit for every this many
// seconds it has waited.
constexpr double kAgeSeconds = 10.0;

// Admission key: the predicted cost less the credit for the time waited; a
// job that gave its memory back goes to the head.
inline double admission_key(double predicted, double waited_s, bool gave_back) {
  return predicted - waited_s / kAgeSeconds + (gave_back ? -1e9 : 0.0);
}

// The queued job to admit: the first in order of increasing key whose
// reservation fits (fits[k]), unless a job before it in that order has been
// passed kMaxBypass times already.  Every job before the chosen one in that
// order counts one more bypass.  Returns the chosen index, or -1.
inline long pick_admission(const std::vector<double>& key, const std::vector<char>& fits,
                           std::vector<int>& bypassed) {
  std::vector<std::pair<double, size_t>> order;
  order.reserve(key.size());
  for (size_t k = 0; k < key.size(); ++k) order.emplace_back(key[k], k);
  std::sort(order.begin(), order.end());
  for (size_t r = 0; r < order.size(); ++r) {
    const size_t k = order[r].second;
    if (fits[k]) {
      for (size_t q = 0; q < r; ++q) bypassed[order[q].second]++;
      return (long)k;
    }
    if (bypassed[k] >= kMaxBypass) return -1;
  }
  return -1;
}

// The GPU's co-resident blocks, in share units handed to the layers of
// running jobs: a job's persistent layer launch holds its units while it
// runs, and the units held at any time add up to at most the whole GPU, so
// the cooperative launches of all jobs fit at once.
constexpr int kShareUnits = 1024;

// Units a layer takes when `units_free` are free: at least 1/slots of the
// GPU, up to an equal share among the `running` jobs, and no more than its
// launch would use (`wanted`, a fraction of the GPU).  0 means wait: less
// than 1/slots is free.
inline int share_units(int slots, int64_t running, double wanted, int units_free) {
  const int floor_units = std::max(1, kShareUnits / std::max(slots, 1));
  if (units_free < floor_units) return 0;
  const int fair = std::max(floor_units, kShareUnits / (int)std::max<int64_t>(1, running));
  const int want = std::max(floor_units, std::min(fair, (int)std::ceil(wanted * kShareUnits)));
  return std::min(want, units_free);
}

}  // namespace ppadm
