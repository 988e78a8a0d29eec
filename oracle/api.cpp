// C entry points of the oracle library (test infrastructure; see oracle.h).
// Multi-chain runs are Alg. 1 executed independently per chain, spread over
// host threads; every chain is sequential and deterministic.
#include "oracle.h"
#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

using namespace ora;

extern "C" {

void ora_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  Block b = philox(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1]);
  for (int i = 0; i < 4; ++i) out[i] = b.w[i];
}

double ora_uniform(uint32_t hi, uint32_t lo) { return uniform(hi, lo); }
double ora_uniform32(uint32_t w) { return uniform32(w); }

void ora_normals(uint64_t seed, uint32_t chain, uint32_t sample, uint32_t tag, uint32_t draw0,
                 int d, double* z) {
  Stream s{seed, chain, sample};
  normals(s, tag, draw0, d, z);
}

double ora_logp(int kind, int d, int n_data, const double* params, const double* x, double* grad) {
  Target t{kind, d, n_data, params};
  return t.logp(x, grad);
}

void ora_leapfrog(int kind, int d, int n_data, const double* params, double* x, double* p,
                  double eps, int n_steps) {
  Target t{kind, d, n_data, params};
  std::vector<double> g(d);
  double lp = t.logp(x, g.data());
  for (int i = 0; i < n_steps; ++i) leapfrog(t, x, p, g.data(), &lp, eps);
}

double ora_log1mexp(double a) { return log1mexp(a); }
double ora_dr_log_alpha1(double a, double b) { return dr_log_alpha1(a, b); }
double ora_dr_log_alpha2(double a, double b, double c, double q1, double q2) {
  return dr_log_alpha2(a, b, c, q1, q2);
}
double ora_dr_log_alpha3(double lp0, double lp1, double lp2, double lp3, double q1xy1,
                         double q2xy2, double q1y3y2, double q2y3y1, double q1y1y2) {
  return dr_log_alpha3(lp0, lp1, lp2, lp3, q1xy1, q2xy2, q1y3y2, q2y3y1, q1y1y2);
}

double ora_dr_stage_log_alpha(int k, int d, const double* x, const double* ys, const double* lps,
                              const double* sig) {
  return dr_stage_log_alpha(k, d, x, ys, lps, sig);
}

double ora_sdr_log_alpha(double lp_x, double lp_star, double lp_y) { return sdr_log_alpha(lp_x, lp_star, lp_y); }

// One ESS transition with its bracket recorded after every shrink.
int ora_ess_trace(int kind, int d, int n_data, const double* params, double* x, uint64_t seed,
                  uint32_t chain, uint32_t sample, double* trace, int trace_cap) {
  Target t{kind, d, n_data, params};
  double ell = t.logp(x, nullptr);
  Stream s{seed, chain, sample};
  return ess_transition(t, s, x, &ell, trace, trace_cap);
}

// Run n_samples transitions of `algo` (0 ESS, 1 DR, 2 NUTS, 3 symmetric DR) on chains
// chain0 .. chain0+n_chains-1, starting from x0[n_chains][d].
//   samples [n_chains][n_samples][d]  (nullable)
//   counts  [n_chains][n_samples]     loop-body count N_ij (nullable)
//   aux     [n_chains][n_samples]     NUTS tree depth (nullable)
//   x_final [n_chains][d]             (nullable)
// algo_params: DR {n_stages, scale0, factor}; NUTS {eps, max_depth, max_dH}; symmetric DR
// {n_stages = M, scale0 = sigma}; ESS unused.
// Returns 0, or -1 for an invalid argument.
// Sampler settings from the algo_params array (nullptr: defaults); false when invalid.
static bool sampler_params(int algo, const double* algo_params, DRParams* dp, NUTSParams* np) {
  *dp = DRParams{3, 1.0, 0.5};
  *np = NUTSParams{0.05, 10, 1000.0};
  if (algo == 1 && algo_params) *dp = DRParams{(int)algo_params[0], algo_params[1], algo_params[2]};
  if (algo == 2 && algo_params) *np = NUTSParams{algo_params[0], (int)algo_params[1], algo_params[2]};
  if (algo == 3) *dp = algo_params ? DRParams{(int)algo_params[0], algo_params[1], 1.0} : DRParams{100, 0.1, 1.0};
  if (algo == 1 && (dp->n_stages < 1 || dp->n_stages > 3)) return false;
  if (algo == 3 && (dp->n_stages < 1 || dp->n_stages > 1000 || !(dp->scale0 > 0))) return false;
  return true;
}

static bool slice_params(int algo, const double* algo_params, SliceParams* sp) {
  *sp = SliceParams{1.0, 100};
  if (algo == 4 && algo_params) *sp = SliceParams{algo_params[0], (int)algo_params[1]};
  return algo != 4 || (sp->w > 0 && sp->m >= 1 && sp->m <= 1000000);
}

// One transition of `algo` for sample index `sample` of chain `chain` (Alg. 1's loop body).
static int transition(int algo, const Target& t, const DRParams& dp, const NUTSParams& np,
                      const SliceParams& sp, uint64_t seed, uint32_t chain, uint32_t sample, double* x,
                      double* lp, double* g, int* depth) {
  Stream s{seed, chain, sample};
  *depth = 0;
  if (algo == 0) return ess_transition(t, s, x, lp, nullptr, 0);
  if (algo == 4) return slice_transition(t, s, sp, x, lp, depth);
  if (algo == 1) return dr_transition(t, s, dp, x, lp);
  if (algo == 3) return sdr_transition(t, s, dp, x, lp);
  return nuts_transition(t, s, np, x, lp, g, depth);
}

}  // extern "C"

template <typename F>
static void parallel_for(int64_t n, int n_threads, F work) {
  int nt = std::max(1, std::min<int>(n_threads, (int)std::max<int64_t>(1, n)));
  if (nt == 1) {
    work(0, n);
    return;
  }
  std::vector<std::thread> pool;
  for (int k = 0; k < nt; ++k) pool.emplace_back(work, n * k / nt, n * (k + 1) / nt);
  for (auto& th : pool) th.join();
}

extern "C" {

int ora_run(int algo, int kind, int d, int n_data, const double* params, const double* algo_params,
            int64_t chain0, int64_t n_chains, int64_t n_samples, const double* x0, uint64_t seed,
            int n_threads, double* samples, int32_t* counts, int32_t* aux, double* x_final) {
  if (d <= 0 || n_chains < 0 || n_samples < 0 || algo < 0 || algo > 4) return -1;
  Target t{kind, d, n_data, params};
  if (algo == 0 && t.prior_chol() == nullptr) return -1;
  DRParams dp;
  NUTSParams np;
  SliceParams sp;
  if (!sampler_params(algo, algo_params, &dp, &np) || !slice_params(algo, algo_params, &sp)) return -1;
  parallel_for(n_chains, n_threads, [&](int64_t c_begin, int64_t c_end) {
    std::vector<double> x(d), g(d);
    for (int64_t c = c_begin; c < c_end; ++c) {
      std::copy(x0 + c * d, x0 + (c + 1) * d, x.begin());
      double lp = t.logp(x.data(), algo == 2 ? g.data() : nullptr);
      for (int64_t i = 0; i < n_samples; ++i) {
        int depth = 0;
        const int n = transition(algo, t, dp, np, sp, seed, (uint32_t)(chain0 + c), (uint32_t)i, x.data(), &lp,
                                 g.data(), &depth);
        if (samples) std::copy(x.begin(), x.end(), samples + (c * n_samples + i) * d);
        if (counts) counts[c * n_samples + i] = n;
        if (aux) aux[c * n_samples + i] = depth;
      }
      if (x_final) std::copy(x.begin(), x.end(), x_final + c * d);
    }
  });
  return 0;
}

// Independent single transitions: item i starts at x_in[i] as sample sample[i] of chain chain[i]
// (the same random numbers as in a run) and writes the state it moves to.
// margin (nullable) [n_items]: the smallest decision margin of each transition (oracle.h).
int ora_transitions(int algo, int kind, int d, int n_data, const double* params, const double* algo_params,
                    int64_t n_items, const uint32_t* chain, const uint32_t* sample, const double* x_in,
                    uint64_t seed, int n_threads, double* x_out, int32_t* counts, int32_t* aux,
                    double* margin) {
  if (d <= 0 || n_items < 0 || algo < 0 || algo > 4) return -1;
  Target t{kind, d, n_data, params};
  if (algo == 0 && t.prior_chol() == nullptr) return -1;
  DRParams dp;
  NUTSParams np;
  SliceParams sp;
  if (!sampler_params(algo, algo_params, &dp, &np) || !slice_params(algo, algo_params, &sp)) return -1;
  parallel_for(n_items, n_threads, [&](int64_t b, int64_t e) {
    std::vector<double> x(d), g(d);
    for (int64_t i = b; i < e; ++i) {
      std::copy(x_in + i * d, x_in + (i + 1) * d, x.begin());
      double lp = t.logp(x.data(), algo == 2 ? g.data() : nullptr);
      int depth = 0;
      margin_reset();
      const int n = transition(algo, t, dp, np, sp, seed, chain[i], sample[i], x.data(), &lp, g.data(), &depth);
      std::copy(x.begin(), x.end(), x_out + i * d);
      counts[i] = n;
      aux[i] = depth;
      if (margin) margin[i] = margin_min();
    }
  });
  return 0;
}

// R(m) estimate from recorded loop counts: mean_i max_j N_ij / mean_ij N_ij (Sec. 4.2).
double ora_R_hat(const int32_t* counts, int64_t m, int64_t n) {
  double sum_max = 0, sum_all = 0;
  for (int64_t i = 0; i < n; ++i) {
    int32_t mx = 0;
    for (int64_t j = 0; j < m; ++j) {
      int32_t v = counts[j * n + i];
      mx = std::max(mx, v);
      sum_all += v;
    }
    sum_max += mx;
  }
  if (sum_all == 0) return 1.0;
  return (sum_max / (double)n) / (sum_all / (double)(n * m));
}

}  // extern "C"
