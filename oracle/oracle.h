// FP64 CPU oracle for multi-chain MCMC (arXiv 2503.17405) -- TEST INFRASTRUCTURE.
//
// This directory is a plain, slow, sequential reference implementation of the
// single-chain samplers the paper vectorises (Alg. 1 run once per chain).  Only
// the test suite, the smoke check and the benchmark's CPU-baseline leg may
// load it.  It shares no code with the CUDA path: its own counter-based RNG,
// its own targets, its own samplers.  Everything is double precision.
//
// Parity status per function (see the pins in tests/test_oracle_*.py):
//   philox            pinned: published known-answer vectors
//   ess               pinned: conjugate-Gaussian closed form, flat-likelihood
//                     special case, bracket invariant
//   dr (3 stages)     pinned: exact detailed balance on a discrete ring,
//                     funnel closed-form marginals
//   nuts              pinned: harmonic-oscillator leapfrog closed form,
//                     reversibility, Gaussian moments
//   nuts on logistic regression: no closed form; pinned by self-normalised
//                     importance sampling of the same posterior expectations
//   decision margins  pinned: a one-stage DR transition's margin rebuilt from the
//                     oracle's own random numbers and density
#pragma once
#include <cstdint>
#include <cstddef>

namespace ora {

// ---- counter-based RNG: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) --
struct Block { uint32_t w[4]; };
Block philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1);

// Keying used by every sampler: key = (chain, seed_lo), counter = (draw, sample, tag, seed_hi).
struct Stream {
  uint64_t seed;
  uint32_t chain;
  uint32_t sample;
  Block block(uint32_t tag, uint32_t draw) const {
    return philox(draw, sample, tag, (uint32_t)(seed >> 32), chain, (uint32_t)seed);
  }
};

// Uniform in (0,1) from two 32-bit words: ((hi:lo >> 12) + 1/2) * 2^-52.
double uniform(uint32_t hi, uint32_t lo);
// Uniform in (0,1) from one 32-bit word: (w + 1/2) * 2^-32.
double uniform32(uint32_t w);
// Four normals from one block: Box-Muller on (u32(w0), u32(w1)) and on (u32(w2), u32(w3)).
void normal_quad(const Block& b, double* z);
// z[0..d) from blocks draw0, draw0+1, ... of stream `tag` (normals 4q .. 4q+3 from block q).
void normals(const Stream& s, uint32_t tag, uint32_t draw0, int d, double* z);

// ---- targets ------------------------------------------------------------------
enum TargetKind {
  TGT_GAUSS_CONJ = 0,  // ESS likelihood  -|y-x|^2/(2 s2);           params: L[d*d], y[d], s2
  TGT_GP_LOGIT = 1,    // ESS likelihood  -sum softplus(-s_i x_i);   params: L[d*d], s[d]
  TGT_FUNNEL = 2,      // Neal funnel log-density (v, x_1..x_{d-1});  params: none
  TGT_LOGREG = 3,      // logistic-regression log-posterior;         params: X[n*d], y[n]
  TGT_GAUSS_DIAG = 4,  // N(mu, diag sigma^2) log-density;           params: mu[d], sigma[d]
  TGT_FLAT = 5,        // ESS likelihood f == 1;                      params: L[d*d]
  TGT_MOG = 6,         // mixture of K = n_data Gaussians N(mu_k, S), S = (1-rho) I + rho 1 1^T
                       // (unit variances, correlation rho), weights w_k;
                       //                                  params: rho, w[K], mu[K*d]
  TGT_GP_REG = 7,      // ESS likelihood of GP-regression hyperparameters x = (sigma, tau, lambda)
                       // (d = 3): log N(y; 0, tau^2 exp(-lambda^2 D) + sigma^2 I) over n = n_data
                       // points;                          params: L[3*3], D[n*n], y[n]
};

struct Target {
  int kind;
  int d;
  int n_data;
  const double* params;
  // log f (ESS likelihood) or log pi (DR / NUTS).  grad (optional) = d/dx.
  double logp(const double* x, double* grad) const;
  const double* prior_chol() const;  // ESS kinds: lower-triangular L with Sigma = L L^T
};

// ---- samplers (one chain, one transition each) ----------------------------------
// Elliptical slice sampling, Alg. 8.  x[d] in/out, *ell in/out caches log f(x).
// Returns the number of bracket shrinks N (the loop-body count of Alg. 8).
int ess_transition(const Target& t, const Stream& s, double* x, double* ell,
                   double* trace /* nullable: 3 doubles (theta, theta_min, theta_max) per shrink */,
                   int trace_cap);

// Delayed rejection, 3 stages, x-centred Gaussian proposals with scales
// scale0 * factor^k.  Returns the number of stages tried (1..n_stages).
struct DRParams { int n_stages; double scale0; double factor; };
int dr_transition(const Target& t, const Stream& s, const DRParams& p, double* x, double* lp);

// log acceptance probabilities of the general delayed-rejection scheme.
// Arguments are log target values and log proposal densities (see dr.cpp).
double dr_log_alpha1(double lp_cur, double lp_prop);
double dr_log_alpha2(double lp_cur, double lp_first, double lp_second,
                     double lq1_cur_first, double lq1_second_first);
double dr_log_alpha3(double lp0, double lp1, double lp2, double lp3,
                     double lq1_x_y1, double lq2_x_y2,
                     double lq1_y3_y2, double lq2_y3_y1, double lq1_y1_y2);
double log1mexp(double a);
double dr_stage_log_alpha(int k, int d, const double* x, const double* ys, const double* lps,
                          const double* sig);

// Symmetric delayed rejection (Mira 2001; Sec. 7.1's toy experiment): every try re-centres a
// symmetric proposal y_k ~ N(y_{k-1}, sigma^2 I) (y_0 = x) on the last rejected point, at most
// M = n_stages tries, constant sigma = scale0.  Returns the number of tries (1..M).
int sdr_transition(const Target& t, const Stream& s, const DRParams& p, double* x, double* lp);
// log alpha_k = min(0, log [(pi(y_k) - pi*)+ / (pi(x) - pi*)]), pi* = max over rejected tries
double sdr_log_alpha(double lp_x, double lp_star, double lp_y);

// Slice sampling (Neal 2003) along a random direction: stepping-out with the expansion limit m
// split into J = floor(m V) left and K = m - 1 - J right steps of width w, then shrinkage
// (Fig. 2's slice sampler: an expansion loop followed by a shrink loop).  x[d] in/out, *lp in/out
// caches log pi(x).  Returns the number of log-density evaluations N (expansion checks plus
// proposals); *n_prop receives the number of proposals (>= 1).
struct SliceParams { double w; int m; };
int slice_transition(const Target& t, const Stream& s, const SliceParams& p, double* x, double* lp,
                     int* n_prop);

// Multinomial NUTS with momentum-sum U-turn criterion.  x[d] in/out,
// *lp in/out caches log pi(x), grad[d] in/out caches its gradient.
// Returns the number of leapfrog steps; *depth receives the number of doublings.
struct NUTSParams { double eps; int max_depth; double max_dH; };
int nuts_transition(const Target& t, const Stream& s, const NUTSParams& p, double* x,
                    double* lp, double* grad, int* depth);
void leapfrog(const Target& t, double* x, double* p, double* grad, double* lp, double eps);

// ---- decision margins (instrumentation for single-precision comparisons) -----------
// Every accept/reject, shrink/stop, merge and U-turn decision of a transition compares a
// computed value with its threshold.  The samplers record, per thread, the smallest margin
// they met: |a - b| / max(1, |b|) for a value a tested against a threshold b (log densities
// against log y, log u against log alpha, H - H0 against the divergence bound), and
// |rho . p| / (|rho| |p|) for a U-turn test.  A transition whose smallest margin lies within
// the rounding error of single precision can take the other branch there; the values of the
// transition do not depend on this bookkeeping.
void margin_reset();
double margin_min();

}  // namespace ora
