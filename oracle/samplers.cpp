// Oracle samplers: ESS (Alg. 8), 3-stage delayed rejection, multinomial NUTS.
// Test infrastructure; see oracle.h.  Plain sequential double-precision code.
#include "oracle.h"
#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

namespace ora {

static const double kPi = 3.14159265358979323846;
static const double kNegInf = -std::numeric_limits<double>::infinity();
static const int kMaxShrinks = 10000;  // safety cap; never reached in double precision

static int normal_blocks(int d) { return (d + 3) / 4; }  // four normals per Philox block

// smallest decision margin of the current transition on this thread (see oracle.h)
static thread_local double t_margin = std::numeric_limits<double>::infinity();
void margin_reset() { t_margin = std::numeric_limits<double>::infinity(); }
double margin_min() { return t_margin; }
static void note(double a, double b) {
  const double m = std::fabs(a - b) / std::max(1.0, std::fabs(b));
  if (m < t_margin) t_margin = m;  // NaN margins (non-finite values) are not recorded
}
static void note_cos(double dt, double nr, double np) {
  const double den = std::sqrt(nr) * std::sqrt(np);
  if (den > 0) {
    const double m = std::fabs(dt) / den;
    if (m < t_margin) t_margin = m;
  }
}

// ------------------------------------------------------------------------------------
// Elliptical slice sampling (appendix Alg. 8), with these readings:
//  * the loop continues while the proposal is NOT above the threshold (the printed
//    loop condition is inverted; the text of Sec. 2.2 says "until it exceeds");
//  * "log p" is the log-likelihood f, the Gaussian prior being carried by nu;
//  * acceptance is strict (>), ties shrink;
//  * N counts bracket shrinks (the paper's "sub-iterations"), so N can be 0.
// Random numbers for sample i of a chain (tag 0):
//   draws 0..D-1       : z for nu = L z   (D = ceil(d/4), four normals per draw)
//   draw D, words 0-1  : u for the threshold log y = log f(x) + log u
//   draw D, words 2-3  : u' for the initial angle theta = 2 pi u'
//   draw D+1+s         : u_s for the s-th shrink, theta ~ U[theta_min, theta_max]
int ess_transition(const Target& t, const Stream& s, double* x, double* ell,
                   double* trace, int trace_cap) {
  const int d = t.d;
  const int D = normal_blocks(d);
  const double* L = t.prior_chol();
  std::vector<double> z(d), nu(d, 0.0), xp(d);

  // Choose ellipse nu ~ N(0, Sigma) with Sigma = L L^T.
  normals(s, 0, 0, d, z.data());
  for (int r = 0; r < d; ++r) {
    double acc = 0;
    for (int c = 0; c <= r; ++c) acc += L[(size_t)r * d + c] * z[c];
    nu[r] = acc;
  }
  // Threshold and initial bracket.
  Block b = s.block(0, (uint32_t)D);
  double log_y = *ell + std::log(uniform(b.w[0], b.w[1]));
  double theta = 2.0 * kPi * uniform(b.w[2], b.w[3]);
  double theta_min = theta - 2.0 * kPi;
  double theta_max = theta;

  auto propose = [&](double th) {
    double c = std::cos(th), sn = std::sin(th);
    for (int k = 0; k < d; ++k) xp[k] = x[k] * c + nu[k] * sn;
    return t.logp(xp.data(), nullptr);
  };
  double ellp = propose(theta);
  int n = 0;
  note(ellp, log_y);
  while (!(ellp > log_y)) {
    if (n == kMaxShrinks) return n;  // keep x (never happens in double precision)
    if (theta < 0) theta_min = theta; else theta_max = theta;
    Block bs = s.block(0, (uint32_t)(D + 1 + n));
    theta = theta_min + (theta_max - theta_min) * uniform(bs.w[0], bs.w[1]);
    if (trace && n < trace_cap) {
      trace[3 * n] = theta; trace[3 * n + 1] = theta_min; trace[3 * n + 2] = theta_max;
    }
    ellp = propose(theta);
    note(ellp, log_y);
    ++n;
  }
  for (int k = 0; k < d; ++k) x[k] = xp[k];
  *ell = ellp;
  return n;
}

// ------------------------------------------------------------------------------------
// Delayed rejection (Tierney & Mira) with proposals centred at the current point:
// stage k (k = 1, 2, 3) proposes y_k ~ N(x, sigma_k^2 I), sigma_k = scale0 * factor^(k-1).
// A stage is tried only after every earlier stage rejected.  All quantities are in
// log space; lq_k(a -> b) is the log stage-k proposal density up to a constant that
// cancels (numerator and denominator always carry the same set of stages).

// log(1 - e^a) for a < 0, -inf for a >= 0.
double log1mexp(double a) {
  if (!(a < 0)) return kNegInf;
  return a > -0.6931471805599453 ? std::log(-std::expm1(a)) : std::log1p(-std::exp(a));
}

// alpha_1(cur -> prop) = min(1, pi(prop) / pi(cur)); a proposal of zero density is never
// accepted, also from a current state of zero density (where the ratio would be 0 / 0)
double dr_log_alpha1(double lp_cur, double lp_prop) {
  if (lp_prop == kNegInf) return kNegInf;
  return std::min(0.0, lp_prop - lp_cur);
}

// alpha_2(cur, first, second): second-stage acceptance after `first` was rejected.
//   min(1, pi(second) q1(second->first) (1 - alpha_1(second->first))
//        / [pi(cur) q1(cur->first) (1 - alpha_1(cur->first))])
// The stage-2 proposal densities cancel because they are centred at the current
// point and symmetric in their two arguments.
double dr_log_alpha2(double lp_cur, double lp_first, double lp_second,
                     double lq1_cur_first, double lq1_second_first) {
  double num = lp_second + lq1_second_first + log1mexp(dr_log_alpha1(lp_second, lp_first));
  double den = lp_cur + lq1_cur_first + log1mexp(dr_log_alpha1(lp_cur, lp_first));
  if (num == kNegInf || den == kNegInf) return kNegInf;
  return std::min(0.0, num - den);
}

// alpha_3(x, y1, y2, y3): third-stage acceptance after y1 and y2 were rejected.
//   numerator:   pi(y3) q1(y3->y2) q2(y3->y1) (1 - alpha_1(y3->y2)) (1 - alpha_2(y3, y2, y1))
//   denominator: pi(x)  q1(x->y1)  q2(x->y2)  (1 - alpha_1(x->y1))  (1 - alpha_2(x, y1, y2))
double dr_log_alpha3(double lp0, double lp1, double lp2, double lp3,
                     double lq1_x_y1, double lq2_x_y2,
                     double lq1_y3_y2, double lq2_y3_y1, double lq1_y1_y2) {
  double num = lp3 + lq1_y3_y2 + lq2_y3_y1 + log1mexp(dr_log_alpha1(lp3, lp2)) +
               log1mexp(dr_log_alpha2(lp3, lp2, lp1, lq1_y3_y2, lq1_y1_y2));
  double den = lp0 + lq1_x_y1 + lq2_x_y2 + log1mexp(dr_log_alpha1(lp0, lp1)) +
               log1mexp(dr_log_alpha2(lp0, lp1, lp2, lq1_x_y1, lq1_y1_y2));
  if (num == kNegInf || den == kNegInf) return kNegInf;
  return std::min(0.0, num - den);
}

// log alpha of stage k (0-based) for proposals ys[0..k] (each d values) made from x:
// wires each stage's target values and proposal densities into the acceptance
// functions above.  lps = {log pi(x), log pi(y_1), ..., log pi(y_{k+1})}, sig = stage scales.
double dr_stage_log_alpha(int k, int d, const double* x, const double* ys, const double* lps,
                          const double* sig) {
  // log N(b | a, sigma_s^2 I) up to a constant shared by every call with the same stage s
  auto lq = [&](int st, const double* a, const double* b) {
    double acc = 0;
    for (int c = 0; c < d; ++c) { double r = b[c] - a[c]; acc += r * r; }
    return -acc / (2.0 * sig[st] * sig[st]);
  };
  const double* y1 = ys;
  const double* y2 = ys + d;
  const double* y3 = ys + 2 * d;
  if (k == 0) return dr_log_alpha1(lps[0], lps[1]);
  if (k == 1) return dr_log_alpha2(lps[0], lps[1], lps[2], lq(0, x, y1), lq(0, y2, y1));
  if (k == 2)
    return dr_log_alpha3(lps[0], lps[1], lps[2], lps[3], lq(0, x, y1), lq(1, x, y2),
                         lq(0, y3, y2), lq(1, y3, y1), lq(0, y1, y2));
  return kNegInf;  // more than three stages is not implemented
}

// Random numbers for sample i (tag 0): stage k (0-based) takes its normals from
// draws k(D+1) .. k(D+1)+D-1 and its acceptance uniform from words 0-1 of draw k(D+1)+D.
int dr_transition(const Target& t, const Stream& s, const DRParams& P, double* x, double* lp) {
  const int d = t.d;
  const int D = normal_blocks(d);
  const int K = P.n_stages;
  std::vector<double> ys((size_t)K * d), lps(K + 1), sig(K), eps(d);
  for (int k = 0; k < K; ++k) sig[k] = P.scale0 * std::pow(P.factor, (double)k);
  lps[0] = *lp;
  for (int k = 0; k < K; ++k) {
    const uint32_t base = (uint32_t)(k * (D + 1));
    double* yk = ys.data() + (size_t)k * d;
    normals(s, 0, base, d, eps.data());
    for (int c = 0; c < d; ++c) yk[c] = x[c] + sig[k] * eps[c];
    lps[k + 1] = t.logp(yk, nullptr);
    double la = dr_stage_log_alpha(k, d, x, ys.data(), lps.data(), sig.data());
    Block b = s.block(0, base + (uint32_t)D);
    note(std::log(uniform(b.w[0], b.w[1])), la);
    if (std::log(uniform(b.w[0], b.w[1])) < la) {
      for (int c = 0; c < d; ++c) x[c] = yk[c];
      *lp = lps[k + 1];
      return k + 1;
    }
  }
  return K;
}

// Symmetric delayed rejection with re-centred proposals (Mira 2001), the sampler of the paper's
// Sec. 7.1 toy experiment.  A try's proposal density is symmetric and depends only on the last
// rejected point, so the forward path x -> y_1 -> .. -> y_k and its reverse have the same
// proposal density, and the rejection factors telescope: pi(x) prod_{j<k} (1 - alpha_j) =
// pi(x) - pi*, pi* the largest target value among the rejected tries.  Hence
//   alpha_k = min(1, (pi(y_k) - pi*)+ / (pi(x) - pi*)),
// written here in log space.  Random numbers as for dr_transition: try k (0-based) takes its
// normals from draws k(D+1) .. k(D+1)+D-1 and its uniform from words 0-1 of draw k(D+1)+D.
double sdr_log_alpha(double lp_x, double lp_star, double lp_y) {
  if (!(lp_y > lp_star)) return kNegInf;                      // pi(y) <= pi*: never accepted
  const double num = lp_y + log1mexp(lp_star - lp_y);         // log (pi(y) - pi*)
  const double den = lp_x + log1mexp(lp_star - lp_x);         // log (pi(x) - pi*)
  if (den == kNegInf) return 0.0;
  return std::min(0.0, num - den);
}

// ------------------------------------------------------------------------------------
// Slice sampling (Neal 2003, stepping-out and shrinkage procedures) on the line through x with
// a random direction u (hit-and-run; for d = 1, u = +-1), with these readings:
//  * "inside the slice" is log pi > log y (strict), as for ESS; an end or a proposal exactly on
//    the threshold counts as outside;
//  * the stepping-out loop is Neal's with the limit m: J = floor(m V') steps at most to the
//    left, K = m - 1 - J to the right, the left end expanded before the right one;
//  * N counts log-density evaluations: an end is evaluated only while its step budget is
//    positive, and every proposal is one evaluation.
// Random numbers for sample i (tag 0):
//   draws 0..D-1       : z, u = z / |z|
//   draw D, words 0-1  : U for the threshold log y = log pi(x) + log U
//   draw D, words 2-3  : V for the initial interval L = -w V, R = L + w (in units along u)
//   draw D+1, words 0-1: V' for the limit split J = floor(m V'), K = m - 1 - J
//   draw D+2+s         : U_s for proposal s, theta = L + (R - L) U_s
int slice_transition(const Target& t, const Stream& s, const SliceParams& P, double* x, double* lp,
                     int* n_prop) {
  const int d = t.d;
  const int D = normal_blocks(d);
  std::vector<double> u(d), xp(d);
  normals(s, 0, 0, d, u.data());
  double nrm = 0;
  for (int k = 0; k < d; ++k) nrm += u[k] * u[k];
  nrm = std::sqrt(nrm);
  for (int k = 0; k < d; ++k) u[k] /= nrm;
  auto at = [&](double th) {
    for (int k = 0; k < d; ++k) xp[k] = x[k] + th * u[k];
    return t.logp(xp.data(), nullptr);
  };
  const Block b = s.block(0, (uint32_t)D);
  const double log_y = *lp + std::log(uniform(b.w[0], b.w[1]));
  double L = -P.w * uniform(b.w[2], b.w[3]);
  double R = L + P.w;
  const Block bj = s.block(0, (uint32_t)(D + 1));
  int J = (int)std::floor(P.m * uniform(bj.w[0], bj.w[1]));
  int K = (P.m - 1) - J;
  int n = 0;
  // stepping out
  while (J > 0) {
    ++n;
    const double lpl = at(L);
    note(lpl, log_y);
    if (!(lpl > log_y)) break;
    L -= P.w;
    --J;
  }
  while (K > 0) {
    ++n;
    const double lpr = at(R);
    note(lpr, log_y);
    if (!(lpr > log_y)) break;
    R += P.w;
    --K;
  }
  // shrinkage
  for (int p = 0; p < kMaxShrinks; ++p) {
    const Block bs = s.block(0, (uint32_t)(D + 2 + p));
    const double th = L + (R - L) * uniform(bs.w[0], bs.w[1]);
    const double lpp = at(th);
    ++n;
    note(lpp, log_y);
    if (lpp > log_y) {
      std::copy(xp.begin(), xp.end(), x);
      *lp = lpp;
      *n_prop = p + 1;
      return n;
    }
    if (th < 0) L = th; else R = th;
  }
  *n_prop = kMaxShrinks;  // keep x (never happens in double precision)
  return n;
}

int sdr_transition(const Target& t, const Stream& s, const DRParams& P, double* x, double* lp) {
  const int d = t.d;
  const int D = normal_blocks(d);
  std::vector<double> centre(x, x + d), y(d), eps(d);
  double lp_star = kNegInf;
  for (int k = 0; k < P.n_stages; ++k) {
    const uint32_t base = (uint32_t)(k * (D + 1));
    normals(s, 0, base, d, eps.data());
    for (int c = 0; c < d; ++c) y[c] = centre[c] + P.scale0 * eps[c];
    const double lp_y = t.logp(y.data(), nullptr);
    const double la = sdr_log_alpha(*lp, lp_star, lp_y);
    Block b = s.block(0, base + (uint32_t)D);
    note(std::log(uniform(b.w[0], b.w[1])), la);
    note(lp_y, lp_star);
    if (std::log(uniform(b.w[0], b.w[1])) < la) {
      std::copy(y.begin(), y.end(), x);
      *lp = lp_y;
      return k + 1;
    }
    lp_star = std::max(lp_star, lp_y);
    centre = y;
  }
  return P.n_stages;
}

// ------------------------------------------------------------------------------------
// NUTS (Hoffman & Gelman) in its multinomial form, built recursively.
//  * momentum p ~ N(0, I) (identity mass), H = -log pi(x) + |p|^2 / 2;
//  * doubling j (j = 0 .. max_depth-1) picks a direction and builds 2^j leapfrog steps;
//  * inside a subtree the two halves merge with the right half's proposal chosen with
//    probability W_R / (W_L + W_R), W = sum of exp(-H) over the half;
//  * a (sub)trajectory U-turns when rho . p_first <= 0 or rho . p_last <= 0, where rho is
//    the sum of its momenta; a leaf diverges when H - H0 > max_dH (or H is NaN);
//  * a subtree that U-turns or diverges is discarded and ends the transition;
//  * a valid subtree's proposal replaces the current one with probability
//    min(1, W_subtree / W_old) (biased progressive sampling).
// Random numbers for sample i:
//   tag 0, draws 0..D-1 : momentum
//   tag 1, draw j       : words 0-1 direction (u < 1/2 -> backwards), words 2-3 the
//                         progressive-sampling uniform of doubling j
//   tag 2, draw (j << 16) | (b << 4) | l : the merge at level l of block b (leaves
//                         b 2^l .. (b+1) 2^l - 1 of subtree j)
void leapfrog(const Target& t, double* x, double* p, double* grad, double* lp, double eps) {
  const int d = t.d;
  for (int k = 0; k < d; ++k) p[k] += 0.5 * eps * grad[k];
  for (int k = 0; k < d; ++k) x[k] += eps * p[k];
  *lp = t.logp(x, grad);
  for (int k = 0; k < d; ++k) p[k] += 0.5 * eps * grad[k];
}

namespace {

struct Point {
  std::vector<double> x, p, g;
  double lp;
};

struct Tree {
  Point edge;                    // last leaf in build order: where the next subtree starts
  std::vector<double> p_first;   // momentum of the first leaf in build order
  std::vector<double> rho;       // sum of momenta over the leaves
  Point prop;                    // current proposal
  double logW;                   // log sum of exp(-H) over the leaves
  bool valid;
};

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double acc = 0;
  for (size_t k = 0; k < a.size(); ++k) acc += a[k] * b[k];
  return acc;
}

double logaddexp(double a, double b) {
  if (a == kNegInf) return b;
  if (b == kNegInf) return a;
  double m = std::max(a, b);
  return m + std::log(std::exp(a - m) + std::exp(b - m));
}

struct Builder {
  const Target& t;
  const Stream& s;
  const NUTSParams& P;
  double H0;
  int n_leapfrog = 0;

  Tree build(const Point& start, int v, int level, int j, int leaf0) {
    if (level == 0) {
      Tree tr;
      tr.edge = start;
      leapfrog(t, tr.edge.x.data(), tr.edge.p.data(), tr.edge.g.data(), &tr.edge.lp, v * P.eps);
      ++n_leapfrog;
      double H = -tr.edge.lp + 0.5 * dot(tr.edge.p, tr.edge.p);
      tr.p_first = tr.edge.p;
      tr.rho = tr.edge.p;
      tr.prop = tr.edge;
      tr.logW = -H;
      note(H - H0, P.max_dH);
      tr.valid = (H - H0 <= P.max_dH);  // false for NaN too
      return tr;
    }
    Tree left = build(start, v, level - 1, j, leaf0);
    if (!left.valid) return left;
    Tree right = build(left.edge, v, level - 1, j, leaf0 + (1 << (level - 1)));
    if (!right.valid) return right;
    Tree tr;
    tr.logW = logaddexp(left.logW, right.logW);
    uint32_t draw = ((uint32_t)j << 16) | ((uint32_t)(leaf0 >> level) << 4) | (uint32_t)level;
    Block b = s.block(2, draw);
    note(std::log(uniform(b.w[0], b.w[1])), right.logW - tr.logW);
    tr.prop = (std::log(uniform(b.w[0], b.w[1])) < right.logW - tr.logW) ? right.prop : left.prop;
    tr.rho = left.rho;
    for (size_t k = 0; k < tr.rho.size(); ++k) tr.rho[k] += right.rho[k];
    tr.p_first = left.p_first;
    tr.edge = right.edge;
    const double rr = dot(tr.rho, tr.rho);
    note_cos(dot(tr.rho, tr.p_first), rr, dot(tr.p_first, tr.p_first));
    note_cos(dot(tr.rho, tr.edge.p), rr, dot(tr.edge.p, tr.edge.p));
    tr.valid = dot(tr.rho, tr.p_first) > 0 && dot(tr.rho, tr.edge.p) > 0;
    return tr;
  }
};

}  // namespace

int nuts_transition(const Target& t, const Stream& s, const NUTSParams& P, double* x,
                    double* lp, double* grad, int* depth) {
  const int d = t.d;
  Point start;
  start.x.assign(x, x + d);
  start.g.assign(grad, grad + d);
  start.lp = *lp;
  start.p.resize(d);
  normals(s, 0, 0, d, start.p.data());
  double H0 = -start.lp + 0.5 * dot(start.p, start.p);

  Point left = start, right = start, prop = start;
  double logW = -H0;
  std::vector<double> rho = start.p;
  Builder B{t, s, P, H0};
  int j = 0;
  for (; j < P.max_depth; ++j) {
    Block b = s.block(1, (uint32_t)j);
    int v = uniform(b.w[0], b.w[1]) < 0.5 ? -1 : 1;
    double log_u = std::log(uniform(b.w[2], b.w[3]));
    Tree sub = B.build(v < 0 ? left : right, v, j, j, 0);
    if (!sub.valid) { ++j; break; }
    note(log_u, sub.logW - logW);
    if (log_u < sub.logW - logW) prop = sub.prop;
    logW = logaddexp(logW, sub.logW);
    for (int k = 0; k < d; ++k) rho[k] += sub.rho[k];
    if (v < 0) left = sub.edge; else right = sub.edge;
    const double rr = dot(rho, rho);
    note_cos(dot(rho, left.p), rr, dot(left.p, left.p));
    note_cos(dot(rho, right.p), rr, dot(right.p, right.p));
    if (!(dot(rho, left.p) > 0 && dot(rho, right.p) > 0)) { ++j; break; }
  }
  for (int k = 0; k < d; ++k) { x[k] = prop.x[k]; grad[k] = prop.g[k]; }
  *lp = prop.lp;
  if (depth) *depth = j;
  return B.n_leapfrog;
}

}  // namespace ora
