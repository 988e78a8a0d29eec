// Oracle RNG and targets (test infrastructure; see oracle.h).
#include "oracle.h"
#include <algorithm>
#include <cmath>
#include <vector>

namespace ora {

// Philox4x32 with 10 rounds, from the definition in Salmon et al. (SC'11), Sec. 4:
// each round multiplies counter words 0 and 2 by the two round multipliers,
// XORs the high halves with the other counter words and the key, and the key is
// bumped by the Weyl constants between rounds.
Block philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
  const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = M0 * (uint64_t)c0;
    uint64_t p1 = M1 * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  Block b;
  b.w[0] = c0; b.w[1] = c1; b.w[2] = c2; b.w[3] = c3;
  return b;
}

double uniform(uint32_t hi, uint32_t lo) {
  uint64_t v = ((uint64_t)hi << 32) | lo;
  v >>= 12;                                  // 52 bits
  return ((double)v + 0.5) * 0x1p-52;        // exact; in [2^-53, 1 - 2^-53]
}

double uniform32(uint32_t w) {
  return ((double)w + 0.5) * 0x1p-32;        // exact; in [2^-33, 1 - 2^-33]
}

// Four normals from one block: the Box-Muller transform of (u(w0), u(w1)) and of
// (u(w2), u(w3)), with r = sqrt(-2 ln u_a) and phi = 2 pi u_b giving (r cos phi, r sin phi).
void normal_quad(const Block& b, double* z) {
  const double kPi = 3.14159265358979323846;
  for (int h = 0; h < 2; ++h) {
    double r = std::sqrt(-2.0 * std::log(uniform32(b.w[2 * h])));
    double phi = 2.0 * kPi * uniform32(b.w[2 * h + 1]);
    z[2 * h] = r * std::cos(phi);
    z[2 * h + 1] = r * std::sin(phi);
  }
}

void normals(const Stream& s, uint32_t tag, uint32_t draw0, int d, double* z) {
  for (int q = 0; 4 * q < d; ++q) {
    double v[4];
    normal_quad(s.block(tag, draw0 + (uint32_t)q), v);
    for (int i = 0; i < 4 && 4 * q + i < d; ++i) z[4 * q + i] = v[i];
  }
}

// softplus(t) = log(1 + e^t), written so that neither branch overflows.
static double softplus(double t) {
  return t > 0 ? t + std::log1p(std::exp(-t)) : std::log1p(std::exp(t));
}

static const double kPiOracle = 3.14159265358979323846;

const double* Target::prior_chol() const {
  switch (kind) {
    case TGT_GAUSS_CONJ: case TGT_GP_LOGIT: case TGT_FLAT: case TGT_GP_REG: return params;
    default: return nullptr;
  }
}

double Target::logp(const double* x, double* grad) const {
  switch (kind) {
    case TGT_FLAT:
      return 0.0;
    case TGT_GAUSS_CONJ: {
      // y ~ N(x, s2 I): log f(x) = -|y - x|^2 / (2 s2)   (constants dropped)
      const double* y = params + (size_t)d * d;
      double s2 = y[d];
      double acc = 0;
      for (int k = 0; k < d; ++k) { double r = y[k] - x[k]; acc += r * r; }
      return -acc / (2.0 * s2);
    }
    case TGT_GP_LOGIT: {
      // Bernoulli-logistic labels s_i in {-1,+1}: log f(x) = -sum softplus(-s_i x_i)
      const double* sg = params + (size_t)d * d;
      double acc = 0;
      for (int k = 0; k < d; ++k) acc += softplus(-sg[k] * x[k]);
      return -acc;
    }
    case TGT_FUNNEL: {
      // v ~ N(0, 3^2), x_i | v ~ N(0, e^v), i = 1..d-1  (constants dropped)
      double v = x[0];
      double ss = 0;
      for (int k = 1; k < d; ++k) ss += x[k] * x[k];
      double ev = std::exp(-v);
      double m = (double)(d - 1);
      if (grad) {
        grad[0] = -v / 9.0 - m / 2.0 + 0.5 * ev * ss;
        for (int k = 1; k < d; ++k) grad[k] = -ev * x[k];
      }
      return -v * v / 18.0 - m * v / 2.0 - 0.5 * ev * ss;
    }
    case TGT_LOGREG: {
      // beta ~ N(0, I), y_i ~ Bernoulli(sigmoid(x_i . beta))
      const double* X = params;
      const double* yv = params + (size_t)n_data * d;
      double acc = 0;
      if (grad) for (int k = 0; k < d; ++k) grad[k] = -x[k];
      for (int k = 0; k < d; ++k) acc -= 0.5 * x[k] * x[k];
      for (int i = 0; i < n_data; ++i) {
        const double* row = X + (size_t)i * d;
        double eta = 0;
        for (int k = 0; k < d; ++k) eta += row[k] * x[k];
        acc += yv[i] * eta - softplus(eta);
        if (grad) {
          double r = yv[i] - 1.0 / (1.0 + std::exp(-eta));
          for (int k = 0; k < d; ++k) grad[k] += row[k] * r;
        }
      }
      return acc;
    }
    case TGT_MOG: {
      // log pi(x) = log sum_k w_k exp(-q_k / 2), q_k = (x - mu_k)^T S^-1 (x - mu_k), with the
      // Sherman-Morrison inverse S^-1 = (I - c 1 1^T) / (1 - rho), c = rho / (1 + (d - 1) rho).
      // The Gaussian normaliser is the same for every component and is dropped.
      // grad = -sum_k r_k S^-1 (x - mu_k), r_k the component responsibilities.
      const int K = n_data;
      const double rho = params[0];
      const double* w = params + 1;
      const double* mu = params + 1 + K;
      const double c = rho / (1.0 + (d - 1) * rho);
      std::vector<double> lw(K), sum_v(K);
      double lmax = -INFINITY;
      for (int k = 0; k < K; ++k) {
        const double* m = mu + (size_t)k * d;
        double vv = 0, sv = 0;
        for (int i = 0; i < d; ++i) { const double v = x[i] - m[i]; vv += v * v; sv += v; }
        const double q = (vv - c * sv * sv) / (1.0 - rho);
        lw[k] = std::log(w[k]) - 0.5 * q;
        sum_v[k] = sv;
        lmax = std::max(lmax, lw[k]);
      }
      double z = 0;
      for (int k = 0; k < K; ++k) z += std::exp(lw[k] - lmax);
      const double lse = lmax + std::log(z);
      if (grad) {
        for (int i = 0; i < d; ++i) grad[i] = 0;
        for (int k = 0; k < K; ++k) {
          const double r = std::exp(lw[k] - lse);
          const double* m = mu + (size_t)k * d;
          for (int i = 0; i < d; ++i) grad[i] -= r * (x[i] - m[i] - c * sum_v[k]) / (1.0 - rho);
        }
      }
      return lse;
    }
    case TGT_GP_REG: {
      // Sec. 7.2: y = f(x) + eps, f ~ GP(0, tau^2 exp(-lambda^2 |x - x'|^2)), eps ~ N(0, sigma^2):
      // the marginal likelihood log N(y; 0, C) with C_ij = tau^2 exp(-lambda^2 D_ij) + sigma^2
      // delta_ij, D_ij = |x_i - x_j|^2, by the Cholesky factorisation C = G G^T:
      // log f = -|G^-1 y|^2 / 2 - sum_i log G_ii - n log(2 pi) / 2.  -inf if C is not positive
      // definite in double precision.
      const int n = n_data;
      const double* D = params + (size_t)d * d;
      const double* y = D + (size_t)n * n;
      const double s2 = x[0] * x[0], t2 = x[1] * x[1], l2 = x[2] * x[2];
      std::vector<double> G((size_t)n * n, 0.0);
      for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j)
          G[(size_t)i * n + j] = t2 * std::exp(-l2 * D[(size_t)i * n + j]) + (i == j ? s2 : 0.0);
      for (int j = 0; j < n; ++j) {  // Cholesky-Crout, column by column
        double dj = G[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) dj -= G[(size_t)j * n + k] * G[(size_t)j * n + k];
        if (!(dj > 0)) return -INFINITY;
        const double gjj = std::sqrt(dj);
        G[(size_t)j * n + j] = gjj;
        for (int i = j + 1; i < n; ++i) {
          double v = G[(size_t)i * n + j];
          for (int k = 0; k < j; ++k) v -= G[(size_t)i * n + k] * G[(size_t)j * n + k];
          G[(size_t)i * n + j] = v / gjj;
        }
      }
      double quad = 0, logdet_half = 0;
      std::vector<double> a(n);
      for (int i = 0; i < n; ++i) {  // forward substitution G a = y
        double v = y[i];
        for (int k = 0; k < i; ++k) v -= G[(size_t)i * n + k] * a[k];
        a[i] = v / G[(size_t)i * n + i];
        quad += a[i] * a[i];
        logdet_half += std::log(G[(size_t)i * n + i]);
      }
      return -0.5 * quad - logdet_half - 0.5 * n * std::log(2.0 * kPiOracle);
    }
    case TGT_GAUSS_DIAG: {
      const double* mu = params;
      const double* sd = params + d;
      double acc = 0;
      for (int k = 0; k < d; ++k) {
        double z = (x[k] - mu[k]) / sd[k];
        acc -= 0.5 * z * z;
        if (grad) grad[k] = -z / sd[k];
      }
      return acc;
    }
  }
  return std::nan("");
}

}  // namespace ora
