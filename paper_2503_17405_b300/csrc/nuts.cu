// The No-U-Turn sampler (multinomial form) as a finite state machine.
//
// States (Fig. 2, "HMC-NUTS"): INIT draws the momentum and opens the trajectory; DOUBLE
// picks the direction of the next subtree; INTEGRATE (the inner loop body) takes one
// leapfrog step, adds the new leaf to the subtree and merges completed blocks; CHECK (the
// outer loop body's tail) accepts the finished subtree progressively and tests the whole
// trajectory for a U-turn; DONE emits the sample.  One FSM step is Alg. 9's bundled step
// inside an amortised step: the cheap states run inline until the next gradient is
// needed, then exactly one gradient evaluation (one leapfrog) is made.  A sample costs as
// many steps as it takes leapfrog steps.
//
// The subtree is built iteratively: after leaf L (0-based) of subtree j, every block of
// 2^(l+1) leaves that L completes is merged with its left half, which waits in a per-level
// slot; a block that U-turns, or a leaf that diverges, ends the transition.  The random
// numbers are keyed exactly like the recursive definition (direction and progressive
// acceptance of doubling j: tag 1, draw j; the merge at level l of block b of subtree j:
// tag 2, draw (j << 16) | (b << 4) | l; momentum: tag 0).
//
// Layout: one chain per warp; lane l holds coordinates l, l + 32, ....
#include <algorithm>
#include <cstring>
#include "engine_internal.h"
#include "fsmc_device.cuh"
#include "fsmc_kernels.h"

namespace fsmc {

enum NutsState : int { N_INIT = 0, N_DOUBLE = 1, N_INTEGRATE = 2, N_CHECK = 3, N_DONE = 4 };
enum NutsVec : int { V_GX = 0, V_XL, V_PL, V_GL, V_XR, V_PR, V_GR, V_RHO, V_XP, V_GP, NV };
enum NutsSc : int { S_LPX = 0, S_LPL, S_LPR, S_LPP, S_H0, S_LOGW, NSC };
enum NutsInt : int { I_ST = 0, I_J, I_L, I_V, I_NLEAP, NI };
constexpr int kBatchChains = 8;  // chains per block sharing one batched gradient
constexpr int kLevels = 10;   // slots for levels 0..9
constexpr int kWarpsMax = 8;  // warps per block (threads <= 256)
constexpr int kWsm = 160;     // per-warp scratch: theta (<= 128) + 32 residuals

template <typename T>
struct NutsView : ChainsView<T> {
  TargetView<T> tg;
  T eps, max_dH;
  int max_depth;
  T* vec;   // [NV][m][d]
  T* sc;    // [NSC][m]
  int* iv;  // [NI][m]
  T* stk;   // [m][kLevels][4][d]: p_first, rho, prop x, prop grad
  T* stks;  // [m][kLevels][2]: prop log-density, log-weight
  T* sub;   // [3][m][d]: completed subtree rho, prop x, prop grad (synchronised mode)
  T* subs;  // [2][m]: its prop log-density and log-weight
  int* aux; // [m][n] tree depth
  int* sched;  // [2]: group rotation and block ticket of the batched FSM launch
};

template <typename T>
__device__ __forceinline__ T t_exp(T a) { if constexpr (sizeof(T) == 4) return __expf(a); else return exp(a); }
template <typename T>
__device__ __forceinline__ T t_log(T a) { if constexpr (sizeof(T) == 4) return __logf(a); else return log(a); }

template <typename T>
__device__ __forceinline__ T logaddexp(T a, T b) {
  if (a == neg_inf<T>()) return b;
  if (b == neg_inf<T>()) return a;
  const T m = a > b ? a : b;
  if constexpr (sizeof(T) == 4) return m + __logf(1.f + __expf(-fabsf(a - b)));
  else return m + log(exp(a - m) + exp(b - m));
}

template <typename T, int E>
__device__ __forceinline__ T wdot(const T (&a)[E], const T (&b)[E]) {
  T s = T(0);
#pragma unroll
  for (int e = 0; e < E; ++e) s = fma(a[e], b[e], s);  // padded coordinates hold 0
  return group_sum<32>(s);
}

// Mixture of K Gaussians with the shared equicorrelated covariance S (Sec. 7.3), one chain per
// warp.  For component k, with v = x - mu_k split into its mean part s_k / d (s_k = 1^T v) and the
// residual u = v - (s_k / d) 1:  q_k = s_k^2 c_par / d + |u|^2 c_perp and
// S^-1 v = (s_k c_par / d) 1 + c_perp u.  s_k is summed from v itself, not as 1^T x - 1^T mu_k:
// the residual force c_perp u is ~1 / (1 - rho) times stiffer than the force along 1, so the
// rounding of a difference of two large sums would swamp the latter in single precision.  For
// the same reason the residual is re-centred once more: the roundings of v_i - mean leave
// 1^T u ~ sqrt(d) ulp, which c_perp would turn into a spurious force along 1 (errors of ~1e-4
// after 1000 single-precision leapfrog steps, ~1e-6 re-centred).
// log pi = logsumexp_k (log w_k - q_k / 2) and grad = -sum_k r_k S^-1 v_k are accumulated over
// the components, rescaled whenever the running maximum of the log-terms grows.  This adds the
// KC components k0 .. k0 + KC - 1, their three warp reductions interleaved.
template <typename T, int E, int KC>
__device__ __forceinline__ void mog_terms(const TargetView<T>& tg, const T (&x)[E], int k0, int lane, T inv_d,
                                          T& lmax, T& wsum, T (&gacc)[E]) {
  const int d = tg.d;
  T u[KC][E], sk[KC], mean[KC], su[KC], uu[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    const T* mk = tg.X + (size_t)(k0 + c) * d;
    sk[c] = T(0);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int i = lane + 32 * e;
      u[c][e] = i < d ? x[e] - mk[i] : T(0);
      sk[c] += u[c][e];
    }
  }
  group_sum_n<32, KC>(sk);
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    mean[c] = sk[c] * inv_d;
    su[c] = T(0);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if (lane + 32 * e < d) u[c][e] -= mean[c];
      su[c] += u[c][e];
    }
  }
  group_sum_n<32, KC>(su);
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    const T du = su[c] * inv_d;
    uu[c] = T(0);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if (lane + 32 * e < d) u[c][e] -= du;
      uu[c] = fma(u[c][e], u[c][e], uu[c]);
    }
  }
  group_sum_n<32, KC>(uu);  // the same bits in every lane: the branches below are warp-uniform
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    const T lk = tg.vec[k0 + c] - T(0.5) * fma(sk[c] * mean[c], tg.c_par, uu[c] * tg.c_perp);
    const T gpar = mean[c] * tg.c_par;
    T wk = T(1);
    if (lk > lmax) {
      const T sc = t_exp(lmax - lk);  // 0 for the first component
      wsum *= sc;
#pragma unroll
      for (int e = 0; e < E; ++e) gacc[e] *= sc;
      lmax = lk;
    } else {
      wk = t_exp(lk - lmax);
    }
    wsum += wk;
#pragma unroll
    for (int e = 0; e < E; ++e) gacc[e] = fma(wk, fma(u[c][e], tg.c_perp, gpar), gacc[e]);
  }
}

// log pi(x) and its gradient, one chain per warp.  wsm: this warp's shared scratch.
template <typename T, int E>
__device__ T logp_grad(const TargetView<T>& tg, const T (&x)[E], T (&g)[E], int lane, T* wsm) {
  const int d = tg.d;
  if (tg.kind == TGT_GAUSS_DIAG) {
    T acc = T(0);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = lane + 32 * e;
      if (k < d) {
        const T z = (x[e] - tg.vec[k]) / tg.vec2[k];
        acc = fma(z, z, acc);
        g[e] = -z / tg.vec2[k];
      } else {
        g[e] = T(0);
      }
    }
    return -T(0.5) * group_sum<32>(acc);
  }
  if (tg.kind == TGT_FUNNEL) {
    const T v = __shfl_sync(0xffffffffu, x[0], 0);
    T ss = T(0);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = lane + 32 * e;
      if (k >= 1 && k < d) ss = fma(x[e], x[e], ss);
    }
    ss = group_sum<32>(ss);
    const T ev = t_exp(-v);
    const T m1 = T(d - 1);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = lane + 32 * e;
      g[e] = (k >= 1 && k < d) ? -ev * x[e] : T(0);
    }
    if (lane == 0) g[0] = -v / T(9) - m1 / T(2) + T(0.5) * ev * ss;
    return -v * v / T(18) - m1 * v / T(2) - T(0.5) * ev * ss;
  }
  if (tg.kind == TGT_MOG) {
    const int K = tg.n_data;
    const T inv_d = T(1) / T(d);
    T lmax = neg_inf<T>(), wsum = T(0), gacc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) gacc[e] = T(0);
    int k0 = 0;
    for (; k0 + 4 <= K; k0 += 4) mog_terms<T, E, 4>(tg, x, k0, lane, inv_d, lmax, wsum, gacc);
    switch (K - k0) {
      case 3: mog_terms<T, E, 3>(tg, x, k0, lane, inv_d, lmax, wsum, gacc); break;
      case 2: mog_terms<T, E, 2>(tg, x, k0, lane, inv_d, lmax, wsum, gacc); break;
      case 1: mog_terms<T, E, 1>(tg, x, k0, lane, inv_d, lmax, wsum, gacc); break;
      default: break;
    }
    const T inv_w = T(1) / wsum;
#pragma unroll
    for (int e = 0; e < E; ++e) g[e] = lane + 32 * e < d ? -gacc[e] * inv_w : T(0);
    return lmax + t_log(wsum);
  }
  // TGT_LOGREG: eta = X theta row by row (lanes over rows), then grad = X^T r (lanes over
  // coordinates), 32 rows at a time through the warp's shared scratch.
  const int n = tg.n_data;
  T* th = wsm;
  T* rs = wsm + 128;
  T sq = T(0);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = lane + 32 * e;
    if (k < d) { th[k] = x[e]; sq = fma(x[e], x[e], sq); }
    g[e] = T(0);
  }
  __syncwarp();
  T lpart = T(0);
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int i = i0 + lane;
    T r = T(0);
    if (i < n) {
      const T* row = tg.X + (size_t)i * d;
      T eta = T(0);
      for (int k = 0; k < d; ++k) eta = fma(row[k], th[k], eta);
      const T yi = tg.vec[i];
      const T sig = T(1) / (T(1) + t_exp(-eta));
      r = yi - sig;
      lpart += yi * eta - softplus<T>(eta);
    }
    rs[lane] = r;
    __syncwarp();
    const int q_end = min(32, n - i0);
    for (int q = 0; q < q_end; ++q) {
      const T rq = rs[q];
      const T* row = tg.X + (size_t)(i0 + q) * d;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = lane + 32 * e;
        if (k < d) g[e] = fma(row[k], rq, g[e]);
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = lane + 32 * e;
    if (k < d) g[e] -= x[e];
  }
  return group_sum<32>(lpart) - T(0.5) * group_sum<32>(sq);
}

// ---- per-chain register state ---------------------------------------------------------------------
template <typename T, int E>
struct Chain {
  T x[E], gx[E], xl[E], pl[E], gl[E], xr[E], pr[E], gr[E], rho[E], xp[E], gp[E];
  T lpx, lpl, lpr, lpp, H0, logW;
  int st, j, L, v, nleap, t;
};

template <typename T, int E>
__device__ __forceinline__ void vload(const NutsView<T>& v, const T* base, int64_t c, int lane, T (&a)[E]) {
  const int d = v.tg.d;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = lane + 32 * e;
    a[e] = k < d ? base[(size_t)c * d + k] : T(0);
  }
}

template <typename T, int E>
__device__ __forceinline__ void vstore(const NutsView<T>& v, T* base, int64_t c, int lane, const T (&a)[E]) {
  const int d = v.tg.d;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = lane + 32 * e;
    if (k < d) base[(size_t)c * d + k] = a[e];
  }
}

template <typename T, int E>
__device__ void chain_load(const NutsView<T>& v, int64_t c, int lane, Chain<T, E>& s) {
  const size_t md = (size_t)v.m * v.tg.d;
  vload<T, E>(v, v.x, c, lane, s.x);
  vload<T, E>(v, v.vec + V_GX * md, c, lane, s.gx);
  vload<T, E>(v, v.vec + V_XL * md, c, lane, s.xl);
  vload<T, E>(v, v.vec + V_PL * md, c, lane, s.pl);
  vload<T, E>(v, v.vec + V_GL * md, c, lane, s.gl);
  vload<T, E>(v, v.vec + V_XR * md, c, lane, s.xr);
  vload<T, E>(v, v.vec + V_PR * md, c, lane, s.pr);
  vload<T, E>(v, v.vec + V_GR * md, c, lane, s.gr);
  vload<T, E>(v, v.vec + V_RHO * md, c, lane, s.rho);
  vload<T, E>(v, v.vec + V_XP * md, c, lane, s.xp);
  vload<T, E>(v, v.vec + V_GP * md, c, lane, s.gp);
  const int64_t m = v.m;
  s.lpx = v.sc[S_LPX * m + c]; s.lpl = v.sc[S_LPL * m + c]; s.lpr = v.sc[S_LPR * m + c];
  s.lpp = v.sc[S_LPP * m + c]; s.H0 = v.sc[S_H0 * m + c]; s.logW = v.sc[S_LOGW * m + c];
  s.st = v.iv[I_ST * m + c]; s.j = v.iv[I_J * m + c]; s.L = v.iv[I_L * m + c];
  s.v = v.iv[I_V * m + c]; s.nleap = v.iv[I_NLEAP * m + c];
  s.t = v.t[c];
}

template <typename T, int E>
__device__ void chain_store(const NutsView<T>& v, int64_t c, int lane, const Chain<T, E>& s) {
  const size_t md = (size_t)v.m * v.tg.d;
  vstore<T, E>(v, v.x, c, lane, s.x);
  vstore<T, E>(v, v.vec + V_GX * md, c, lane, s.gx);
  vstore<T, E>(v, v.vec + V_XL * md, c, lane, s.xl);
  vstore<T, E>(v, v.vec + V_PL * md, c, lane, s.pl);
  vstore<T, E>(v, v.vec + V_GL * md, c, lane, s.gl);
  vstore<T, E>(v, v.vec + V_XR * md, c, lane, s.xr);
  vstore<T, E>(v, v.vec + V_PR * md, c, lane, s.pr);
  vstore<T, E>(v, v.vec + V_GR * md, c, lane, s.gr);
  vstore<T, E>(v, v.vec + V_RHO * md, c, lane, s.rho);
  vstore<T, E>(v, v.vec + V_XP * md, c, lane, s.xp);
  vstore<T, E>(v, v.vec + V_GP * md, c, lane, s.gp);
  if (lane == 0) {
    const int64_t m = v.m;
    v.sc[S_LPX * m + c] = s.lpx; v.sc[S_LPL * m + c] = s.lpl; v.sc[S_LPR * m + c] = s.lpr;
    v.sc[S_LPP * m + c] = s.lpp; v.sc[S_H0 * m + c] = s.H0; v.sc[S_LOGW * m + c] = s.logW;
    v.iv[I_ST * m + c] = s.st; v.iv[I_J * m + c] = s.j; v.iv[I_L * m + c] = s.L;
    v.iv[I_V * m + c] = s.v; v.iv[I_NLEAP * m + c] = s.nleap;
    v.t[c] = s.t;
  }
}

template <typename T>
__device__ __forceinline__ T* stk_vec(const NutsView<T>& v, int64_t c, int lvl, int f) {
  return v.stk + (((size_t)c * kLevels + lvl) * 4 + f) * v.tg.d;
}

// INIT (S1): momentum, H0, a one-point trajectory.
template <typename T, int E>
__device__ void nuts_init(const NutsView<T>& v, const Key& key, int lane, Chain<T, E>& s) {
  const int d = v.tg.d;
  T p[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = lane + 32 * e;
    p[e] = T(0);
    if (k < d) {
      T z[4];
      Conv<T>::normal_quad(key.block((uint32_t)s.t, 0, (uint32_t)(k >> 2)), z);
      const int i = k & 3;
      p[e] = i == 0 ? z[0] : i == 1 ? z[1] : i == 2 ? z[2] : z[3];
    }
  }
  s.H0 = -s.lpx + T(0.5) * wdot<T, E>(p, p);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    s.xl[e] = s.xr[e] = s.xp[e] = s.x[e];
    s.gl[e] = s.gr[e] = s.gp[e] = s.gx[e];
    s.pl[e] = s.pr[e] = s.rho[e] = p[e];
  }
  s.lpl = s.lpr = s.lpp = s.lpx;
  s.logW = -s.H0;
  s.j = 0;
  s.nleap = 0;
  s.st = N_DOUBLE;
}

// DOUBLE (S2): direction of subtree j.
template <typename T, int E>
__device__ __forceinline__ void nuts_double(const Key& key, Chain<T, E>& s) {
  const P4 b = key.block((uint32_t)s.t, 1, (uint32_t)s.j);
  s.v = (b.w0 & 0x80000000u) ? 1 : -1;  // u(w0, w1) < 1/2 exactly when the top bit is clear
  s.L = 0;
  s.st = N_INTEGRATE;
}

// Completed subtree summary handed from INTEGRATE to CHECK.
template <typename T, int E>
struct Sub {
  T rho[E], xp[E], gp[E];
  T lpp, logW;
};

// INTEGRATE (S3), split around the gradient so that a block can batch it over its chains.
// First half: the momentum half-kick and the position drift from the edge on side v.
template <typename T, int E>
struct Leaf {
  T xe[E], pe[E], ge[E];
  T half;
  bool left;
};

template <typename T, int E>
__device__ __forceinline__ void nuts_lf_pre(const NutsView<T>& v, const Chain<T, E>& s, Leaf<T, E>& lf) {
  lf.left = s.v < 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    lf.xe[e] = lf.left ? s.xl[e] : s.xr[e];
    lf.pe[e] = lf.left ? s.pl[e] : s.pr[e];
    lf.ge[e] = lf.left ? s.gl[e] : s.gr[e];
  }
  const T es = s.v < 0 ? -v.eps : v.eps;
  lf.half = T(0.5) * es;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    lf.pe[e] += lf.half * lf.ge[e];
    lf.xe[e] += es * lf.pe[e];
  }
}

template <typename T, int E>
__device__ int nuts_lf_post(const NutsView<T>& v, const Key& key, int64_t c, int lane, Chain<T, E>& s,
                            Leaf<T, E>& lf, T lpe, Sub<T, E>& out);

// One leapfrog from the edge on side v, then the merges this leaf completes.
// Returns 0: keep integrating; 1: subtree complete (summary in `out`); 2: subtree invalid.
template <typename T, int E>
__device__ int nuts_integrate(const NutsView<T>& v, const Key& key, int64_t c, int lane, T* wsm,
                              Chain<T, E>& s, Sub<T, E>& out) {
  Leaf<T, E> lf;
  nuts_lf_pre<T, E>(v, s, lf);
  const T lpe = logp_grad<T, E>(v.tg, lf.xe, lf.ge, lane, wsm);
  return nuts_lf_post<T, E>(v, key, c, lane, s, lf, lpe, out);
}

// Second half: the closing half-kick with the new gradient, the divergence test and the
// merges of every block this leaf completes.
template <typename T, int E>
__device__ int nuts_lf_post(const NutsView<T>& v, const Key& key, int64_t c, int lane, Chain<T, E>& s,
                            Leaf<T, E>& lf, T lpe, Sub<T, E>& out) {
  const int d = v.tg.d;
  T (&xe)[E] = lf.xe;
  T (&pe)[E] = lf.pe;
  T (&ge)[E] = lf.ge;
  const bool left = lf.left;
#pragma unroll
  for (int e = 0; e < E; ++e) pe[e] += lf.half * ge[e];
  s.nleap += 1;
  if (!(lpe == lpe)) { lpe = neg_inf<T>(); atomicOr(v.err, ERR_NONFINITE); }
  // the new leaf becomes the trajectory's edge on side v
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (left) { s.xl[e] = xe[e]; s.pl[e] = pe[e]; s.gl[e] = ge[e]; }
    else { s.xr[e] = xe[e]; s.pr[e] = pe[e]; s.gr[e] = ge[e]; }
  }
  if (left) s.lpl = lpe; else s.lpr = lpe;
  const T H = -lpe + T(0.5) * wdot<T, E>(pe, pe);
  bool valid = (H - s.H0 <= v.max_dH);
  if (!valid) return 2;
  // leaf summary
  T cpf[E], crho[E], cxp[E], cgp[E];
#pragma unroll
  for (int e = 0; e < E; ++e) { cpf[e] = pe[e]; crho[e] = pe[e]; cxp[e] = xe[e]; cgp[e] = ge[e]; }
  T clpp = lpe, clogW = -H;
  int lvl = 0;
  while (((s.L >> lvl) & 1) != 0) {
    // merge with the waiting left half of level lvl
    T spf[E], srho[E];
    const T* sp = stk_vec(v, c, lvl, 0);
    const T* sr = stk_vec(v, c, lvl, 1);
    const T slpp = v.stks[((size_t)c * kLevels + lvl) * 2];
    const T slogW = v.stks[((size_t)c * kLevels + lvl) * 2 + 1];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = lane + 32 * e;
      spf[e] = k < d ? sp[k] : T(0);
      srho[e] = k < d ? sr[k] : T(0);
    }
    const T nlogW = logaddexp(slogW, clogW);
    const uint32_t blk = (uint32_t)(s.L >> (lvl + 1));
    const uint32_t draw = ((uint32_t)s.j << 16) | (blk << 4) | (uint32_t)(lvl + 1);
    const P4 b = key.block((uint32_t)s.t, 2, draw);
    if (!(Conv<T>::log_u(b.w0, b.w1) < clogW - nlogW)) {  // keep the left half's proposal
      const T* sx = stk_vec(v, c, lvl, 2);
      const T* sg = stk_vec(v, c, lvl, 3);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = lane + 32 * e;
        cxp[e] = k < d ? sx[k] : T(0);
        cgp[e] = k < d ? sg[k] : T(0);
      }
      clpp = slpp;
    }
#pragma unroll
    for (int e = 0; e < E; ++e) { crho[e] = srho[e] + crho[e]; cpf[e] = spf[e]; }
    clogW = nlogW;
    ++lvl;
    valid = wdot<T, E>(crho, cpf) > T(0) && wdot<T, E>(crho, pe) > T(0);
    if (!valid) return 2;
  }
  if (s.L == (1 << s.j) - 1) {
#pragma unroll
    for (int e = 0; e < E; ++e) { out.rho[e] = crho[e]; out.xp[e] = cxp[e]; out.gp[e] = cgp[e]; }
    out.lpp = clpp;
    out.logW = clogW;
    return 1;
  }
  // this block waits as the left half of level lvl
  T* dp = stk_vec(v, c, lvl, 0);
  T* dr = stk_vec(v, c, lvl, 1);
  T* dx = stk_vec(v, c, lvl, 2);
  T* dg = stk_vec(v, c, lvl, 3);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = lane + 32 * e;
    if (k < d) { dp[k] = cpf[e]; dr[k] = crho[e]; dx[k] = cxp[e]; dg[k] = cgp[e]; }
  }
  if (lane == 0) {
    v.stks[((size_t)c * kLevels + lvl) * 2] = clpp;
    v.stks[((size_t)c * kLevels + lvl) * 2 + 1] = clogW;
  }
  __syncwarp();
  s.L += 1;
  return 0;
}

// CHECK (S4): progressive acceptance of the finished subtree and the trajectory U-turn test.
// Returns true when the transition continues with another doubling.
template <typename T, int E>
__device__ bool nuts_check(const NutsView<T>& v, const Key& key, Chain<T, E>& s, const Sub<T, E>& sb) {
  const P4 b = key.block((uint32_t)s.t, 1, (uint32_t)s.j);
  if (Conv<T>::log_u(b.w2, b.w3) < sb.logW - s.logW) {
#pragma unroll
    for (int e = 0; e < E; ++e) { s.xp[e] = sb.xp[e]; s.gp[e] = sb.gp[e]; }
    s.lpp = sb.lpp;
  }
  s.logW = logaddexp(s.logW, sb.logW);
#pragma unroll
  for (int e = 0; e < E; ++e) s.rho[e] += sb.rho[e];
  const bool turn = !(wdot<T, E>(s.rho, s.pl) > T(0) && wdot<T, E>(s.rho, s.pr) > T(0));
  if (turn || s.j + 1 >= v.max_depth) return false;
  s.j += 1;
  s.st = N_DOUBLE;
  return true;
}

// DONE (S5): the proposal becomes the sample.
template <typename T, int E>
__device__ void nuts_done(const NutsView<T>& v, int64_t c, int lane, Chain<T, E>& s) {
  const int d = v.tg.d;
#pragma unroll
  for (int e = 0; e < E; ++e) { s.x[e] = s.xp[e]; s.gx[e] = s.gp[e]; }
  s.lpx = s.lpp;
  if (v.out) {
    T* dst = v.out + ((size_t)c * v.n + s.t) * d;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = lane + 32 * e;
      if (k < d) dst[k] = s.x[e];
    }
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = lane + 32 * e;
      if (k >= d) continue;
      const size_t o = (size_t)c * d + k;
      const size_t st = v.mom_stride;
      T* mo = v.mom;
      T y = s.x[e] - mo[o + st]; T tt = mo[o] + y; mo[o + st] = (tt - mo[o]) - y; mo[o] = tt;
      const T x2 = s.x[e] * s.x[e];
      y = x2 - mo[o + 3 * st]; tt = mo[o + 2 * st] + y; mo[o + 3 * st] = (tt - mo[o + 2 * st]) - y;
      mo[o + 2 * st] = tt;
    }
  }
  if (lane == 0) {
    v.counts[(size_t)c * v.n + s.t] = s.nleap;
    v.aux[(size_t)c * v.n + s.t] = s.j + 1;
  }
  s.t += 1;
  s.st = N_INIT;
  if (s.t == v.n && lane == 0) atomicAdd(v.chains_done, 1);
}

// ---- FSM kernel: each chain advances `budget` leapfrog steps ---------------------------------------
template <typename T, int E>
__device__ __forceinline__ void nuts_advance_chain(const NutsView<T>& v, int64_t c, int budget, int lane,
                                                   T* wsm) {
  Chain<T, E> s;
  chain_load<T, E>(v, c, lane, s);
  if (s.t >= v.n) return;
  const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
  long long steps = 0;
  for (int b = 0; b < budget && s.t < v.n; ++b) {
    if (s.st == N_INIT) nuts_init<T, E>(v, key, lane, s);
    if (s.st == N_DOUBLE) nuts_double<T, E>(key, s);
    Sub<T, E> sb;
    const int r = nuts_integrate<T, E>(v, key, c, lane, wsm, s, sb);
    ++steps;
    if (r == 1 && nuts_check<T, E>(v, key, s, sb)) continue;
    if (r != 0) nuts_done<T, E>(v, c, lane, s);
  }
  chain_store<T, E>(v, c, lane, s);
  if (lane == 0) v.steps[c] += steps;
}

// A chain per warp.  (A resident grid with balanced warp times, as the batched kernel has, was
// measured slower here: 240 against 236 ms per 4096-chain mixture job; the chains' states vary
// in cost, and the hardware's block scheduler already evens out the blocks' times.)
template <typename T, int E>
__global__ void __launch_bounds__(256) nuts_fsm_kernel(NutsView<T> v, int budget) {
  __shared__ T wsm_all[kWarpsMax][kWsm];
  const int lane = threadIdx.x & 31;
  T* wsm = wsm_all[threadIdx.x >> 5];
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < v.m; c += nwarps) nuts_advance_chain<T, E>(v, c, budget, lane, wsm);
}

// Fused launch over several NUTS jobs (serving): job k owns chains off[k] .. off[k+1].
template <typename T, int E>
__global__ void __launch_bounds__(256) nuts_fsm_multi_kernel(const NutsView<T>* views, const int64_t* off,
                                                             int njobs, int64_t total, int budget) {
  __shared__ T wsm_all[kWarpsMax][kWsm];
  const int lane = threadIdx.x & 31;
  T* wsm = wsm_all[threadIdx.x >> 5];
  const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (item >= total) return;
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= item) lo = mid; else hi = mid - 1;
  }
  const NutsView<T> v = views[lo];
  nuts_advance_chain<T, E>(v, item - off[lo], budget, lane, wsm);
}

// ---- block-batched gradient (logistic regression) ------------------------------------------------------
// Every FSM step makes exactly one gradient evaluation per chain, so the C chains of a block
// share one evaluation: eta = X Theta (n x C) with rows split over the threads (4 rows x C chains
// register tile per thread, X^T read as 4-row vectors), r = y - sigmoid(eta), then
// g = X^T R (d x C) with (coordinate, row-range) pairs split over the threads, and the prior
// term -theta.  Rows are processed in chunks of 4 x blockDim rows through shared memory.
template <typename T, int C>
struct GradSmem {
  T* th;     // [128][C] positions of the block's chains
  T* G;      // [128][C] gradients
  T* lp;     // [C] log densities
  T* R;      // [4 * 32 C][C] residuals of one row chunk
  T* part;   // [C][32 C] per-thread partial gradients (chain-major)
  T* lpart;  // [C][C] per-warp partial log densities
};

template <typename T, int C>
__device__ __forceinline__ GradSmem<T, C> grad_smem(T* base) {
  constexpr int NT = 32 * C;
  GradSmem<T, C> g;
  g.th = base;
  g.G = g.th + 128 * C;
  g.lp = g.G + 128 * C;
  g.R = g.lp + C;
  g.part = g.R + 4 * NT * C;
  g.lpart = g.part + NT * C;
  return g;
}

template <typename T, int C>
constexpr size_t grad_smem_bytes() {
  constexpr int NT = 32 * C;
  return sizeof(T) * ((size_t)128 * C * 2 + C + 4 * NT * C + NT * C + C * C);
}

template <typename T, int C>
__device__ void block_logreg_grad(const TargetView<T>& tg, const GradSmem<T, C>& sm) {
  constexpr int NT = 32 * C;
  constexpr int RPT = 4;
  constexpr int RC = RPT * NT;
  const int n = tg.n_data, d = tg.d, np = tg.n_pad;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int nsub = NT / d;
  const int kk = t % d, sub = t / d;
  const bool c_role = sub < nsub;
  T gacc[C], lpacc[C];
  // FP32: each chain's gradient partial as an (even rows, odd rows) pair for the packed
  // multiply-add; the two halves are added at the end
  float2 gacc2[C];
#pragma unroll
  for (int c = 0; c < C; ++c) { gacc[c] = T(0); lpacc[c] = T(0); gacc2[c] = make_float2(0.f, 0.f); }
  for (int i0 = 0; i0 < n; i0 += RC) {
    // eta for rows ib .. ib+3 and all C chains
    const int ib = i0 + RPT * t;
    T eta[RPT][C];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
      for (int c = 0; c < C; ++c) eta[r][c] = T(0);
    if (ib < np) {
      // unrolled so that several rows of X^T are in flight from L2 at once
#pragma unroll 2
      for (int k = 0; k < d; ++k) {
        const T* xr = tg.XT + (size_t)k * np + ib;
        T x4[RPT];
        if constexpr (sizeof(T) == 4) {
          const float4 f = __ldg(reinterpret_cast<const float4*>(xr));
          x4[0] = f.x; x4[1] = f.y; x4[2] = f.z; x4[3] = f.w;
        } else {
          const double2 a = __ldg(reinterpret_cast<const double2*>(xr));
          const double2 b = __ldg(reinterpret_cast<const double2*>(xr) + 1);
          x4[0] = a.x; x4[1] = a.y; x4[2] = b.x; x4[3] = b.y;
        }
        if constexpr (sizeof(T) == 4 && C % 2 == 0) {
          // chain pairs with the packed FP32 multiply-add (each lane of the pair rounds as fmaf)
          float2 th2[C / 2];
#pragma unroll
          for (int c = 0; c < C / 2; ++c) th2[c] = reinterpret_cast<const float2*>(sm.th + k * C)[c];
#pragma unroll
          for (int r = 0; r < RPT; ++r) {
            const float2 xr = make_float2(x4[r], x4[r]);
#pragma unroll
            for (int c = 0; c < C / 2; ++c) {
              const float2 e2 = __ffma2_rn(xr, th2[c], make_float2(eta[r][2 * c], eta[r][2 * c + 1]));
              eta[r][2 * c] = e2.x;
              eta[r][2 * c + 1] = e2.y;
            }
          }
        } else {
          T th[C];
#pragma unroll
          for (int c = 0; c < C; ++c) th[c] = sm.th[k * C + c];
#pragma unroll
          for (int r = 0; r < RPT; ++r)
#pragma unroll
            for (int c = 0; c < C; ++c) eta[r][c] = fma(x4[r], th[c], eta[r][c]);
        }
      }
    }
    // residuals, chain-major [C][RC]: each thread stores its 4 rows of a chain as one vector
#pragma unroll
    for (int c = 0; c < C; ++c) {
      T rv[RPT];
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const int i = ib + r;
        const bool ok = i < n;
        const T yi = ok ? tg.vec[i] : T(0);
        const T e = eta[r][c];
        const T sig = T(1) / (T(1) + t_exp(-e));
        rv[r] = ok ? yi - sig : T(0);
        if (ok) lpacc[c] += yi * e - softplus<T>(e);
      }
      T* dst = sm.R + c * RC + RPT * t;
      if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(dst) = make_float4(rv[0], rv[1], rv[2], rv[3]);
      } else {
        reinterpret_cast<double2*>(dst)[0] = make_double2(rv[0], rv[1]);
        reinterpret_cast<double2*>(dst)[1] = make_double2(rv[2], rv[3]);
      }
    }
    __syncthreads();
    if (c_role) {
      // rows of this chunk in 4-row groups: g_k += X^T[k][rows] . R[c][rows]
      const int rows = min(RC, n - i0);
      const int groups = (rows + RPT - 1) / RPT;
      const int gseg = (groups + nsub - 1) / nsub;
      const int g_beg = sub * gseg, g_end = min(groups, g_beg + gseg);
      const T* xk = tg.XT + (size_t)kk * np + i0;
#pragma unroll 2
      for (int gi = g_beg; gi < g_end; ++gi) {
        T x4[RPT];
        if constexpr (sizeof(T) == 4) {
          const float4 f = __ldg(reinterpret_cast<const float4*>(xk + RPT * gi));
          x4[0] = f.x; x4[1] = f.y; x4[2] = f.z; x4[3] = f.w;
        } else {
          const double2 a = __ldg(reinterpret_cast<const double2*>(xk + RPT * gi));
          const double2 b = __ldg(reinterpret_cast<const double2*>(xk + RPT * gi) + 1);
          x4[0] = a.x; x4[1] = a.y; x4[2] = b.x; x4[3] = b.y;
        }
        if constexpr (sizeof(T) == 4) {
          const float2 x01 = make_float2(x4[0], x4[1]), x23 = make_float2(x4[2], x4[3]);
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const float4 r4 = *reinterpret_cast<const float4*>(sm.R + c * RC + RPT * gi);
            gacc2[c] = __ffma2_rn(x01, make_float2(r4.x, r4.y), gacc2[c]);
            gacc2[c] = __ffma2_rn(x23, make_float2(r4.z, r4.w), gacc2[c]);
          }
        } else {
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const T* rc = sm.R + c * RC + RPT * gi;
#pragma unroll
            for (int r = 0; r < RPT; ++r) gacc[c] = fma(x4[r], rc[r], gacc[c]);
          }
        }
      }
    }
    __syncthreads();
  }
  // reduce the gradient partials over row ranges, the log-density partials over warps
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int c = 0; c < C; ++c) gacc[c] = gacc2[c].x + gacc2[c].y;
  }
  // chain-major [C][NT]: consecutive threads write consecutive words (no bank conflicts)
#pragma unroll
  for (int c = 0; c < C; ++c) sm.part[c * NT + t] = c_role ? gacc[c] : T(0);
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const T s = group_sum<32>(lpacc[c]);
    if (lane == 0) sm.lpart[warp * C + c] = s;
  }
  __syncthreads();
  for (int o = t; o < d * C; o += NT) {
    const int k = o % d, c = o / d;
    T acc = T(0);
    for (int sb = 0; sb < nsub; ++sb) acc += sm.part[c * NT + sb * d + k];
    sm.G[k * C + c] = acc - sm.th[k * C + c];
  }
  if (t < C) {
    T acc = T(0), sq = T(0);
    for (int w = 0; w < C; ++w) acc += sm.lpart[w * C + t];
    for (int k = 0; k < d; ++k) sq = fma(sm.th[k * C + t], sm.th[k * C + t], sq);
    sm.lp[t] = acc - T(0.5) * sq;
  }
  __syncthreads();
}

// FSM kernel with the batched gradient: C chains per block (one per warp), every warp runs its
// chain's cheap states, the block evaluates the C gradients together, and every warp finishes
// its leapfrog step; blocks whose chains are all finished stop early.
template <typename T, int E, int C>
__device__ __forceinline__ void nuts_batched_block(const NutsView<T>& v, int64_t block, int budget,
                                                   const GradSmem<T, C>& sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int d = v.tg.d;
  const int64_t c = block * C + warp;
  const bool has_chain = c < v.m;
  Chain<T, E> s;
  if (has_chain) chain_load<T, E>(v, c, lane, s);
  else s.t = v.n;
  const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
  long long steps = 0;
  for (int b = 0; b < budget; ++b) {
    const bool act = has_chain && s.t < v.n;
    if (!__syncthreads_or(act)) break;
    Leaf<T, E> lf;
    if (act) {
      if (s.st == N_INIT) nuts_init<T, E>(v, key, lane, s);
      if (s.st == N_DOUBLE) nuts_double<T, E>(key, s);
      nuts_lf_pre<T, E>(v, s, lf);
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = lane + 32 * e;
      if (k < d) sm.th[k * C + warp] = act ? lf.xe[e] : T(0);
    }
    __syncthreads();
    block_logreg_grad<T, C>(v.tg, sm);
    if (act) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = lane + 32 * e;
        lf.ge[e] = k < d ? sm.G[k * C + warp] : T(0);
      }
      Sub<T, E> sb;
      const int r = nuts_lf_post<T, E>(v, key, c, lane, s, lf, sm.lp[warp], sb);
      ++steps;
      if (r == 1 && nuts_check<T, E>(v, key, s, sb)) continue;
      if (r != 0) nuts_done<T, E>(v, c, lane, s);
    }
  }
  if (has_chain) {
    chain_store<T, E>(v, c, lane, s);
    if (lane == 0) v.steps[c] += steps;
  }
}

// The grid is at most the blocks that can be resident at once; with more chain groups than
// blocks each block runs several groups in turn, the block times balanced (balanced_run).
template <typename T, int E, int C>
__global__ void __launch_bounds__(32 * C) nuts_fsm_batched_kernel(NutsView<T> v, int budget) {
  extern __shared__ __align__(16) unsigned char nb_smem[];
  const GradSmem<T, C> sm = grad_smem<T, C>(reinterpret_cast<T*>(nb_smem));
  const int64_t G = (v.m + C - 1) / C, P = gridDim.x;
  const int rot = G > P ? *(volatile int*)&v.sched[0] : 0;
  const BalancedRun q = balanced_run(G, P, blockIdx.x, budget);
  for (int64_t k = 0; k < q.count; ++k) nuts_batched_block<T, E, C>(v, (q.first + k + rot) % G, q.budget, sm);
  balanced_done(v.sched, G, P, rot);
}

// Fused launch over several logistic-regression NUTS jobs (serving): job k owns blocks
// off[k] .. off[k+1], so every block's chains share one design matrix.
template <typename T, int E, int C>
__global__ void __launch_bounds__(32 * C) nuts_fsm_batched_multi_kernel(const NutsView<T>* views,
                                                                        const int64_t* off, int njobs,
                                                                        int budget) {
  extern __shared__ __align__(16) unsigned char nb_smem[];
  const GradSmem<T, C> sm = grad_smem<T, C>(reinterpret_cast<T*>(nb_smem));
  const int64_t item = blockIdx.x;
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= item) lo = mid; else hi = mid - 1;
  }
  const NutsView<T> v = views[lo];
  nuts_batched_block<T, E, C>(v, item - off[lo], budget, sm);
}

// ---- synchronised kernel (Alg. 6 with nested loops) --------------------------------------------------
// Per sample: INIT and DOUBLE for all chains; then the inner loop -- one leapfrog for every
// chain still building its subtree, grid barrier, until no chain is building -- then CHECK
// for all chains whose subtree completed; repeat while any chain doubles again; then DONE.
template <typename T, int E>
__device__ void sub_store(const NutsView<T>& v, int64_t c, int lane, const Sub<T, E>& sb) {
  const size_t md = (size_t)v.m * v.tg.d;
  vstore<T, E>(v, v.sub, c, lane, sb.rho);
  vstore<T, E>(v, v.sub + md, c, lane, sb.xp);
  vstore<T, E>(v, v.sub + 2 * md, c, lane, sb.gp);
  if (lane == 0) { v.subs[c] = sb.lpp; v.subs[v.m + c] = sb.logW; }
}

template <typename T, int E>
__device__ void sub_load(const NutsView<T>& v, int64_t c, int lane, Sub<T, E>& sb) {
  const size_t md = (size_t)v.m * v.tg.d;
  vload<T, E>(v, v.sub, c, lane, sb.rho);
  vload<T, E>(v, v.sub + md, c, lane, sb.xp);
  vload<T, E>(v, v.sub + 2 * md, c, lane, sb.gp);
  sb.lpp = v.subs[c];
  sb.logW = v.subs[v.m + c];
}

template <typename T, int E>
__global__ void __launch_bounds__(256) nuts_sync_kernel(NutsView<T> v, int t_begin, int t_end,
                                                        GridBarrier bar, unsigned* active_cnt,
                                                        unsigned long long* iterations) {
  __shared__ T wsm_all[kWarpsMax][kWsm];
  __shared__ unsigned blk_active;
  const int lane = threadIdx.x & 31;
  T* wsm = wsm_all[threadIdx.x >> 5];
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  int iter = 0;
  // one grid-wide count of chains in state `want`; false on barrier timeout
  auto count_state = [&](int want, unsigned& total) -> bool {
    if (threadIdx.x == 0) blk_active = 0;
    __syncthreads();
    unsigned mine = 0;
    for (int64_t c = warp0; c < v.m; c += nwarps)
      if (v.iv[I_ST * v.m + c] == want) ++mine;
    if (lane == 0 && mine) atomicAdd(&blk_active, mine);
    __syncthreads();
    const int slot = iter % 3;
    if (threadIdx.x == 0 && blk_active) atomicAdd(&active_cnt[slot], blk_active);
    if (!grid_sync<kBarFlag>(bar, v.err)) return false;
    total = read_after_grid_sync(&active_cnt[slot]);
    if (leader) active_cnt[(iter + 2) % 3] = 0;
    ++iter;
    return true;
  };
  for (int t = t_begin; t < t_end; ++t) {
    for (int64_t c = warp0; c < v.m; c += nwarps) {
      Chain<T, E> s;
      chain_load<T, E>(v, c, lane, s);
      const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
      nuts_init<T, E>(v, key, lane, s);
      nuts_double<T, E>(key, s);
      chain_store<T, E>(v, c, lane, s);
    }
    while (true) {  // outer loop: doublings
      while (true) {  // inner loop: leapfrog steps of the current subtrees
        for (int64_t c = warp0; c < v.m; c += nwarps) {
          if (v.iv[I_ST * v.m + c] != N_INTEGRATE) continue;
          Chain<T, E> s;
          chain_load<T, E>(v, c, lane, s);
          const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
          Sub<T, E> sb;
          const int r = nuts_integrate<T, E>(v, key, c, lane, wsm, s, sb);
          if (r == 1) { sub_store<T, E>(v, c, lane, sb); s.st = N_CHECK; }
          if (r == 2) s.st = N_DONE;
          chain_store<T, E>(v, c, lane, s);
          if (lane == 0) v.steps[c] += 1;
        }
        unsigned building = 0;
        if (!count_state(N_INTEGRATE, building)) return;
        if (leader) *iterations += 1;
        if (building == 0) break;
      }
      for (int64_t c = warp0; c < v.m; c += nwarps) {
        if (v.iv[I_ST * v.m + c] != N_CHECK) continue;
        Chain<T, E> s;
        chain_load<T, E>(v, c, lane, s);
        const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
        Sub<T, E> sb;
        sub_load<T, E>(v, c, lane, sb);
        if (nuts_check<T, E>(v, key, s, sb)) nuts_double<T, E>(key, s);
        else s.st = N_DONE;
        chain_store<T, E>(v, c, lane, s);
      }
      unsigned doubling = 0;
      if (!count_state(N_INTEGRATE, doubling)) return;
      if (doubling == 0) break;
    }
    for (int64_t c = warp0; c < v.m; c += nwarps) {
      Chain<T, E> s;
      chain_load<T, E>(v, c, lane, s);
      nuts_done<T, E>(v, c, lane, s);
      chain_store<T, E>(v, c, lane, s);
    }
  }
}

// Synchronised kernel for logistic regression with the batched gradient: the program of
// nuts_sync_kernel (the same states, iterations and grid barriers), but in each leapfrog iteration
// the C warps of a block compute the gradients of their chains together (block_logreg_grad, as
// the FSM's batched kernel does), slot by slot: slot j is chain warp + j nwarps of every warp.
// A chain's gradient does not depend on which chains share its block, so the samples equal the
// FSM's bit for bit.
template <typename T, int E, int C>
__global__ void __launch_bounds__(32 * C) nuts_sync_batched_kernel(NutsView<T> v, int t_begin, int t_end,
                                                                   GridBarrier bar, unsigned* active_cnt,
                                                                   unsigned long long* iterations) {
  extern __shared__ __align__(16) unsigned char nbs_smem[];
  const GradSmem<T, C> sm = grad_smem<T, C>(reinterpret_cast<T*>(nbs_smem));
  __shared__ unsigned blk_active;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int d = v.tg.d;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t slots = (v.m + nwarps - 1) / nwarps;  // chains per warp, the same for every warp
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  int iter = 0;
  auto count_state = [&](int want, unsigned& total) -> bool {
    if (threadIdx.x == 0) blk_active = 0;
    __syncthreads();
    unsigned mine = 0;
    for (int64_t c = warp0; c < v.m; c += nwarps)
      if (v.iv[I_ST * v.m + c] == want) ++mine;
    if (lane == 0 && mine) atomicAdd(&blk_active, mine);
    __syncthreads();
    const int slot = iter % 3;
    if (threadIdx.x == 0 && blk_active) atomicAdd(&active_cnt[slot], blk_active);
    if (!grid_sync<kBarFlag>(bar, v.err)) return false;
    total = read_after_grid_sync(&active_cnt[slot]);
    if (leader) active_cnt[(iter + 2) % 3] = 0;
    ++iter;
    return true;
  };
  for (int t = t_begin; t < t_end; ++t) {
    for (int64_t c = warp0; c < v.m; c += nwarps) {
      Chain<T, E> s;
      chain_load<T, E>(v, c, lane, s);
      const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
      nuts_init<T, E>(v, key, lane, s);
      nuts_double<T, E>(key, s);
      chain_store<T, E>(v, c, lane, s);
    }
    while (true) {  // outer loop: doublings
      while (true) {  // inner loop: leapfrog steps of the current subtrees
        for (int64_t j = 0; j < slots; ++j) {
          const int64_t c = warp0 + j * nwarps;
          const bool act = c < v.m && v.iv[I_ST * v.m + c] == N_INTEGRATE;
          if (!__syncthreads_or(act)) continue;  // no chain of the block integrates in this slot
          Chain<T, E> s;
          Leaf<T, E> lf;
          if (act) {
            chain_load<T, E>(v, c, lane, s);
            nuts_lf_pre<T, E>(v, s, lf);
          }
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int k = lane + 32 * e;
            if (k < d) sm.th[k * C + warp] = act ? lf.xe[e] : T(0);
          }
          __syncthreads();
          block_logreg_grad<T, C>(v.tg, sm);
          if (act) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
              const int k = lane + 32 * e;
              lf.ge[e] = k < d ? sm.G[k * C + warp] : T(0);
            }
            const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
            Sub<T, E> sb;
            const int r = nuts_lf_post<T, E>(v, key, c, lane, s, lf, sm.lp[warp], sb);
            if (r == 1) { sub_store<T, E>(v, c, lane, sb); s.st = N_CHECK; }
            if (r == 2) s.st = N_DONE;
            chain_store<T, E>(v, c, lane, s);
            if (lane == 0) v.steps[c] += 1;
          }
        }
        unsigned building = 0;
        if (!count_state(N_INTEGRATE, building)) return;
        if (leader) *iterations += 1;
        if (building == 0) break;
      }
      for (int64_t c = warp0; c < v.m; c += nwarps) {
        if (v.iv[I_ST * v.m + c] != N_CHECK) continue;
        Chain<T, E> s;
        chain_load<T, E>(v, c, lane, s);
        const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
        Sub<T, E> sb;
        sub_load<T, E>(v, c, lane, sb);
        if (nuts_check<T, E>(v, key, s, sb)) nuts_double<T, E>(key, s);
        else s.st = N_DONE;
        chain_store<T, E>(v, c, lane, s);
      }
      unsigned doubling = 0;
      if (!count_state(N_INTEGRATE, doubling)) return;
      if (doubling == 0) break;
    }
    for (int64_t c = warp0; c < v.m; c += nwarps) {
      Chain<T, E> s;
      chain_load<T, E>(v, c, lane, s);
      nuts_done<T, E>(v, c, lane, s);
      chain_store<T, E>(v, c, lane, s);
    }
  }
}

template <typename T, int E>
__global__ void __launch_bounds__(256) nuts_init_kernel(NutsView<T> v) {
  __shared__ T wsm_all[kWarpsMax][kWsm];
  const int lane = threadIdx.x & 31;
  T* wsm = wsm_all[threadIdx.x >> 5];
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const size_t md = (size_t)v.m * v.tg.d;
  for (int64_t c = warp; c < v.m; c += nwarps) {
    T x[E], g[E];
    vload<T, E>(v, v.x, c, lane, x);
    T lp = logp_grad<T, E>(v.tg, x, g, lane, wsm);
    if (!(lp == lp)) { lp = neg_inf<T>(); if (lane == 0) atomicOr(v.err, ERR_NONFINITE); }
    vstore<T, E>(v, v.vec + V_GX * md, c, lane, g);
    if (lane == 0) v.sc[S_LPX * v.m + c] = lp;
  }
}

// ---- host side --------------------------------------------------------------------------------------------
template <typename T>
static NutsView<T> nuts_view(const fsmc_job* j) {
  NutsView<T> v{};
  char* b = j->dev;
  v.m = j->m;
  v.n = (int)j->n;
  v.chain0 = j->chain0;
  v.seed_lo = (uint32_t)j->seed;
  v.seed_hi = (uint32_t)(j->seed >> 32);
  v.x = (T*)(b + j->o_x);
  v.t = (int*)(b + j->o_t);
  v.out = j->store ? (T*)(b + j->o_out) : nullptr;
  v.mom = j->store ? nullptr : (T*)(b + j->o_mom);
  v.mom_stride = (size_t)j->m * j->d;
  v.counts = (int*)(b + j->o_counts);
  v.steps = (long long*)(b + j->o_steps);
  v.err = (int*)(b + j->o_err);
  v.chains_done = (int*)(b + j->o_done);
  if constexpr (sizeof(T) == 8) v.tg = j->tg->tv64; else v.tg = j->tg->tv32;
  v.eps = (T)j->nuts.eps;
  v.max_dH = (T)j->nuts.max_dH;
  v.max_depth = j->nuts.max_depth;
  const size_t es = sizeof(T);
  const size_t m = (size_t)j->m, d = (size_t)j->d;
  size_t o = j->o_nuts;
  auto take = [&](size_t bytes) { size_t r = o; o = (o + bytes + 255) / 256 * 256; return r; };
  v.vec = (T*)(b + take(NV * m * d * es));
  v.sc = (T*)(b + take(NSC * m * es));
  v.iv = (int*)(b + take(NI * m * 4));
  v.stk = (T*)(b + take(m * kLevels * 4 * d * es));
  v.stks = (T*)(b + take(m * kLevels * 2 * es));
  v.sub = (T*)(b + take(3 * m * d * es));
  v.subs = (T*)(b + take(2 * m * es));
  v.sched = (int*)(b + take(64));
  v.aux = (int*)(b + j->o_aux);
  return v;
}

}  // namespace fsmc

using namespace fsmc;

void nuts_layout(fsmc_job* j, size_t& off) {
  const size_t es = j->prec == FSMC_FP64 ? 8 : 4;
  const size_t m = (size_t)j->m, d = (size_t)j->d;
  auto take = [&](size_t bytes) { size_t r = off; off = (off + bytes + 255) / 256 * 256; return r; };
  j->o_aux = take(m * (size_t)j->n * 4);
  j->o_nuts = off;
  take(NV * m * d * es);
  take(NSC * m * es);
  take(NI * m * 4);
  take(m * kLevels * 4 * d * es);
  take(m * kLevels * 2 * es);
  take(3 * m * d * es);
  take(2 * m * es);
  take(64);  // batched FSM launch schedule (rotation, ticket)
  j->o_nuts_end = off;
}

#define FSMC_NUTS_DISPATCH(FN, ...)                   \
  do {                                                \
    const int d = j->d;                               \
    if (d <= 32) return FN<T, 1>(__VA_ARGS__);        \
    if (d <= 64) return FN<T, 2>(__VA_ARGS__);        \
    if (d <= 128) return FN<T, 4>(__VA_ARGS__);       \
    return cudaErrorInvalidValue;                     \
  } while (0)

template <typename T, int E>
static cudaError_t nuts_init_launch(fsmc_job* j, cudaStream_t st) {
  const NutsView<T> v = nuts_view<T>(j);
  const int threads = 128;
  const int64_t blocks = (j->m * 32 + threads - 1) / threads;
  nuts_init_kernel<T, E><<<(unsigned)blocks, threads, 0, st>>>(v);
  return cudaGetLastError();
}

template <typename T, int E>
static cudaError_t nuts_fsm_launch(fsmc_job* j, cudaStream_t st) {
  const NutsView<T> v = nuts_view<T>(j);
  if (j->tg->kind == FSMC_TGT_LOGREG && j->tun.lanes_per_chain == 32) {
    constexpr int C = kBatchChains;
    auto kern = nuts_fsm_batched_kernel<T, E, C>;
    const size_t smem = grad_smem_bytes<T, C>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * C, smem);
    if (e != cudaSuccess) return e;
    // at most the resident blocks; more groups than that are balanced over them
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((j->m + C - 1) / C, (int64_t)per_sm * j->e->sms));
    kern<<<(unsigned)blocks, 32 * C, smem, st>>>(v, j->tun.steps_per_launch);
    return cudaGetLastError();
  }
  const int threads = j->tun.threads_per_block;
  const int64_t blocks = (j->m * 32 + threads - 1) / threads;
  nuts_fsm_kernel<T, E><<<(unsigned)blocks, threads, 0, st>>>(v, j->tun.steps_per_launch);
  return cudaGetLastError();
}

template <typename T, int E>
static cudaError_t nuts_sync_launch(fsmc_job* j, int t0, int t1, GridBarrier bar, unsigned* active,
                                    unsigned long long* iters, cudaStream_t st) {
  NutsView<T> v = nuts_view<T>(j);
  if (j->tg->kind == FSMC_TGT_LOGREG && j->tun.lanes_per_chain == 32) {  // the batched gradient
    constexpr int C = kBatchChains;
    auto kern = nuts_sync_batched_kernel<T, E, C>;
    const size_t smem = grad_smem_bytes<T, C>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * C, smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = std::min<int64_t>((int64_t)per_sm * j->e->sms, (j->m + C - 1) / C);
    if (blocks < 1) blocks = 1;
    void* args[] = {(void*)&v, (void*)&t0, (void*)&t1, (void*)&bar, (void*)&active, (void*)&iters};
    return cudaLaunchCooperativeKernel((void*)kern, dim3((unsigned)blocks), dim3(32 * C), args, smem, st);
  }
  auto kern = nuts_sync_kernel<T, E>;
  const int threads = j->tun.threads_per_block;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
  if (e != cudaSuccess) return e;
  int64_t blocks = std::min<int64_t>((int64_t)per_sm * j->e->sms, (j->m * 32 + threads - 1) / threads);
  if (blocks < 1) blocks = 1;
  void* args[] = {(void*)&v, (void*)&t0, (void*)&t1, (void*)&bar, (void*)&active, (void*)&iters};
  return cudaLaunchCooperativeKernel((void*)kern, dim3((unsigned)blocks), dim3(threads), args, 0, st);
}

template <typename T>
static cudaError_t nuts_init_t(fsmc_job* j, cudaStream_t st) { FSMC_NUTS_DISPATCH(nuts_init_launch, j, st); }
template <typename T>
static cudaError_t nuts_fsm_t(fsmc_job* j, cudaStream_t st) { FSMC_NUTS_DISPATCH(nuts_fsm_launch, j, st); }
template <typename T>
static cudaError_t nuts_sync_t(fsmc_job* j, int t0, int t1, GridBarrier bar, unsigned* active,
                               unsigned long long* iters, cudaStream_t st) {
  FSMC_NUTS_DISPATCH(nuts_sync_launch, j, t0, t1, bar, active, iters, st);
}

fsmc_status nuts_init_state(fsmc_job* j, cudaStream_t st) {
  if (j->d > 128) return fsmc_fail(FSMC_EINVAL, "NUTS supports d <= 128");
  char* b = j->dev;
  const size_t m = (size_t)j->m;
  // the NUTS state block starts zeroed (state INIT = 0)
  cudaError_t e = cudaMemsetAsync(b + j->o_nuts, 0, j->o_nuts_end - j->o_nuts, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b + j->o_aux, 0, m * (size_t)j->n * 4, st);
  if (e == cudaSuccess) e = j->prec == FSMC_FP64 ? nuts_init_t<double>(j, st) : nuts_init_t<float>(j, st);
  if (e != cudaSuccess) return fsmc_cuda_fail(e, "NUTS init");
  return FSMC_OK;
}

cudaError_t nuts_fsm_round(fsmc_job* j, cudaStream_t st) {
  return j->prec == FSMC_FP64 ? nuts_fsm_t<double>(j, st) : nuts_fsm_t<float>(j, st);
}

int nuts_group_E(int d) { return d <= 32 ? 1 : d <= 64 ? 2 : 4; }

// One fused FSM launch over jobs that share precision and E (serving scheduler).
template <typename T, int E>
static cudaError_t nuts_multi_launch_t(const std::vector<fsmc_job*>& jobs, MultiBuf& b, cudaStream_t st) {
  const int nj = (int)jobs.size();
  const size_t vb = sizeof(NutsView<T>);
  const size_t views_bytes = (nj * vb + 15) / 16 * 16;
  char* hs = (char*)b.h_stage;
  int64_t* hoff = (int64_t*)(hs + views_bytes);
  hoff[0] = 0;
  for (int k = 0; k < nj; ++k) {
    const NutsView<T> v = nuts_view<T>(jobs[k]);
    std::memcpy(hs + k * vb, &v, vb);
    hoff[k + 1] = hoff[k] + jobs[k]->m;
  }
  const bool batched = jobs[0]->tg->kind == FSMC_TGT_LOGREG && jobs[0]->tun.lanes_per_chain == 32;
  if (batched) {  // offsets in blocks of kBatchChains chains, as the single-job launch uses
    hoff[0] = 0;
    for (int k = 0; k < nj; ++k) hoff[k + 1] = hoff[k] + (jobs[k]->m + kBatchChains - 1) / kBatchChains;
  }
  const size_t bytes = views_bytes + (nj + 1) * sizeof(int64_t);
  cudaError_t e = cudaMemcpyAsync(b.d_buf, hs, bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  const NutsView<T>* dv = (const NutsView<T>*)b.d_buf;
  const int64_t* doff = (const int64_t*)((char*)b.d_buf + views_bytes);
  if (batched) {
    constexpr int C = kBatchChains;
    auto kern = nuts_fsm_batched_multi_kernel<T, E, C>;
    const size_t smem = grad_smem_bytes<T, C>();
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)hoff[nj], 32 * C, smem, st>>>(dv, doff, nj, jobs[0]->tun.steps_per_launch);
    return cudaGetLastError();
  }
  const int threads = 128;
  const int64_t total = hoff[nj];
  const int64_t blocks = (total * 32 + threads - 1) / threads;
  nuts_fsm_multi_kernel<T, E><<<(unsigned)blocks, threads, 0, st>>>(dv, doff, nj, total,
                                                                    jobs[0]->tun.steps_per_launch);
  return cudaGetLastError();
}

cudaError_t nuts_group_round(const std::vector<fsmc_job*>& jobs, MultiBuf& b, cudaStream_t st) {
  if (jobs.empty()) return cudaSuccess;
  const bool f64 = jobs[0]->prec == FSMC_FP64;
  const int E = nuts_group_E(jobs[0]->d);
  if (f64) {
    if (E == 1) return nuts_multi_launch_t<double, 1>(jobs, b, st);
    if (E == 2) return nuts_multi_launch_t<double, 2>(jobs, b, st);
    return nuts_multi_launch_t<double, 4>(jobs, b, st);
  }
  if (E == 1) return nuts_multi_launch_t<float, 1>(jobs, b, st);
  if (E == 2) return nuts_multi_launch_t<float, 2>(jobs, b, st);
  return nuts_multi_launch_t<float, 4>(jobs, b, st);
}

fsmc_status nuts_run_sync(fsmc_job* j, cudaStream_t st) {
  char* b = j->dev;
  GridBarrier bar = job_grid_barrier(j);
  unsigned* active = (unsigned*)(b + j->o_bar) + 4;
  unsigned long long* iters = (unsigned long long*)(b + j->o_iters);
  const int chunk = 100;
  for (int64_t t0 = 0; t0 < j->n; t0 += chunk) {
    const int t1 = (int)std::min<int64_t>(t0 + chunk, j->n);
    cudaError_t e = clear_sync_counters(j, st);
    if (e == cudaSuccess) {
      ProfScope p(j, 2, st);
      e = j->prec == FSMC_FP64 ? nuts_sync_t<double>(j, (int)t0, t1, bar, active, iters, st)
                               : nuts_sync_t<float>(j, (int)t0, t1, bar, active, iters, st);
    }
    if (e != cudaSuccess) return fsmc_cuda_fail(e, "NUTS synchronised launch");
    j->launches += 1;
  }
  return FSMC_OK;
}
