// Delayed-rejection Metropolis-Hastings with up to three stages as a finite state machine.
//
// Fig. 2 ("Delayed Rejection MH") has INIT, PROPOSE (the loop body) and DONE; INIT and
// DONE are nearly empty, so the FSM is condensed to the single PROPOSE state (Sec. 7.1,
// "FSM-condensed"): one step proposes the next stage's y_k ~ N(x, sigma_k^2 I), evaluates
// log pi(y_k) (the amortised g), and either accepts, rejects for good after the last
// stage, or keeps y_k for the next stage's acceptance ratio.  A sample takes exactly as
// many steps as stages were tried.
//
// Acceptance is the general (Tierney-Mira) delayed-rejection rule for proposals centred
// at the current point, in log space:
//   a1(x, y1)         = min(0, lp(y1) - lp(x))
//   a2(x, y1, y2)     = min(0, [lp(y2) + lq1(y2->y1) + l1m(a1(y2,y1))] - [lp(x) + lq1(x->y1) + l1m(a1(x,y1))])
//   a3(x, y1, y2, y3) = min(0, [lp(y3) + lq1(y3->y2) + lq2(y3->y1) + l1m(a1(y3,y2)) + l1m(a2(y3,y2,y1))]
//                             - [lp(x) + lq1(x->y1) + lq2(x->y2) + l1m(a1(x,y1)) + l1m(a2(x,y1,y2))])
// with lq_s(a->b) = -|b-a|^2 / (2 sigma_s^2) and l1m(a) = log(1 - e^a).
#include <algorithm>
#include "fsmc_device.cuh"
#include "fsmc_kernels.h"
#include "target_logp.cuh"

namespace fsmc {

// log(1 - e^a), a < 0.  Single precision takes log(-expm1(a)) for every a: for a << 0 the
// argument rounds near 1 and the result keeps an absolute error of ~1e-7, which is what matters
// where it is added to the other log terms, and one branch-free form keeps a warp's chains on
// one path whatever their values.
template <typename T>
__device__ __forceinline__ T l1m(T a) {
  if (!(a < T(0))) return neg_inf<T>();
  if constexpr (sizeof(T) == 4)
    return logf(-expm1f(a));
  else
    return a > -0.6931471805599453 ? log(-expm1(a)) : log1p(-exp(a));
}

// alpha_1 = min(1, pi(prop) / pi(cur)), and 0 for a proposal of zero density even when the current
// state has zero density too (0 / 0: a proposal outside the support is never accepted)
template <typename T>
__device__ __forceinline__ T la1(T lp_cur, T lp_prop) {
  return lp_prop == neg_inf<T>() ? neg_inf<T>() : fmin(T(0), lp_prop - lp_cur);
}

template <typename T, int E>
__device__ __forceinline__ T sqdist(const T (&a)[E], const T (&b)[E], int d) {
  T acc = T(0);
#pragma unroll
  for (int e = 0; e < E; ++e)
    if (e < d) { const T r = b[e] - a[e]; acc = fma(r, r, acc); }
  return acc;
}

template <typename T, int E>
__device__ __forceinline__ void dr_emit(const DrView<T>& v, int64_t c, int t, const T (&x)[E],
                                        const MomSmem<T, E>& ms = MomSmem<T, E>{nullptr}) {
  chain_emit<T, E>(v, v.tg.d, c, t, x, ms);
}

// The PROPOSE body of stage k in four parts: draw y_k ~ N(x, sigma_k^2 I); evaluate log pi(y_k);
// the stage's acceptance ratio; the decision.  dr_step runs all four in one FSM step.
template <typename T, int E>
__device__ __forceinline__ void dr_draw(const DrView<T>& v, const Key& key, int t, int k, const T (&x)[E],
                                        T (&y)[E]) {
  const int d = v.tg.d;
  const int D = (d + 3) / 4;  // Philox blocks per stage (four normals each)
  const uint32_t base = (uint32_t)(k * (D + 1));
  const T sg = v.symmetric ? v.sig[0] : v.sig[k];
#pragma unroll
  for (int q = 0; q < (E + 3) / 4; ++q) {
    T z[4] = {T(0), T(0), T(0), T(0)};
    if (q < D) Conv<T>::normal_quad(key.block((uint32_t)t, 0, base + q), z);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (4 * q + i < E) y[4 * q + i] = q < D ? fma(sg, z[i], x[4 * q + i]) : T(0);
  }
}

template <typename T, int E>
__device__ __forceinline__ T dr_eval(const DrView<T>& v, const T (&y)[E], int& err) {
  T lpy = full_logp<T, E>(v.tg, y);
  if (!(lpy == lpy)) { lpy = neg_inf<T>(); err |= ERR_NONFINITE; }
  return lpy;
}

// The terms of a sample's later-stage ratios that do not involve the new proposal, kept from the
// stage where they first appear: after stage 1 rejects, l1m(a1(x, y1)); after stage 2 rejects,
// the stage-2 ratio's l1m(a2(x, y1, y2)), l1m(a1(y1, y2)) and the proposal-density terms between
// x, y1 and y2.  Stage 3 then evaluates two l1m instead of eight (and stage 2 one instead of
// two), on the values the full stage-2 and stage-3 ratios would recompute.
template <typename T>
struct DrCache {
  T a1;       // l1m(a1(x, y1))
  T q1xy1;    // lq1(x -> y1)
  T q1y1y2;   // lq1(y1 -> y2)
  T a2;       // l1m(a2(x, y1, y2))
  T a1y1y2;   // l1m(a1(y1, y2))
  T q2xy2;    // lq2(x -> y2)
};

// Explicitly rounded add and multiply: the ratio terms below are written with them (and fma) so
// that the per-stage form (dr_ratio, dr_decide: the synchronised kernel, whose iterations are
// stage-uniform, and the four-state ablation) and the all-stages form of the FSM step
// (dr_ratio_all, dr_decide_all) round every operation alike whatever the compiler would contract.
template <typename T>
__device__ __forceinline__ T add_rn(T a, T b) {
  if constexpr (sizeof(T) == 4) return __fadd_rn(a, b); else return __dadd_rn(a, b);
}
template <typename T>
__device__ __forceinline__ T mul_rn(T a, T b) {
  if constexpr (sizeof(T) == 4) return __fmul_rn(a, b); else return __dmul_rn(a, b);
}
template <typename T>
__device__ __forceinline__ T clip_ratio(T num, T den) {
  return (num == neg_inf<T>() || den == neg_inf<T>()) ? neg_inf<T>() : fmin(T(0), num - den);
}

template <typename T, int E>
__device__ __forceinline__ T dr_ratio(const DrView<T>& v, int k, const T (&x)[E], T lp, const T (&y1)[E], T lp1,
                                      const T (&y2)[E], T lp2, const T (&y)[E], T lpy, const DrCache<T>& cc) {
  const int d = v.tg.d;
  if (k == 0) return la1(lp, lpy);
  const T i1 = T(-0.5) / (v.sig[0] * v.sig[0]);
  if (k == 1) {  // log alpha_2(x, y1, y) with its l1m(a1(x, y1)) kept
    const T num = add_rn(add_rn(lpy, mul_rn(i1, sqdist(y, y1, d))), l1m(la1(lpy, lp1)));
    const T den = add_rn(add_rn(lp, mul_rn(i1, sqdist(x, y1, d))), cc.a1);
    return clip_ratio(num, den);
  }
  // log alpha_3(x, y1, y2, y) with the terms of x, y1, y2 kept
  const T i2 = T(-0.5) / (v.sig[1] * v.sig[1]);
  const T q1_y3_y2 = mul_rn(i1, sqdist(y, y2, d));
  const T a1_32 = l1m(la1(lpy, lp2));
  const T n2 = add_rn(add_rn(lp1, cc.q1y1y2), cc.a1y1y2);  // log alpha_2(y, y2, y1): numerator
  const T d2 = add_rn(add_rn(lpy, q1_y3_y2), a1_32);
  const T num = add_rn(add_rn(add_rn(add_rn(lpy, q1_y3_y2), mul_rn(i2, sqdist(y, y1, d))), a1_32),
                       l1m(clip_ratio(n2, d2)));
  const T den = add_rn(add_rn(add_rn(add_rn(lp, cc.q1xy1), cc.q2xy2), cc.a1), cc.a2);
  return clip_ratio(num, den);
}

// dr_ratio for every stage in one instruction stream (same bits): a warp's chains sit at
// different stages, so the terms of stages 2 and 3 are computed by every thread and selected;
// stage 3 pairs the new proposal with y2 where stage 2 pairs it with y1.
template <typename T, int E>
__device__ __forceinline__ T dr_ratio_all(const DrView<T>& v, int k, const T (&x)[E], T lp, const T (&y1)[E],
                                          T lp1, const T (&y2)[E], T lp2, const T (&y)[E], T lpy,
                                          const DrCache<T>& cc) {
  const int d = v.tg.d;
  const T r1 = la1(lp, lpy);
  if (v.n_stages < 2) return r1;
  const bool k2 = k >= 2;
  const T i1 = T(-0.5) / (v.sig[0] * v.sig[0]);
  T a[E];
#pragma unroll
  for (int e = 0; e < E; ++e) a[e] = k2 ? y2[e] : y1[e];
  const T q1_ya = mul_rn(i1, sqdist(y, a, d));  // stage 2: lq1(y -> y1); stage 3: lq1(y -> y2)
  const T a1_ya = l1m(la1(lpy, k2 ? lp2 : lp1));
  T num = add_rn(lpy, q1_ya);
  T den = add_rn(lp, k2 ? cc.q1xy1 : mul_rn(i1, sqdist(x, y1, d)));
  if (v.n_stages > 2) {  // stage-uniform for the launch
    const T i2 = T(-0.5) / (v.sig[1] * v.sig[1]);
    const T n2 = add_rn(add_rn(lp1, cc.q1y1y2), cc.a1y1y2);
    const T d2 = add_rn(add_rn(lpy, q1_ya), a1_ya);
    const T a2_321 = l1m(clip_ratio(n2, d2));
    const T num3 = add_rn(add_rn(add_rn(num, mul_rn(i2, sqdist(y, y1, d))), a1_ya), a2_321);
    const T den3 = add_rn(add_rn(add_rn(den, cc.q2xy2), cc.a1), cc.a2);
    num = k2 ? num3 : add_rn(num, a1_ya);
    den = k2 ? den3 : add_rn(den, cc.a1);
  } else {
    num = add_rn(num, a1_ya);
    den = add_rn(den, cc.a1);
  }
  return k == 0 ? r1 : clip_ratio(num, den);
}

// Returns true when the sample is finished (accepted, or rejected at the last stage); then x/lp
// hold the sample.  Otherwise y becomes y1 (stage 0) or y2 (stage 1).
template <typename T, int E>
__device__ __forceinline__ bool dr_decide(const DrView<T>& v, const Key& key, int t, int k, T la, T (&x)[E],
                                          T& lp, T (&y1)[E], T& lp1, T (&y2)[E], T& lp2, const T (&y)[E], T lpy,
                                          DrCache<T>& cc) {
  const int D = (v.tg.d + 3) / 4;
  const P4 r = key.block((uint32_t)t, 0, (uint32_t)(k * (D + 1) + D));
  if (Conv<T>::log_u(r.w0, r.w1) < la) {
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = y[e];
    lp = lpy;
    return true;
  }
  if (k + 1 >= v.n_stages) return true;
  const int d = v.tg.d;
  if (k == 0) {
#pragma unroll
    for (int e = 0; e < E; ++e) y1[e] = y[e];
    lp1 = lpy;
    cc.a1 = l1m(la);
  } else {
    const T i1 = T(-0.5) / (v.sig[0] * v.sig[0]), i2 = T(-0.5) / (v.sig[1] * v.sig[1]);
    cc.q1xy1 = mul_rn(i1, sqdist(x, y1, d));
    cc.q1y1y2 = mul_rn(i1, sqdist(y, y1, d));
    cc.a2 = l1m(la);
    cc.a1y1y2 = l1m(la1(lp1, lpy));
    cc.q2xy2 = mul_rn(i2, sqdist(x, y, d));
#pragma unroll
    for (int e = 0; e < E; ++e) y2[e] = y[e];
    lp2 = lpy;
  }
  return false;
}

// dr_decide for every stage in one instruction stream (same bits): the terms a stage-2 rejection
// keeps are computed by every rejecting thread and selected, l1m of the ratio is taken once
// (stage 1 keeps it as a1, stage 2 as a2).
template <typename T, int E>
__device__ __forceinline__ bool dr_decide_all(const DrView<T>& v, const Key& key, int t, int k, T la, T (&x)[E],
                                              T& lp, T (&y1)[E], T& lp1, T (&y2)[E], T& lp2, const T (&y)[E],
                                              T lpy, DrCache<T>& cc) {
  const int D = (v.tg.d + 3) / 4;
  const P4 r = key.block((uint32_t)t, 0, (uint32_t)(k * (D + 1) + D));
  if (Conv<T>::log_u(r.w0, r.w1) < la) {
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = y[e];
    lp = lpy;
    return true;
  }
  if (k + 1 >= v.n_stages) return true;
  const int d = v.tg.d;
  const bool k1 = k == 1;
  const T l1m_la = l1m(la);
  if (v.n_stages > 2) {  // stage-uniform for the launch: a stage-2 rejection is possible
    const T i1 = T(-0.5) / (v.sig[0] * v.sig[0]), i2 = T(-0.5) / (v.sig[1] * v.sig[1]);
    const T q1xy1 = mul_rn(i1, sqdist(x, y1, d));
    const T q1y1y2 = mul_rn(i1, sqdist(y, y1, d));
    const T a1y1y2 = l1m(la1(lp1, lpy));
    const T q2xy2 = mul_rn(i2, sqdist(x, y, d));
    if (k1) {
      cc.q1xy1 = q1xy1; cc.q1y1y2 = q1y1y2; cc.a1y1y2 = a1y1y2; cc.q2xy2 = q2xy2;
    }
  }
  cc.a1 = k1 ? cc.a1 : l1m_la;
  cc.a2 = k1 ? l1m_la : cc.a2;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    y1[e] = k1 ? y1[e] : y[e];
    y2[e] = k1 ? y[e] : y2[e];
  }
  lp1 = k1 ? lp1 : lpy;
  lp2 = k1 ? lpy : lp2;
  return false;
}

// Symmetric delayed rejection (Mira 2001), try k: y ~ N(centre, sig[0]^2 I) with the centre the
// last rejected point (x for the first try), accepted with
//   alpha_k = min(1, (pi(y) - pi*)+ / (pi(x) - pi*)),
// pi* the largest target value among the rejected tries (the rejection factors of a re-centred
// symmetric proposal telescope to pi(x) - pi*).  centre and lp_star are kept in y1 and lp1.
// Same random numbers as the staged sampler: try k's normals from draws k(D+1) + q, its uniform
// from draw k(D+1) + D.
template <typename T>
__device__ __forceinline__ T sdr_log_alpha(T lp_x, T lp_star, T lp_y) {
  if (!(lp_y > lp_star)) return neg_inf<T>();
  const T num = lp_y + l1m(lp_star - lp_y);
  const T den = lp_x + l1m(lp_star - lp_x);
  if (den == neg_inf<T>()) return T(0);
  return fmin(T(0), num - den);
}

template <typename T, int E>
__device__ __forceinline__ void sdr_begin(const T (&x)[E], T (&centre)[E], T& lp_star) {
#pragma unroll
  for (int e = 0; e < E; ++e) centre[e] = x[e];
  lp_star = neg_inf<T>();
}

// Try k's decision; true when the sample is finished (accepted, or the M-th try rejected).
template <typename T, int E>
__device__ __forceinline__ bool sdr_decide(const DrView<T>& v, const Key& key, int t, int k, T la, T (&x)[E],
                                           T& lp, T (&centre)[E], T& lp_star, const T (&y)[E], T lpy) {
  const int D = (v.tg.d + 3) / 4;
  const P4 r = key.block((uint32_t)t, 0, (uint32_t)(k * (D + 1) + D));
  if (Conv<T>::log_u(r.w0, r.w1) < la) {
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = y[e];
    lp = lpy;
    return true;
  }
  lp_star = fmax(lp_star, lpy);
#pragma unroll
  for (int e = 0; e < E; ++e) centre[e] = y[e];
  return k + 1 >= v.n_stages;
}

template <typename T, int E>
__device__ __forceinline__ bool sdr_step(const DrView<T>& v, const Key& key, int t, int k, T (&x)[E], T& lp,
                                         T (&centre)[E], T& lp_star, int& err) {
  if (k == 0) sdr_begin<T, E>(x, centre, lp_star);  // a new sample: the first try is centred at x
  T y[E];
  dr_draw<T, E>(v, key, t, k, centre, y);
  const T lpy = dr_eval<T, E>(v, y, err);
  return sdr_decide<T, E>(v, key, t, k, sdr_log_alpha<T>(lp, lp_star, lpy), x, lp, centre, lp_star, y, lpy);
}

// One PROPOSE step of stage k for one chain (all four parts); the symmetric sampler's try k.
// ALL: the stage-dependent parts in one instruction stream (the FSM step, whose warps hold chains
// at every stage); otherwise per stage (the synchronised kernel, stage-uniform).  Same bits.
template <typename T, int E, bool ALL = false>
__device__ __forceinline__ bool dr_step(const DrView<T>& v, const Key& key, int t, int k, T (&x)[E],
                                        T& lp, T (&y1)[E], T& lp1, T (&y2)[E], T& lp2, DrCache<T>& cc, int& err) {
  if (v.symmetric) return sdr_step<T, E>(v, key, t, k, x, lp, y1, lp1, err);
  T y[E];
  dr_draw<T, E>(v, key, t, k, x, y);
  const T lpy = dr_eval<T, E>(v, y, err);
  if constexpr (ALL) {
    const T la = dr_ratio_all<T, E>(v, k, x, lp, y1, lp1, y2, lp2, y, lpy, cc);
    return dr_decide_all<T, E>(v, key, t, k, la, x, lp, y1, lp1, y2, lp2, y, lpy, cc);
  } else {
    const T la = dr_ratio<T, E>(v, k, x, lp, y1, lp1, y2, lp2, y, lpy, cc);
    return dr_decide<T, E>(v, key, t, k, la, x, lp, y1, lp1, y2, lp2, y, lpy, cc);
  }
}

// The kept terms live in lpy[4 + i][m] between launches (and between synchronised iterations).
template <typename T>
__device__ __forceinline__ DrCache<T> dr_cache_load(const DrView<T>& v, int64_t c) {
  const T* q = v.lpy + 4 * v.m + c;
  return DrCache<T>{q[0], q[v.m], q[2 * v.m], q[3 * v.m], q[4 * v.m], q[5 * v.m]};
}

template <typename T>
__device__ __forceinline__ void dr_cache_store(const DrView<T>& v, int64_t c, const DrCache<T>& cc) {
  T* q = v.lpy + 4 * v.m + c;
  q[0] = cc.a1; q[v.m] = cc.q1xy1; q[2 * v.m] = cc.q1y1y2; q[3 * v.m] = cc.a2; q[4 * v.m] = cc.a1y1y2;
  q[5 * v.m] = cc.q2xy2;
}

template <typename T, int E>
__device__ __forceinline__ void dr_load(const DrView<T>& v, int64_t c, T (&x)[E], T (&y1)[E],
                                        T (&y2)[E]) {
  const int d = v.tg.d;
  const size_t md = (size_t)v.m * d;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    x[e] = e < d ? v.x[(size_t)c * d + e] : T(0);
    y1[e] = e < d ? v.y[(size_t)c * d + e] : T(0);
    y2[e] = e < d ? v.y[md + (size_t)c * d + e] : T(0);
  }
}

template <typename T, int E>
__device__ __forceinline__ void dr_store(const DrView<T>& v, int64_t c, const T (&x)[E],
                                         const T (&y1)[E], const T (&y2)[E], int k) {
  const int d = v.tg.d;
  const size_t md = (size_t)v.m * d;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (e >= d) continue;
    v.x[(size_t)c * d + e] = x[e];
    if (k >= 1) v.y[(size_t)c * d + e] = y1[e];
    if (k >= 2) v.y[md + (size_t)c * d + e] = y2[e];
  }
}

// FSM kernel: chain-per-thread, every chain advances `budget` FSM steps.
// CONDENSED (Sec. 7.1): the single PROPOSE state, with INIT and DONE run inline -- a sample takes
// as many steps as stages tried; k is the next stage.  !CONDENSED (the paper's ablation, Sec. 7.1):
// the PROPOSE body unrolled into four states run one per step -- draw, evaluate, ratio, decide
// (k = 4 j + u for stage (try) j, part u) -- with the proposal, its log density and the ratio kept
// in the chain state between steps; a warp whose chains are in different parts runs each part's
// code.  Both forms compute the same samples, for the staged and the symmetric sampler (whose
// centre and pi* are y1 and lp1).

// MOMC: a moments-only job whose chains keep their running sums in dynamic shared memory
// during the launch (MomSmem); the other instantiations update device memory per sample.
template <typename T, int E, bool CONDENSED, bool MOMC = false>
__global__ void __launch_bounds__(256) dr_fsm_kernel(DrView<T> v, int budget) {
  extern __shared__ __align__(16) unsigned char dr_mom_smem[];
  const MomSmem<T, E> ms{MOMC ? reinterpret_cast<T*>(dr_mom_smem) + (size_t)threadIdx.x * MomSmem<T, E>::kSlot : nullptr};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < v.m; c += stride) {
    if constexpr (MOMC) mom_smem_load<T, E>(v, v.tg.d, c, ms);
    T x[E], y1[E], y2[E];
    dr_load<T, E>(v, c, x, y1, y2);
    T lp = v.lp[c], lp1 = v.lpy[c], lp2 = v.lpy[v.m + c];
    DrCache<T> cc = dr_cache_load<T>(v, c);
    int t = v.t[c], k = v.k[c];
    const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
    int err = 0, steps = 0;
    // !CONDENSED: the current stage's proposal, log density and ratio between parts
    T yc[E], lpc = T(0), lac = T(0);
    const size_t md = (size_t)v.m * v.tg.d;
    if constexpr (!CONDENSED) {
#pragma unroll
      for (int e = 0; e < E; ++e) yc[e] = e < v.tg.d ? v.y[2 * md + (size_t)c * v.tg.d + e] : T(0);
      lpc = v.lpy[2 * v.m + c];
      lac = v.lpy[3 * v.m + c];
    }
    for (int b = 0; b < budget && t < v.n; ++b) {
      ++steps;
      if constexpr (CONDENSED) {
        if (dr_step<T, E, true>(v, key, t, k, x, lp, y1, lp1, y2, lp2, cc, err)) {
          dr_emit<T, E>(v, c, t, x, ms);
          v.counts[(size_t)c * v.n + t] = k + 1;
          ++t;
          k = 0;
          if (t == v.n) atomicAdd(v.chains_done, 1);
        } else {
          ++k;
        }
      } else {
        const int j = k >> 2, u = k & 3;
        if (u == 0) {
          if (v.symmetric && j == 0) sdr_begin<T, E>(x, y1, lp1);
          dr_draw<T, E>(v, key, t, j, v.symmetric ? y1 : x, yc);
          ++k;
        } else if (u == 1) {
          lpc = dr_eval<T, E>(v, yc, err);
          ++k;
        } else if (u == 2) {
          lac = v.symmetric ? sdr_log_alpha<T>(lp, lp1, lpc)
                            : dr_ratio<T, E>(v, j, x, lp, y1, lp1, y2, lp2, yc, lpc, cc);
          ++k;
        } else if (v.symmetric ? sdr_decide<T, E>(v, key, t, j, lac, x, lp, y1, lp1, yc, lpc)
                               : dr_decide<T, E>(v, key, t, j, lac, x, lp, y1, lp1, y2, lp2, yc, lpc, cc)) {
          dr_emit<T, E>(v, c, t, x, ms);
          v.counts[(size_t)c * v.n + t] = j + 1;
          ++t;
          k = 0;
          if (t == v.n) atomicAdd(v.chains_done, 1);
        } else {
          k = 4 * (j + 1);
        }
      }
    }
    if constexpr (!CONDENSED) {
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (e < v.tg.d) v.y[2 * md + (size_t)c * v.tg.d + e] = yc[e];
      v.lpy[2 * v.m + c] = lpc;
      v.lpy[3 * v.m + c] = lac;
    }
    // y1 / y2 are live while stages 2 / 3 are pending
    const int pending = CONDENSED ? k : (k >> 2);
    dr_store<T, E>(v, c, x, y1, y2, pending);
    v.lp[c] = lp; v.lpy[c] = lp1; v.lpy[v.m + c] = lp2;
    if (pending) dr_cache_store<T>(v, c, cc);
    v.t[c] = t; v.k[c] = k;
    v.steps[c] += steps;
    if (err) atomicOr(v.err, err);
    if constexpr (MOMC) mom_smem_store<T, E>(v, v.tg.d, c, ms);
  }
}

// Synchronised kernel (Alg. 6): for every sample, stage 1 for all chains, then stage 2 for
// the chains that rejected, ..., with a grid barrier between stages.
template <typename T, int E>
__global__ void __launch_bounds__(256) dr_sync_kernel(DrView<T> v, int t_begin, int t_end,
                                                      GridBarrier bar, unsigned* active_cnt,
                                                      unsigned long long* iterations) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t c_first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  __shared__ unsigned blk_active;
  int iter = 0, err = 0;
  if (stride >= v.m) {
    // At most one chain per thread (the grid is sized to cover the job when it fits): the chain's
    // state stays in the thread's registers for the whole launch -- loaded once, stored once --
    // instead of a load and a store around every stage; same steps in the same order.
    const int64_t c = c_first;
    const bool has = c < v.m;
    T x[E], y1[E], y2[E];
    T lp = T(0), lp1 = T(0), lp2 = T(0);
    DrCache<T> cc{};
    if (has) {
      dr_load<T, E>(v, c, x, y1, y2);
      lp = v.lp[c]; lp1 = v.lpy[c]; lp2 = v.lpy[v.m + c];
      cc = dr_cache_load<T>(v, c);
    }
    const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
    long long steps = 0;
    for (int t = t_begin; t < t_end; ++t) {
      int kc = 0;  // next stage of this chain's sample t
      for (int k = 0; k < v.n_stages; ++k) {
        if (threadIdx.x == 0) blk_active = 0;
        __syncthreads();
        unsigned mine = 0;
        if (has && kc == k) {
          ++steps;
          if (dr_step<T, E>(v, key, t, k, x, lp, y1, lp1, y2, lp2, cc, err)) {
            dr_emit<T, E>(v, c, t, x);
            v.counts[(size_t)c * v.n + t] = k + 1;
            kc = v.n_stages;
            if (t + 1 == v.n) atomicAdd(v.chains_done, 1);
          } else {
            kc = k + 1;
            mine = 1;
          }
        }
        if (mine) atomicAdd(&blk_active, 1u);
        __syncthreads();
        const int slot = iter % 3;
        if (threadIdx.x == 0 && blk_active) atomicAdd(&active_cnt[slot], blk_active);
        if (!grid_sync(bar, v.err)) return;
        const unsigned total = read_after_grid_sync(&active_cnt[slot]);
        if (leader) {
          active_cnt[(iter + 2) % 3] = 0;
          *iterations += 1;
        }
        ++iter;
        if (total == 0) break;
      }
    }
    if (has) {
      dr_store<T, E>(v, c, x, y1, y2, 0);
      v.lp[c] = lp;
      v.t[c] = t_end;
      v.k[c] = 0;
      v.steps[c] += steps;
    }
    if (err) atomicOr(v.err, err);
    return;
  }
  for (int t = t_begin; t < t_end; ++t) {
    for (int k = 0; k < v.n_stages; ++k) {
      if (threadIdx.x == 0) blk_active = 0;
      __syncthreads();
      unsigned mine = 0;
      for (int64_t c = c_first; c < v.m; c += stride) {
        if (v.k[c] != k) continue;  // masked: finished this sample at an earlier stage
        T x[E], y1[E], y2[E];
        dr_load<T, E>(v, c, x, y1, y2);
        T lp = v.lp[c], lp1 = v.lpy[c], lp2 = v.lpy[v.m + c];
        DrCache<T> cc = dr_cache_load<T>(v, c);
        const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
        v.steps[c] += 1;
        if (dr_step<T, E>(v, key, t, k, x, lp, y1, lp1, y2, lp2, cc, err)) {
          dr_emit<T, E>(v, c, t, x);
          v.counts[(size_t)c * v.n + t] = k + 1;
          dr_store<T, E>(v, c, x, y1, y2, 0);
          v.lp[c] = lp;
          v.k[c] = v.n_stages;  // done with sample t
          v.t[c] = t + 1;
          if (t + 1 == v.n) atomicAdd(v.chains_done, 1);
        } else {
          dr_store<T, E>(v, c, x, y1, y2, k + 1);
          v.lpy[c] = lp1; v.lpy[v.m + c] = lp2;
          dr_cache_store<T>(v, c, cc);
          v.k[c] = k + 1;
          mine = 1;
        }
      }
      if (mine) atomicAdd(&blk_active, 1u);
      __syncthreads();
      const int slot = iter % 3;
      if (threadIdx.x == 0 && blk_active) atomicAdd(&active_cnt[slot], blk_active);
      if (!grid_sync(bar, v.err)) return;
      const unsigned total = read_after_grid_sync(&active_cnt[slot]);
      if (leader) {
        active_cnt[(iter + 2) % 3] = 0;
        *iterations += 1;
      }
      ++iter;
      if (total == 0) break;
    }
    // every chain starts the next sample at stage 0 (each thread resets its own chains)
    for (int64_t c = c_first; c < v.m; c += stride) v.k[c] = 0;
  }
  if (err) atomicOr(v.err, err);
}

template <typename T, int E>
__global__ void dr_init_kernel(DrView<T> v) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= v.m) return;
  T x[E];
#pragma unroll
  for (int e = 0; e < E; ++e) x[e] = e < v.tg.d ? v.x[(size_t)c * v.tg.d + e] : T(0);
  T lp = full_logp<T, E>(v.tg, x);
  if (!(lp == lp)) { lp = neg_inf<T>(); atomicOr(v.err, ERR_NONFINITE); }
  v.lp[c] = lp;
}

// ---- a chain per warp (32 < d <= 1024: the layout for log-densities too wide for one thread) -------
// Lane l holds coordinates k = e 32 + l (e < E) of x, y1, y2 and the proposal; every sum over
// coordinates (the log density's, the proposal densities' squared distances) is a warp sum, and
// the chain's scalars (log pi values, the kept ratio terms, the stage) are the same in every lane.
// The random numbers are those of the chain-per-thread step: coordinate k's normal is element
// k mod 4 of Philox block floor(k / 4) of the stage, and each lane draws the Box-Muller pair that
// holds its coordinate.  Same stages, acceptance formulas and kept terms as above; the 4-state
// ablation form is chain-per-thread only.
template <typename T, int E>
__device__ __forceinline__ void drw_draw(const DrView<T>& v, const Key& key, int t, int k, const T (&c)[E],
                                         T (&y)[E], int lane) {
  const int d = v.tg.d;
  const int D = (d + 3) / 4;
  const uint32_t base = (uint32_t)(k * (D + 1));
  const T sg = v.symmetric ? v.sig[0] : v.sig[k];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int kk = e * 32 + lane;
    y[e] = T(0);
    if (kk < d) {
      const P4 r = key.block((uint32_t)t, 0, base + (uint32_t)(kk >> 2));
      T z0, z1;
      if ((kk & 3) < 2) Conv<T>::bm(r.w0, r.w1, z0, z1);
      else Conv<T>::bm(r.w2, r.w3, z0, z1);
      y[e] = fma(sg, (kk & 1) ? z1 : z0, c[e]);
    }
  }
}

template <typename T, int E>
__device__ __forceinline__ T drw_eval(const DrView<T>& v, const T (&y)[E], int lane, int& err) {
  T lpy = warp_logp<T, E>(v.tg, y, lane);
  if (!(lpy == lpy)) { lpy = neg_inf<T>(); err |= ERR_NONFINITE; }
  return lpy;
}

template <typename T, int E>
__device__ __forceinline__ T drw_sqdist(const T (&a)[E], const T (&b)[E], int d, int lane) {
  T acc = T(0);
#pragma unroll
  for (int e = 0; e < E; ++e)
    if (e * 32 + lane < d) { const T r = b[e] - a[e]; acc = fma(r, r, acc); }
  return group_sum<32>(acc);
}

template <typename T, int E>
__device__ __forceinline__ T drw_ratio(const DrView<T>& v, int k, const T (&x)[E], T lp, const T (&y1)[E], T lp1,
                                       const T (&y2)[E], T lp2, const T (&y)[E], T lpy, const DrCache<T>& cc,
                                       int lane) {
  const int d = v.tg.d;
  if (k == 0) return la1(lp, lpy);
  const T i1 = T(-0.5) / (v.sig[0] * v.sig[0]);
  if (k == 1) {
    const T num = lpy + i1 * drw_sqdist(y, y1, d, lane) + l1m(la1(lpy, lp1));
    const T den = lp + i1 * drw_sqdist(x, y1, d, lane) + cc.a1;
    if (num == neg_inf<T>() || den == neg_inf<T>()) return neg_inf<T>();
    return fmin(T(0), num - den);
  }
  const T i2 = T(-0.5) / (v.sig[1] * v.sig[1]);
  const T q1_y3_y2 = i1 * drw_sqdist(y, y2, d, lane);
  const T a1_32 = l1m(la1(lpy, lp2));
  const T n2 = lp1 + cc.q1y1y2 + cc.a1y1y2;
  const T d2 = lpy + q1_y3_y2 + a1_32;
  const T a2_321 = (n2 == neg_inf<T>() || d2 == neg_inf<T>()) ? neg_inf<T>() : fmin(T(0), n2 - d2);
  const T num = lpy + q1_y3_y2 + i2 * drw_sqdist(y, y1, d, lane) + a1_32 + l1m(a2_321);
  const T den = lp + cc.q1xy1 + cc.q2xy2 + cc.a1 + cc.a2;
  if (num == neg_inf<T>() || den == neg_inf<T>()) return neg_inf<T>();
  return fmin(T(0), num - den);
}

template <typename T, int E>
__device__ __forceinline__ bool drw_decide(const DrView<T>& v, const Key& key, int t, int k, T la, T (&x)[E],
                                           T& lp, T (&y1)[E], T& lp1, T (&y2)[E], T& lp2, const T (&y)[E],
                                           T lpy, DrCache<T>& cc, int lane) {
  const int D = (v.tg.d + 3) / 4;
  const P4 r = key.block((uint32_t)t, 0, (uint32_t)(k * (D + 1) + D));
  if (Conv<T>::log_u(r.w0, r.w1) < la) {
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = y[e];
    lp = lpy;
    return true;
  }
  if (k + 1 >= v.n_stages) return true;
  const int d = v.tg.d;
  if (k == 0) {
#pragma unroll
    for (int e = 0; e < E; ++e) y1[e] = y[e];
    lp1 = lpy;
    cc.a1 = l1m(la);
  } else {
    const T i1 = T(-0.5) / (v.sig[0] * v.sig[0]), i2 = T(-0.5) / (v.sig[1] * v.sig[1]);
    cc.q1xy1 = i1 * drw_sqdist(x, y1, d, lane);
    cc.q1y1y2 = i1 * drw_sqdist(y, y1, d, lane);
    cc.a2 = l1m(la);
    cc.a1y1y2 = l1m(la1(lp1, lpy));
    cc.q2xy2 = i2 * drw_sqdist(x, y, d, lane);
#pragma unroll
    for (int e = 0; e < E; ++e) y2[e] = y[e];
    lp2 = lpy;
  }
  return false;
}

template <typename T, int E>
__device__ __forceinline__ bool drw_step(const DrView<T>& v, const Key& key, int t, int k, T (&x)[E], T& lp,
                                         T (&y1)[E], T& lp1, T (&y2)[E], T& lp2, DrCache<T>& cc, int lane, int& err) {
  T y[E];
  if (v.symmetric) {  // y1 / lp1 hold the centre and pi*
    if (k == 0) sdr_begin<T, E>(x, y1, lp1);
    drw_draw<T, E>(v, key, t, k, y1, y, lane);
    const T lpy = drw_eval<T, E>(v, y, lane, err);
    return sdr_decide<T, E>(v, key, t, k, sdr_log_alpha<T>(lp, lp1, lpy), x, lp, y1, lp1, y, lpy);
  }
  drw_draw<T, E>(v, key, t, k, x, y, lane);
  const T lpy = drw_eval<T, E>(v, y, lane, err);
  const T la = drw_ratio<T, E>(v, k, x, lp, y1, lp1, y2, lp2, y, lpy, cc, lane);
  return drw_decide<T, E>(v, key, t, k, la, x, lp, y1, lp1, y2, lp2, y, lpy, cc, lane);
}

template <typename T, int E>
__device__ __forceinline__ void drw_load(const DrView<T>& v, int64_t c, T (&x)[E], T (&y1)[E], T (&y2)[E],
                                         int lane) {
  const int d = v.tg.d;
  const size_t md = (size_t)v.m * d;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = e * 32 + lane;
    x[e] = k < d ? v.x[(size_t)c * d + k] : T(0);
    y1[e] = k < d ? v.y[(size_t)c * d + k] : T(0);
    y2[e] = k < d ? v.y[md + (size_t)c * d + k] : T(0);
  }
}

template <typename T, int E>
__device__ __forceinline__ void drw_store(const DrView<T>& v, int64_t c, const T (&x)[E], const T (&y1)[E],
                                          const T (&y2)[E], int pending, int lane) {
  const int d = v.tg.d;
  const size_t md = (size_t)v.m * d;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = e * 32 + lane;
    if (k >= d) continue;
    v.x[(size_t)c * d + k] = x[e];
    if (pending >= 1) v.y[(size_t)c * d + k] = y1[e];
    if (pending >= 2) v.y[md + (size_t)c * d + k] = y2[e];
  }
}

// FSM kernel, a chain per warp, condensed step (one PROPOSE state per FSM step)
template <typename T, int E>
__global__ void __launch_bounds__(128) dr_fsm_warp_kernel(DrView<T> v, int budget) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < v.m; c += nwarps) {
    T x[E], y1[E], y2[E];
    drw_load<T, E>(v, c, x, y1, y2, lane);
    T lp = v.lp[c], lp1 = v.lpy[c], lp2 = v.lpy[v.m + c];
    DrCache<T> cc = dr_cache_load<T>(v, c);
    int t = v.t[c], k = v.k[c];
    const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
    int err = 0, steps = 0;
    for (int b = 0; b < budget && t < v.n; ++b) {
      ++steps;
      if (drw_step<T, E>(v, key, t, k, x, lp, y1, lp1, y2, lp2, cc, lane, err)) {
        warp_chain_emit<T, E>(v, v.tg.d, c, t, x, lane);
        if (lane == 0) v.counts[(size_t)c * v.n + t] = k + 1;
        ++t;
        k = 0;
        if (t == v.n && lane == 0) atomicAdd(v.chains_done, 1);
      } else {
        ++k;
      }
    }
    drw_store<T, E>(v, c, x, y1, y2, k, lane);
    if (lane == 0) {
      v.lp[c] = lp; v.lpy[c] = lp1; v.lpy[v.m + c] = lp2;
      if (k) dr_cache_store<T>(v, c, cc);
      v.t[c] = t; v.k[c] = k;
      v.steps[c] += steps;
      if (err) atomicOr(v.err, err);
    }
  }
}

// Synchronised kernel (Alg. 6), a chain per warp: as dr_sync_kernel.
template <typename T, int E>
__global__ void __launch_bounds__(128) dr_sync_warp_kernel(DrView<T> v, int t_begin, int t_end,
                                                           GridBarrier bar, unsigned* active_cnt,
                                                           unsigned long long* iterations) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t c_first = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  __shared__ unsigned blk_active;
  int iter = 0, err = 0;
  for (int t = t_begin; t < t_end; ++t) {
    for (int k = 0; k < v.n_stages; ++k) {
      if (threadIdx.x == 0) blk_active = 0;
      __syncthreads();
      unsigned mine = 0;
      for (int64_t c = c_first; c < v.m; c += nwarps) {
        if (v.k[c] != k) continue;  // masked: finished this sample at an earlier stage
        T x[E], y1[E], y2[E];
        drw_load<T, E>(v, c, x, y1, y2, lane);
        T lp = v.lp[c], lp1 = v.lpy[c], lp2 = v.lpy[v.m + c];
        DrCache<T> cc = dr_cache_load<T>(v, c);
        const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
        const bool done = drw_step<T, E>(v, key, t, k, x, lp, y1, lp1, y2, lp2, cc, lane, err);
        __syncwarp();  // every lane has read the chain's state before lane 0 rewrites it
        if (done) {
          warp_chain_emit<T, E>(v, v.tg.d, c, t, x, lane);
          drw_store<T, E>(v, c, x, y1, y2, 0, lane);
          if (lane == 0) {
            v.steps[c] += 1;
            v.counts[(size_t)c * v.n + t] = k + 1;
            v.lp[c] = lp;
            v.k[c] = v.n_stages;  // done with sample t
            v.t[c] = t + 1;
            if (t + 1 == v.n) atomicAdd(v.chains_done, 1);
          }
        } else {
          drw_store<T, E>(v, c, x, y1, y2, k + 1, lane);
          if (lane == 0) {
            v.steps[c] += 1;
            v.lpy[c] = lp1; v.lpy[v.m + c] = lp2;
            dr_cache_store<T>(v, c, cc);
            v.k[c] = k + 1;
          }
          mine = 1;
        }
      }
      if (mine && lane == 0) atomicAdd(&blk_active, 1u);
      __syncthreads();
      const int slot = iter % 3;
      if (threadIdx.x == 0 && blk_active) atomicAdd(&active_cnt[slot], blk_active);
      if (!grid_sync(bar, v.err)) return;
      const unsigned total = read_after_grid_sync(&active_cnt[slot]);
      if (leader) {
        active_cnt[(iter + 2) % 3] = 0;
        *iterations += 1;
      }
      ++iter;
      if (total == 0) break;
    }
    __syncwarp();
    for (int64_t c = c_first; c < v.m; c += nwarps)
      if (lane == 0) v.k[c] = 0;
    __syncwarp();  // the reset is visible to every lane before the next sample's first stage
  }
  if (err && lane == 0) atomicOr(v.err, err);
}

template <typename T, int E>
__global__ void dr_init_warp_kernel(DrView<T> v) {
  const int lane = threadIdx.x & 31;
  const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= v.m) return;
  T x[E];
#pragma unroll
  for (int e = 0; e < E; ++e) x[e] = e * 32 + lane < v.tg.d ? v.x[(size_t)c * v.tg.d + e * 32 + lane] : T(0);
  T lp = warp_logp<T, E>(v.tg, x, lane);
  if (!(lp == lp)) { lp = neg_inf<T>(); if (lane == 0) atomicOr(v.err, ERR_NONFINITE); }
  if (lane == 0) v.lp[c] = lp;
}

// ------------------------------------------------------------------------------------------
template <typename T, int E>
static cudaError_t fsm_warp_launch(const DrView<T>& v, int budget, int threads, cudaStream_t st) {
  const int64_t blocks = (v.m * 32 + threads - 1) / threads;
  dr_fsm_warp_kernel<T, E><<<(unsigned)blocks, threads, 0, st>>>(v, budget);
  return cudaGetLastError();
}

template <typename T, int E>
static cudaError_t sync_warp_launch(const DrView<T>& v, int t0, int t1, GridBarrier bar, unsigned* active_cnt,
                                    unsigned long long* iters, int threads, cudaStream_t st) {
  auto kern = dr_sync_warp_kernel<T, E>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = std::min<int64_t>((int64_t)per_sm * sms, (v.m * 32 + threads - 1) / threads);
  if (blocks < 1) blocks = 1;
  DrView<T> vv = v;
  void* args[] = {(void*)&vv, (void*)&t0, (void*)&t1, (void*)&bar, (void*)&active_cnt, (void*)&iters};
  return cudaLaunchCooperativeKernel((void*)kern, dim3((unsigned)blocks), dim3(threads), args, 0, st);
}

template <typename T, int E>
static cudaError_t init_warp_launch(const DrView<T>& v, cudaStream_t st) {
  dr_init_warp_kernel<T, E><<<(unsigned)((v.m * 32 + 127) / 128), 128, 0, st>>>(v);
  return cudaGetLastError();
}

#define FSMC_DR_WARP_DISPATCH(FN, ...)                       \
  do {                                                       \
    const int d = v.tg.d;                                    \
    if (d <= 64) return FN<T, 2>(__VA_ARGS__);               \
    if (d <= 128) return FN<T, 4>(__VA_ARGS__);              \
    if (d <= 256) return FN<T, 8>(__VA_ARGS__);              \
    if (d <= 512) return FN<T, 16>(__VA_ARGS__);             \
    if (d <= 1024) return FN<T, 32>(__VA_ARGS__);            \
    return cudaErrorInvalidValue;                            \
  } while (0)

// ------------------------------------------------------------------------------------------
template <typename T, int E>
static cudaError_t fsm_launch(const DrView<T>& v, int budget, int threads, cudaStream_t st) {
  const int64_t blocks = (v.m + threads - 1) / threads;
  const size_t smem = mom_smem_bytes<T, E>(v, threads);
  if (v.step_form == 2) {
    if (smem) dr_fsm_kernel<T, E, false, true><<<(unsigned)blocks, threads, smem, st>>>(v, budget);
    else dr_fsm_kernel<T, E, false><<<(unsigned)blocks, threads, 0, st>>>(v, budget);
  } else {
    if (smem) dr_fsm_kernel<T, E, true, true><<<(unsigned)blocks, threads, smem, st>>>(v, budget);
    else dr_fsm_kernel<T, E, true><<<(unsigned)blocks, threads, 0, st>>>(v, budget);
  }
  return cudaGetLastError();
}

template <typename T, int E>
static cudaError_t sync_launch(const DrView<T>& v, int t0, int t1, GridBarrier bar,
                               unsigned* active_cnt, unsigned long long* iters, int threads,
                               cudaStream_t st) {
  auto kern = dr_sync_kernel<T, E>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = std::min<int64_t>((int64_t)per_sm * sms, (v.m + threads - 1) / threads);
  if (blocks < 1) blocks = 1;
  DrView<T> vv = v;
  void* args[] = {(void*)&vv, (void*)&t0, (void*)&t1, (void*)&bar, (void*)&active_cnt, (void*)&iters};
  return cudaLaunchCooperativeKernel((void*)kern, dim3((unsigned)blocks), dim3(threads), args, 0, st);
}

template <typename T, int E>
static cudaError_t init_launch(const DrView<T>& v, cudaStream_t st) {
  dr_init_kernel<T, E><<<(unsigned)((v.m + 127) / 128), 128, 0, st>>>(v);
  return cudaGetLastError();
}

#define FSMC_DR_DISPATCH(FN, ...)                            \
  do {                                                       \
    const int d = v.tg.d;                                    \
    if (d <= 2) return FN<T, 2>(__VA_ARGS__);                \
    if (d <= 4) return FN<T, 4>(__VA_ARGS__);                \
    if (d <= 8) return FN<T, 8>(__VA_ARGS__);                \
    if (d <= 10) return FN<T, 10>(__VA_ARGS__);              \
    if (d <= 16) return FN<T, 16>(__VA_ARGS__);              \
    if (d <= 32) return FN<T, 32>(__VA_ARGS__);              \
    return cudaErrorInvalidValue;                            \
  } while (0)

template <typename T>
cudaError_t launch_dr_fsm(const DrView<T>& v, int budget, int threads, cudaStream_t st) {
  if (v.lanes == 32) FSMC_DR_WARP_DISPATCH(fsm_warp_launch, v, budget, threads, st);
  FSMC_DR_DISPATCH(fsm_launch, v, budget, threads, st);
}
template <typename T>
cudaError_t launch_dr_sync(const DrView<T>& v, int t0, int t1, GridBarrier bar, unsigned* active_cnt,
                           unsigned long long* iters, int threads, cudaStream_t st) {
  if (v.lanes == 32) FSMC_DR_WARP_DISPATCH(sync_warp_launch, v, t0, t1, bar, active_cnt, iters, threads, st);
  FSMC_DR_DISPATCH(sync_launch, v, t0, t1, bar, active_cnt, iters, threads, st);
}
template <typename T>
cudaError_t launch_dr_init(const DrView<T>& v, cudaStream_t st) {
  if (v.lanes == 32) FSMC_DR_WARP_DISPATCH(init_warp_launch, v, st);
  FSMC_DR_DISPATCH(init_launch, v, st);
}

template cudaError_t launch_dr_fsm<float>(const DrView<float>&, int, int, cudaStream_t);
template cudaError_t launch_dr_fsm<double>(const DrView<double>&, int, int, cudaStream_t);
template cudaError_t launch_dr_sync<float>(const DrView<float>&, int, int, GridBarrier, unsigned*,
                                           unsigned long long*, int, cudaStream_t);
template cudaError_t launch_dr_sync<double>(const DrView<double>&, int, int, GridBarrier, unsigned*,
                                            unsigned long long*, int, cudaStream_t);
template cudaError_t launch_dr_init<float>(const DrView<float>&, cudaStream_t);
template cudaError_t launch_dr_init<double>(const DrView<double>&, cudaStream_t);

}  // namespace fsmc
