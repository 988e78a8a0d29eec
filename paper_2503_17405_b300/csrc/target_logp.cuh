// Full log-densities log pi(y) of the targets the chain-per-thread samplers (delayed
// rejection, slice sampling) run on, with y in registers (E >= d slots, padding ignored), and
// the emission of a finished sample (stored, or folded into Kahan sums of x and x^2).
#pragma once
#include "fsmc_device.cuh"
#include "fsmc_kernels.h"

namespace fsmc {

// log pi for the full-density targets, one chain per thread
template <typename T, int E>
__device__ __forceinline__ T full_logp(const TargetView<T>& tg, const T (&y)[E]) {
  const int d = tg.d;
  if (tg.kind == TGT_FUNNEL) {
    T ss = T(0);
#pragma unroll
    for (int e = 1; e < E; ++e)
      if (e < d) ss = fma(y[e], y[e], ss);
    const T v = y[0];
    const T ev = sizeof(T) == 4 ? (T)expf(-(float)v) : (T)exp(-(double)v);
    return -v * v / T(18) - T(d - 1) * v / T(2) - T(0.5) * ev * ss;
  } else if (tg.kind == TGT_GAUSS_DIAG) {
    T acc = T(0);
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (e < d) { const T z = (y[e] - tg.vec[e]) / tg.vec2[e]; acc = fma(z, z, acc); }
    return -T(0.5) * acc;
  } else if (tg.kind == TGT_MOG) {
    // log sum_k w_k exp(-q_k / 2), q_k = s_k^2 c_par / d + |u_k|^2 c_perp with s_k = 1^T (y - mu_k)
    // (summed from the differences) and u_k = y - mu_k - (s_k / d) 1 (the covariance's two
    // eigenspaces)
    const T inv_d = T(1) / T(d);
    T lmax = neg_inf<T>(), wsum = T(0);
    for (int k = 0; k < tg.n_data; ++k) {
      const T* mk = tg.X + (size_t)k * d;
      T sk = T(0);
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (e < d) sk += y[e] - mk[e];
      const T mean = sk * inv_d;
      T uu = T(0);
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (e < d) { const T u = y[e] - mk[e] - mean; uu = fma(u, u, uu); }
      const T lk = tg.vec[k] - T(0.5) * fma(sk * mean, tg.c_par, uu * tg.c_perp);
      if (lk > lmax) {
        wsum = wsum * (sizeof(T) == 4 ? (T)expf((float)(lmax - lk)) : (T)exp((double)(lmax - lk))) + T(1);
        lmax = lk;
      } else {
        wsum += sizeof(T) == 4 ? (T)expf((float)(lk - lmax)) : (T)exp((double)(lk - lmax));
      }
    }
    return lmax + (sizeof(T) == 4 ? (T)logf((float)wsum) : (T)log((double)wsum));
  } else if (tg.kind == TGT_LOGREG) {
    T acc = T(0);
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (e < d) acc = fma(y[e], y[e], acc);
    acc *= -T(0.5);
    for (int i = 0; i < tg.n_data; ++i) {
      const T* row = tg.X + (size_t)i * d;
      T eta = T(0);
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (e < d) eta = fma(row[e], y[e], eta);
      acc += tg.vec[i] * eta - softplus<T>(eta);
    }
    return acc;
  }
  return neg_inf<T>();
}

template <typename T, int E>
__device__ __forceinline__ void chain_emit(const ChainsView<T>& v, int d, int64_t c, int t, const T (&x)[E]) {
  if (v.out) {
    T* dst = v.out + ((size_t)c * v.n + t) * d;
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (e < d) dst[e] = x[e];
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if (e >= d) continue;
      const size_t o = (size_t)c * d + e;
      T* mo = v.mom;
      const size_t st = v.mom_stride;
      T y = x[e] - mo[o + st]; T tt = mo[o] + y; mo[o + st] = (tt - mo[o]) - y; mo[o] = tt;
      const T x2 = x[e] * x[e];
      y = x2 - mo[o + 3 * st]; tt = mo[o + 2 * st] + y; mo[o + 3 * st] = (tt - mo[o + 2 * st]) - y;
      mo[o + 2 * st] = tt;
    }
  }
}

}  // namespace fsmc
