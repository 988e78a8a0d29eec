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

// log pi with a chain per warp: lane l holds coordinates k = e 32 + l (e < E, k < d) of y; every
// sum over coordinates is a warp sum, and every lane returns the same value.
template <typename T, int E>
__device__ __forceinline__ T warp_logp(const TargetView<T>& tg, const T (&y)[E], int lane) {
  const int d = tg.d;
  if (tg.kind == TGT_FUNNEL) {
    T ss = T(0);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = e * 32 + lane;
      if (k >= 1 && k < d) ss = fma(y[e], y[e], ss);
    }
    ss = group_sum<32>(ss);
    const T v = __shfl_sync(0xffffffffu, y[0], 0);
    const T ev = sizeof(T) == 4 ? (T)expf(-(float)v) : (T)exp(-(double)v);
    return -v * v / T(18) - T(d - 1) * v / T(2) - T(0.5) * ev * ss;
  } else if (tg.kind == TGT_GAUSS_DIAG) {
    T acc = T(0);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = e * 32 + lane;
      if (k < d) { const T z = (y[e] - tg.vec[k]) / tg.vec2[k]; acc = fma(z, z, acc); }
    }
    return -T(0.5) * group_sum<32>(acc);
  } else if (tg.kind == TGT_MOG) {
    const T inv_d = T(1) / T(d);
    T lmax = neg_inf<T>(), wsum = T(0);
    for (int kk = 0; kk < tg.n_data; ++kk) {
      const T* mk = tg.X + (size_t)kk * d;
      T sk = T(0);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = e * 32 + lane;
        if (k < d) sk += y[e] - mk[k];
      }
      sk = group_sum<32>(sk);
      const T mean = sk * inv_d;
      T uu = T(0);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = e * 32 + lane;
        if (k < d) { const T u = y[e] - mk[k] - mean; uu = fma(u, u, uu); }
      }
      uu = group_sum<32>(uu);
      const T lk = tg.vec[kk] - T(0.5) * fma(sk * mean, tg.c_par, uu * tg.c_perp);
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
      if (e * 32 + lane < d) acc = fma(y[e], y[e], acc);
    acc = -T(0.5) * group_sum<32>(acc);
    for (int i = 0; i < tg.n_data; ++i) {
      const T* row = tg.X + (size_t)i * d;
      T eta = T(0);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = e * 32 + lane;
        if (k < d) eta = fma(row[k], y[e], eta);
      }
      eta = group_sum<32>(eta);
      acc += tg.vec[i] * eta - softplus<T>(eta);
    }
    return acc;
  }
  return neg_inf<T>();
}

// One compensated (Kahan) step for the sum and the sum of squares of a coordinate; the square
// is rounded on its own (no contraction into the subtraction), so every caller gets the same bits.
template <typename T>
__device__ __forceinline__ void kahan_moments(T& s, T& cs, T& s2, T& c2, T x) {
  T y = x - cs;
  T tt = s + y;
  cs = (tt - s) - y;
  s = tt;
  T x2;
  if constexpr (sizeof(T) == 4) x2 = __fmul_rn(x, x);
  else x2 = __dmul_rn(x, x);
  y = x2 - c2;
  tt = s2 + y;
  c2 = (tt - s2) - y;
  s2 = tt;
}

// Moments-only jobs, one chain per thread: a chain's four running sums (sum and compensation of
// x and of x^2, per coordinate) can be held in shared memory while a kernel advances the chain
// -- loaded when it starts, written back when it stops -- so that device memory sees one read
// and one write per chain and launch instead of one of each per sample.  Each thread owns a
// slot of 4 E + 1 values ([4][E], padded to an odd stride so that the slots of a warp's 32
// threads start in 32 different banks); every access is the slot base plus a constant.
// slot null: the sums are updated in device memory.
template <typename T, int E>
struct MomSmem {
  T* slot;
  static constexpr int kSlot = 4 * E + 1;
  __device__ __forceinline__ T& at(int q, int e) const { return slot[q * E + e]; }
};

template <typename T, int E>
__device__ __forceinline__ void mom_smem_load(const ChainsView<T>& v, int d, int64_t c, const MomSmem<T, E>& ms) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (e < d) ms.at(q, e) = v.mom[q * v.mom_stride + (size_t)c * d + e];
}

template <typename T, int E>
__device__ __forceinline__ void mom_smem_store(const ChainsView<T>& v, int d, int64_t c, const MomSmem<T, E>& ms) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (e < d) v.mom[q * v.mom_stride + (size_t)c * d + e] = ms.at(q, e);
}

template <typename T, int E>
__device__ __forceinline__ void chain_emit(const ChainsView<T>& v, int d, int64_t c, int t, const T (&x)[E],
                                           const MomSmem<T, E>& ms = MomSmem<T, E>{nullptr}) {
  if (v.out) {
    T* dst = v.out + ((size_t)c * v.n + t) * d;
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (e < d) dst[e] = x[e];
  } else if (ms.slot) {
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (e < d) kahan_moments<T>(ms.at(0, e), ms.at(1, e), ms.at(2, e), ms.at(3, e), x[e]);
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if (e >= d) continue;
      const size_t o = (size_t)c * d + e, st = v.mom_stride;
      T* mo = v.mom;
      kahan_moments<T>(mo[o], mo[o + st], mo[o + 2 * st], mo[o + 3 * st], x[e]);
    }
  }
}

// A finished sample with a chain per warp (lane l: coordinates e 32 + l): stored, or folded into
// the Kahan sums of x and x^2 in device memory.
template <typename T, int E>
__device__ __forceinline__ void warp_chain_emit(const ChainsView<T>& v, int d, int64_t c, int t, const T (&x)[E],
                                                int lane) {
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = e * 32 + lane;
    if (k >= d) continue;
    if (v.out) {
      v.out[((size_t)c * v.n + t) * d + k] = x[e];
    } else {
      const size_t o = (size_t)c * d + k, st = v.mom_stride;
      T* mo = v.mom;
      kahan_moments<T>(mo[o], mo[o + st], mo[o + 2 * st], mo[o + 3 * st], x[e]);
    }
  }
}

// Dynamic shared memory for the moment sums of a chain-per-thread FSM launch: 0 (device memory)
// for jobs that store their samples or when the block's slots would exceed 48 KB.
template <typename T, int E>
inline size_t mom_smem_bytes(const ChainsView<T>& v, int threads) {
  const size_t b = (size_t)MomSmem<T, E>::kSlot * threads * sizeof(T);
  return (v.out || b > 48 * 1024) ? 0 : b;
}

}  // namespace fsmc
