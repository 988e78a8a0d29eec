// Pieces of elliptical slice sampling (Alg. 8) shared by the ESS kernels: the state names, the
// slice threshold and the bracket angle's sine and cosine.
#pragma once
#include "fsmc_device.cuh"

namespace fsmc {

constexpr double kTwoPi = 6.283185307179586476925286766559;
enum EssState : int { ESS_INIT = 0, ESS_SHRINK = 1 };

// The direction ring of a single-precision GP-logit job (other than the ablation step form)
// holds ns = -s nu, s the labels' signs (s_i = +1 where the label of coordinate i is +1): the
// generators fold the sign in when they store a direction (exact), and the GP-logit step and
// synchronised visit, which work on sign-folded coordinates, read the ring as is.  Every other
// job's ring holds nu.
template <typename V>
__host__ __device__ __forceinline__ bool ess_ring_folded(const V& v) {
  return sizeof(*v.nu) == 4 && v.tg.kind == TGT_GP_LOGIT && v.step_form != 2;
}

// Slice threshold log y = log f(x) + log u.  In single precision a u within ~1e-5 of 1 makes
// the sum round back to log f(x); the bracket would then shrink onto theta = 0 without ever
// finding log f(x') > log y.  The threshold is therefore kept at least one ulp below log f(x),
// which moves it by at most one ulp and makes theta -> 0 always accept.
template <typename T>
__device__ __forceinline__ T ess_threshold(T ell, T log_u) {
  T logy = ell + log_u;
  if constexpr (sizeof(T) == 4) {
    if (!(logy < ell) && ell > -INFINITY) logy = nextafterf(ell, -INFINITY);
  }
  return logy;
}

// sin and cos of a bracket angle th in (-2 pi, 2 pi).  Single precision reduces th to
// [-pi, pi], where __sincosf is accurate to ~5e-7; double precision calls sincos.
template <typename T>
__device__ __forceinline__ void ess_sincos(T th, T& sn, T& cs) {
  if constexpr (sizeof(T) == 4) {
    const float red = fmaf(-6.28318530717958647692f, rintf(th * 0.15915494309189533577f), th);
    __sincosf(red, &sn, &cs);
  } else {
    sincos(th, &sn, &cs);
  }
}

}  // namespace fsmc
