// Elliptical slice sampling (appendix Alg. 8) as a finite state machine.
//
// States (Fig. 2, "Elliptical Slice Sampling"): INIT (S1) draws the threshold and the
// initial angle and makes the first proposal; SHRINK (S2, the loop body) narrows the
// bracket and makes a new proposal; DONE (S3) accepts and emits the sample.  One FSM
// step is the bundled step of Alg. 4 amortised as in Alg. 5: it runs INIT or SHRINK,
// then the single expensive call g = log f(x'), then DONE if the proposal clears the
// threshold -- so every step costs exactly one likelihood evaluation and a sample takes
// N + 1 steps (N shrinks).
//
// The ellipse direction nu = L z of INIT does not depend on the chain state, only on
// (chain, sample), so it is produced ahead of time by a separate contraction kernel
// (ess_nu_gen) into a per-chain ring of W slots; this is the paper's amortisation of an
// expensive state-independent computation, moved out of the step altogether.
#include <algorithm>
#include <climits>
#include "ess_common.cuh"
#include "fsmc_device.cuh"
#include "fsmc_kernels.h"

// The build compiles this file as four objects, FSMC_ESS_PART = 1 (FSM step, single precision),
// 2 (FSM step, double precision, and the fused serving launches), 3 (the synchronised program)
// and 4 (the rest), each instantiating its own launchers, so that they compile in parallel;
// without the macro one object holds everything.
#ifndef FSMC_ESS_PART
#define FSMC_ESS_PART 0
#endif
#define FSMC_ESS_HAS(p) (FSMC_ESS_PART == 0 || FSMC_ESS_PART == (p))

namespace fsmc {


// ------------------------------------------------------------------------------------------
// nu = L z for a tile of (chain, sample) columns.  z is generated from the chain's Philox
// stream (tag 0, draws 0..ceil(d/2)-1) directly into shared memory, so it never touches HBM.
// Block: 256 threads = 32 row-groups x 8 column-groups, each thread an 8x8 register tile;
// tile = 256 rows x 64 columns (64 chains at the same ring offset w = by).  The reduction
// dimension is streamed in chunks of 16 through two shared-memory buffers: while the block
// multiplies chunk c, it stages chunk c+1 (L^T rows by one thread each, z by Philox), so one
// barrier per chunk suffices.  Rows above the diagonal are skipped per warp (L is lower
// triangular).  Both staging writes are bank-conflict free.
template <typename T>
__device__ __forceinline__ void ess_nu_gen_tile(const EssView<T>& v, int64_t bx, int by, int bz) {
  constexpr int BM = 256, BN = 64, BK = 16;
  __shared__ __align__(16) T As[2][BK][BM];
  __shared__ __align__(16) T Bs[2][BK][BN + 4];
  __shared__ int col_sample[BN];

  const int d = v.tg.d;
  const int tid = threadIdx.x;
  const int r0 = bz * BM;
  const int w = by;
  const int64_t c0 = bx * BN;
  const bool fold = ess_ring_folded(v);

  int active = 0;
  if (tid < BN) {
    const int64_t c = c0 + tid;
    int smp = -1;
    if (c < v.m) {
      const int s = v.gen_lo[c] + w;
      if (s < v.gen_hi[c]) smp = s;
    }
    col_sample[tid] = smp;
    active = smp >= 0;
  }
  const int n_active = __syncthreads_count(active);
  if (n_active == 0) return;
  if (tid == 0 && bz == 0) atomicAdd(v.gen_cols, (unsigned long long)n_active);

  const int ty = tid >> 3, tx = tid & 7;
  const int warp = tid >> 5;
  const int D = (d + 3) / 4;  // Philox blocks of z (four normals each)
  const int kmax = min(d, r0 + BM);
  // staging roles: z column zc and normals 4*zp .. 4*zp+3 of the chunk; L row lr
  const int zc = tid & 63, zp = tid >> 6;
  const int z_smp = col_sample[zc];
  const Key zkey{(uint32_t)(v.chain0 + c0 + zc), v.seed_lo, v.seed_hi};
  const int lr = r0 + tid;
  const bool vec_rows = (d % 4) == 0 && sizeof(T) == 4;

  auto stage = [&](int buf, int q0) {
    {
      const int blk = q0 / 4 + zp;  // one Philox block: normals q0 + 4 zp .. q0 + 4 zp + 3
      T z[4] = {T(0), T(0), T(0), T(0)};
      if (z_smp >= 0 && blk < D) Conv<T>::normal_quad(zkey.block((uint32_t)z_smp, 0, (uint32_t)blk), z);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int kk = 4 * zp + i;
        Bs[buf][kk][zc] = (q0 + kk < d) ? z[i] : T(0);
      }
    }
    if (lr < d && q0 <= lr) {
      const T* row = v.tg.L + (size_t)lr * d + q0;
      if (vec_rows && q0 + BK <= d) {
#pragma unroll
        for (int q = 0; q < BK / 4; ++q) {
          const float4 f = __ldg(reinterpret_cast<const float4*>(row) + q);
          const int gq = q0 + 4 * q;
          As[buf][4 * q + 0][tid] = gq + 0 <= lr ? (T)f.x : T(0);
          As[buf][4 * q + 1][tid] = gq + 1 <= lr ? (T)f.y : T(0);
          As[buf][4 * q + 2][tid] = gq + 2 <= lr ? (T)f.z : T(0);
          As[buf][4 * q + 3][tid] = gq + 3 <= lr ? (T)f.w : T(0);
        }
      } else {
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
          const int gq = q0 + kk;
          As[buf][kk][tid] = (gq < d && gq <= lr) ? row[kk] : T(0);
        }
      }
    } else {
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) As[buf][kk][tid] = T(0);
    }
  };

  T acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = T(0);

  stage(0, 0);
  __syncthreads();
  int buf = 0;
  for (int q0 = 0; q0 < kmax; q0 += BK) {
    if (q0 + BK < kmax) stage(buf ^ 1, q0 + BK);
    if (r0 + warp * 32 + 31 >= q0) {  // rows of this warp reach the chunk's columns
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[8], b[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = As[buf][kk][ty * 8 + i];
#pragma unroll
        for (int j = 0; j < 8; ++j) b[j] = Bs[buf][kk][tx * 8 + j];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
    }
    __syncthreads();
    buf ^= 1;
  }
  // write nu rows r0+ty*8.. of each active column to its ring slot
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int col = tx * 8 + j;
    const int smp = col_sample[col];
    if (smp < 0) continue;
    const int64_t c = c0 + col;
    T* dst = v.nu + ((size_t)c * v.W + (smp % v.W)) * v.dstride;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = r0 + ty * 8 + i;
      if (r < d) dst[r] = fold && v.tg.vec[r] > T(0) ? -acc[i][j] : acc[i][j];
    }
  }
  __syncthreads();  // the next tile reuses the shared staging
}

template <typename T>
__global__ void __launch_bounds__(256) ess_nu_gen_kernel(EssView<T> v) {
  ess_nu_gen_tile<T>(v, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ------------------------------------------------------------------------------------------
// log-likelihood of x' summed over the chain group (each lane its coordinates)
template <typename T, int G, int E>
__device__ __forceinline__ T ess_loglik(const TargetView<T>& tg, const T (&xp)[E], int lane,
                                        const T (&yv)[E], unsigned gmask) {
  T part = T(0);
  if (tg.kind == TGT_GP_LOGIT) {
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (e * G + lane < tg.d) part += softplus<T>(-yv[e] * xp[e]);
    return -group_sum<G>(part, gmask);
  } else if (tg.kind == TGT_GAUSS_CONJ) {
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (e * G + lane < tg.d) { const T r = yv[e] - xp[e]; part = fma(r, r, part); }
    return -group_sum<G>(part, gmask) / (T(2) * tg.s2);
  }
  return T(0);  // TGT_FLAT
}

// GP-logit likelihood in single precision, in base 2.  With labels s_i = +-1 the lanes keep the
// sign-folded coordinates xs = -s x and ns = -s nu (exact), and the step scales cos(th) and
// sin(th) by log2(e) once, so that t' = log2(e) (-s_i x'_i) = xs cs2 + ns sn2 costs one
// multiply-add per coordinate and
//   softplus(-s_i x'_i) = ln 2 log2(1 + 2^t').
// A lane's coordinates are taken in groups of eight: the group's factors 1 + 2^t' (ex2.approx,
// one add each) are multiplied together and the group contributes log2 of the product
// (lg2.approx), one base-2 logarithm per eight coordinates instead of one per coordinate.  Every
// factor is >= 1, so the product cannot underflow; it overflows only when the group's t' sum to
// more than ~126 (|x'_i| of ~11 on every coordinate, or ~87 on one), and a product above 2^126,
// infinite or NaN sends the group to the per-coordinate form sum log2(1 + 2^min(t', 126)), whose
// terms are finite for finite t'.  Relative error of a product of eight rounded factors: ~1e-6,
// i.e. ~1.5e-6 in its log2, of the order of the per-coordinate form's summed errors (~2e-7 per
// coordinate).
// Coordinates are processed in pairs with the packed FP32 instructions (FFMA2 / FMUL2 / FADD2:
// two single-precision operations, each rounded as its scalar form, per instruction).  Padded
// coordinates (beyond d) contribute the factor 1 exactly, so ragged and full rows give the same
// bits.
constexpr float kLn2f = 0.693147180559945309417f;
constexpr float kLog2ef = 1.44269504088896340736f;

// The factors of group g of this lane's coordinates (n of them, at most eight) and the log2 of
// their product; q is the product (> 2^126, infinite or NaN: overflowed).
template <int G, int E, bool FULL>
__device__ __forceinline__ float ess_gp32_group(const float (&xs)[E], const float (&ns)[E], float cs2, float sn2,
                                                int g, int lane, int d, float& q) {
  constexpr int kGrp = 8;
  const int n = E - g < kGrp ? E - g : kGrp;  // a constant once the callers' loops are unrolled
  const float2 c2 = make_float2(cs2, cs2), s2 = make_float2(sn2, sn2), one = make_float2(1.f, 1.f);
  float f[kGrp];
#pragma unroll
  for (int e = 0; e + 1 < n; e += 2) {
    const int k0 = (g + e) * G + lane, k1 = (g + e + 1) * G + lane;
    const float2 tt = __ffma2_rn(make_float2(xs[g + e], xs[g + e + 1]), c2,
                                 __fmul2_rn(make_float2(ns[g + e], ns[g + e + 1]), s2));
    const float2 y = __fadd2_rn(make_float2(ex2_approx(tt.x), ex2_approx(tt.y)), one);
    f[e] = (FULL || k0 < d) ? y.x : 1.f;
    f[e + 1] = (FULL || k1 < d) ? y.y : 1.f;
  }
  if (n % 2) {
    const int e = n - 1, k = (g + e) * G + lane;
    f[e] = (FULL || k < d) ? ex2_approx(fmaf(xs[g + e], cs2, ns[g + e] * sn2)) + 1.f : 1.f;
  }
  // product of the group's factors: pairwise in packed form, then the two halves
  if (n >= 2) {
    float2 p = make_float2(f[0], f[1]);
#pragma unroll
    for (int e = 2; e + 1 < n; e += 2) p = __fmul2_rn(p, make_float2(f[e], f[e + 1]));
    q = p.x * p.y;
    if (n % 2) q *= f[n - 1];
  } else {
    q = f[0];
  }
  return lg2_approx(q);
}

// The likelihood.  A lane's term a (the sum of its groups' log2 values) is added over the chain
// group.  While no group of the warp overflowed, every group's log2 is at most 126, so a <=
// 126 ceil(E / 8); with 32 lanes the terms are then rounded to the fixed-point grid 2^-kFx (kFx
// = 19 up to eight coordinates per lane: error <= 2^-20 per lane, about 2^-18 root-mean-square
// over 32 lanes; 32 of them sum below 2^31, exactly, in a 32-bit integer) and added by one warp
// reduction (redux.sync) instead of a five-level shuffle tree.  The tree's five roundings and the
// sum's own rounding to single precision (half an ulp: 2^-18 to 2^-17 for sums of 64 to 256) are
// errors of the same order.  Chain groups of fewer lanes add by the tree.
// When some group of the warp overflowed (or is NaN) the whole warp takes the branch in which
// each lane recomputes its overflowed groups in the per-coordinate form and the lanes add by the
// tree.
template <int G, int E, bool FULL = false>
__device__ __forceinline__ float ess_loglik_gp32(const float (&xs)[E], const float (&ns)[E], float cs2, float sn2,
                                                 int lane, int d, unsigned gmask) {
  constexpr int kGrp = 8;
  float acc = 0.f;
  bool over = false;
#pragma unroll
  for (int g = 0; g < E; g += kGrp) {
    float q;
    acc += ess_gp32_group<G, E, FULL>(xs, ns, cs2, sn2, g, lane, d, q);
    over |= !(q <= 0x1p126f);
  }
  if (__any_sync(gmask, over)) {
    acc = 0.f;
#pragma unroll
    for (int g = 0; g < E; g += kGrp) {
      const int n = E - g < kGrp ? E - g : kGrp;
      float q;
      float lq = ess_gp32_group<G, E, FULL>(xs, ns, cs2, sn2, g, lane, d, q);
      if (!(q <= 0x1p126f)) {  // the per-coordinate form, each term finite for finite t' (NaN stays NaN)
        lq = 0.f;
#pragma unroll
        for (int e = 0; e < n; ++e)
          if (FULL || (g + e) * G + lane < d) {
            const float tp = fmaf(xs[g + e], cs2, ns[g + e] * sn2);
            lq += lg2_approx(1.f + ex2_approx(tp > 126.f ? 126.f : tp));
          }
      }
      acc += lq;
    }
    return -kLn2f * group_sum<G>(acc, gmask);
  }
  if constexpr (G == 32) {
    constexpr int kGroups = (E + kGrp - 1) / kGrp;
    constexpr int kFx = kGroups <= 1 ? 19 : kGroups <= 2 ? 18 : kGroups <= 4 ? 17 : 16;
    const int qa = __float2int_rn(acc * (float)(1 << kFx));
    int sum;
    asm volatile("redux.sync.add.s32 %0, %1, 0xffffffff;" : "=r"(sum) : "r"(qa));
    return (float)sum * (-kLn2f / (float)(1 << kFx));
  } else {
    return -kLn2f * group_sum<G>(acc, gmask);
  }
}

// sign of coordinate e flipped where bit e of mask is set (exact)
__device__ __forceinline__ float flip_sign(float v, uint32_t mask, int e) {
  return __int_as_float(__float_as_int(v) ^ (int)((mask >> e) << 31));
}

// The base-2 GP-logit path is taken for every single-precision GP-logit job.
template <typename T, int E>
constexpr bool kEssGpFast = sizeof(T) == 4;

template <typename T>
__device__ __forceinline__ void kahan_add(T& sum, T& comp, T v) {
  const T y = v - comp;
  const T t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

// mslot (moments-only jobs, optional): this lane's shared-memory copy of its coordinates'
// running sums, [4][E] (sum, compensation, sum of squares, compensation), updated in place of
// device memory with the same operations.
template <typename T, int G, int E, bool FULL = false>
__device__ __forceinline__ void ess_emit(const EssView<T>& v, int64_t c, int t, int lane,
                                         const T (&x)[E], T* mslot = nullptr) {
  const int d = FULL ? E * G : v.tg.d;
  if (v.out) {
    T* dst = v.out + ((size_t)c * v.n + t) * d;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = e * G + lane;
      if (FULL || k < d) dst[k] = x[e];
    }
  } else if (mslot) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = e * G + lane;
      if (k < d) {
        T s = mslot[e], cs = mslot[E + e];
        kahan_add(s, cs, x[e]);
        mslot[e] = s; mslot[E + e] = cs;
        T s2 = mslot[2 * E + e], c2 = mslot[3 * E + e];
        kahan_add(s2, c2, x[e] * x[e]);
        mslot[2 * E + e] = s2; mslot[3 * E + e] = c2;
      }
    }
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = e * G + lane;
      if (k < d) {
        const size_t o = (size_t)c * d + k;
        T s = v.mom[o], cs = v.mom[o + v.mom_stride];
        kahan_add(s, cs, x[e]);
        v.mom[o] = s; v.mom[o + v.mom_stride] = cs;
        T s2 = v.mom[o + 2 * v.mom_stride], c2 = v.mom[o + 3 * v.mom_stride];
        kahan_add(s2, c2, x[e] * x[e]);
        v.mom[o + 2 * v.mom_stride] = s2; v.mom[o + 3 * v.mom_stride] = c2;
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// FSM kernel: every chain advances `budget` states (fewer if its ring runs dry or it
// finishes).  Chain-group layout: G lanes own one chain, lane l holds coordinates l, l+G, ...
// Chain groups of 8 or more lanes compute G Philox blocks at once and each state fetches its
// words by shuffle, instead of every lane computing the same block; chain-per-thread computes
// the block it needs.  A sample t uses draws D + off, off = 0 for its INIT and 1 + s for its
// s-th shrink, so the cache holds either
//   narrow: the first kOff offsets of kSamp consecutive samples tb, tb + 1, ...
//           (lane l: sample tb + l / kOff, draw D + l % kOff), or
//   wide:   G consecutive offsets ob, ob + 1, ... of sample tb (lane l: draw D + ob + l),
// refilled when a state asks for a (sample, offset) outside it.  With 32 lanes the narrow layout
// covers two samples of up to 15 shrinks each, so most samples cost half a refill.
template <int G>
struct PhiloxLaneCache {
  static constexpr int kOff = G < 16 ? G : 16;
  static constexpr int kSamp = G >= 8 ? G / kOff : 1;
  P4 cache{0u, 0u, 0u, 0u};
  int tb = -(1 << 30), ob = 0;
  bool wide = false;
  __device__ __forceinline__ P4 fetch(const Key& key, int t, int D, int off, int lane, unsigned gmask) {
    if constexpr (G >= 8) {
      int src;
      if (!wide && (unsigned)t - (unsigned)tb < (unsigned)kSamp && off < kOff) {
        src = (t - tb) * kOff + off;
      } else if (wide && t == tb && (unsigned)(off - ob) < (unsigned)G) {
        src = off - ob;
      } else if (off < kOff) {
        tb = t;
        wide = false;
        cache = key.block((uint32_t)(t + lane / kOff), 0, (uint32_t)(D + lane % kOff));
        src = off;
      } else {
        tb = t;
        ob = off;
        wide = true;
        cache = key.block((uint32_t)t, 0, (uint32_t)(D + off + lane));
        src = 0;
      }
      return P4{__shfl_sync(gmask, cache.w0, src, G), __shfl_sync(gmask, cache.w1, src, G),
                __shfl_sync(gmask, cache.w2, src, G), __shfl_sync(gmask, cache.w3, src, G)};
    } else {
      return key.block((uint32_t)t, 0, (uint32_t)(D + off));
    }
  }
};

// The same cache for the single-precision GP-logit path, holding each lane's block already
// converted to the two uniforms the states use: a = u(w0, w1) (the threshold's u at INIT, the
// shrink's u at SHRINK) and b = u(w2, w3) (the initial angle's u).  A state then moves one float
// (SHRINK) or two (INIT) by shuffle instead of four words, and converts nothing; the values are
// the bits Conv<float>::u gives.  The window of the current sample is kept as (lim, sh): offset
// off < lim sits at lane sh + off.  INIT (offset 0) sets it from the narrow layout, refilling
// that when the sample is not held; the shrinks of a sample ask for offsets 1, 2, ... in turn,
// and the first offset past the window refills the cache wide (refill).  Groups of fewer than
// eight lanes compute each block when it is asked for (lim is then unbounded).
template <int G>
struct UniformLaneCache {
  static constexpr int kOff = G < 16 ? G : 16;
  static constexpr int kSamp = G >= 8 ? G / kOff : 1;
  float a = 0.f, b = 0.f;
  int tb = -(1 << 30);  // first sample of the narrow layout (far below any sample when wide or empty)
  int lim = G >= 8 ? 0 : INT_MAX, sh = 0;
  __device__ __forceinline__ void fill(const P4& r) {
    a = Conv<float>::u(r.w0, r.w1);
    b = Conv<float>::u(r.w2, r.w3);
  }
  // INIT of sample t: the uniforms of offset 0; sets the window of t
  __device__ __forceinline__ float2 init_ab(const Key& key, int t, int D, int lane, unsigned gmask) {
    if constexpr (G >= 8) {
      if ((unsigned)(t - tb) >= (unsigned)kSamp) {
        tb = t;
        fill(key.block((uint32_t)(t + lane / kOff), 0, (uint32_t)(D + lane % kOff)));
      }
      sh = (t - tb) * kOff;
      lim = kOff;
      return make_float2(__shfl_sync(gmask, a, sh, G), __shfl_sync(gmask, b, sh, G));
    } else {
      const P4 r = key.block((uint32_t)t, 0, (uint32_t)D);
      return make_float2(Conv<float>::u(r.w0, r.w1), Conv<float>::u(r.w2, r.w3));
    }
  }
  // offsets off .. off + G - 1 of sample t (off >= lim)
  __device__ __forceinline__ void refill(const Key& key, int t, int D, int off, int lane) {
    if constexpr (G >= 8) {
      tb = -(1 << 30);
      fill(key.block((uint32_t)t, 0, (uint32_t)(D + off + lane)));
      sh = -off;
      lim = off + G;
    }
  }
  // the uniform a of offset off < lim of the current sample t
  __device__ __forceinline__ float shrink_a(const Key& key, int t, int D, int off, int lane, unsigned gmask) {
    if constexpr (G >= 8) {
      return __shfl_sync(gmask, a, sh + off, G);
    } else {
      const P4 r = key.block((uint32_t)t, 0, (uint32_t)(D + off));
      return Conv<float>::u(r.w0, r.w1);
    }
  }
};

// Keeps a value the program does not otherwise use (the masked branch's log-density).
template <typename T>
__device__ __forceinline__ void ess_keep(T v) {
  if constexpr (sizeof(T) == 4) asm volatile("" ::"f"(v));
  else asm volatile("" ::"d"(v));
}

// Any target, any precision: x, nu and x' per lane.  AMORT (the step form of Alg. 5 and
// App. B.2): one log-density evaluation per step, after the state code.  !AMORT (the paper's
// ablation): the bundled step without amortisation, as vmap runs it -- INIT and SHRINK each
// call the log-density, so every step makes both calls, one of them for the state the chain
// is not in (masked: its value is computed and dropped).  Both forms compute the same samples.
template <typename T, int G, int E, bool AMORT = true>
__device__ __forceinline__ void ess_advance_chain_generic(const EssView<T>& v, int64_t c, int budget, int lane) {
  const int d = v.tg.d;
  const int D = (d + 3) / 4;  // Philox blocks of z (four normals each)
  const unsigned gmask = group_mask<G>();
  T x[E], nu[E], yv[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = e * G + lane;
    x[e] = k < d ? v.x[(size_t)c * d + k] : T(0);
    yv[e] = (k < d && v.tg.vec) ? v.tg.vec[k] : T(0);
    nu[e] = T(0);
  }
  T ell = v.ell[c], logy = v.logy[c], th = v.th[c], thmin = v.thmin[c], thmax = v.thmax[c];
  int t = v.t[c], st = v.k[c], s = v.s[c];
  const int hi = v.gen_hi[c];
  const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
  int slot = t % v.W;  // ring slot of sample t, advanced with t
  auto load_nu = [&]() {
    const T* src = v.nu + ((size_t)c * v.W + slot) * v.dstride;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = e * G + lane;
      if (k < d) nu[e] = src[k];
    }
  };
  if (st == ESS_SHRINK && t < v.n) load_nu();
  int steps = 0;
  int err = 0;
  PhiloxLaneCache<G> pc;
  for (int b = 0; b < budget && t < v.n; ++b) {
    T sn, cs, ellp;
    T xp[E];
    auto evaluate = [&]() {  // x' on the ellipse at th, and log f(x')
      ess_sincos<T>(th, sn, cs);
#pragma unroll
      for (int e = 0; e < E; ++e) xp[e] = fma(x[e], cs, nu[e] * sn);
      ellp = ess_loglik<T, G, E>(v.tg, xp, lane, yv, gmask);
    };
    if (st == ESS_INIT) {
      if (t >= hi) break;  // direction not generated yet
      load_nu();
      const P4 r = pc.fetch(key, t, D, 0, lane, gmask);
      logy = ess_threshold<T>(ell, Conv<T>::log_u(r.w0, r.w1));
      th = T(kTwoPi) * Conv<T>::u(r.w2, r.w3);
      thmin = th - T(kTwoPi);
      thmax = th;
      s = 0;
    } else {
      if (th < T(0)) thmin = th; else thmax = th;
      const P4 r = pc.fetch(key, t, D, 1 + s, lane, gmask);
      th = thmin + (thmax - thmin) * Conv<T>::u(r.w0, r.w1);
      ++s;
    }
    if constexpr (!AMORT) {
      // the other state's call, at the bracket's other end (masked)
      const T th_real = th;
      th = th < T(0) ? thmax : thmin;
      evaluate();
      ess_keep<T>(ellp);
      th = th_real;
    }
    evaluate();
    if (!(ellp == ellp)) { ellp = neg_inf<T>(); err |= ERR_NONFINITE; }
    ++steps;
    const bool accept = ellp > logy;
    if (accept || s >= kMaxShrinks) {
      if (accept) {
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = xp[e];
        ell = ellp;
      } else {
        err |= ERR_SHRINK_CAP;
      }
      ess_emit<T, G, E>(v, c, t, lane, x);
      if (lane == 0) v.counts[(size_t)c * v.n + t] = s;
      ++t;
      if (++slot == v.W) slot = 0;
      st = ESS_INIT;
      if (t == v.n && lane == 0) atomicAdd(v.chains_done, 1);
    } else {
      st = ESS_SHRINK;
    }
  }
#pragma unroll
  for (int e = 0; e < E; ++e) { const int k = e * G + lane; if (k < d) v.x[(size_t)c * d + k] = x[e]; }
  if (lane == 0) {
    v.ell[c] = ell; v.logy[c] = logy; v.th[c] = th; v.thmin[c] = thmin; v.thmax[c] = thmax;
    v.t[c] = t; v.k[c] = st; v.s[c] = s;
    v.steps[c] += steps;
    if (v.own_window) {
      v.gen_lo[c] = hi;
      v.gen_hi[c] = min(t + v.W, v.n);
    }
    if (err) atomicOr(v.err, err);
  }
}

// Moments-only single-precision GP-logit jobs sum each lane's samples in blocks of up to
// kEssMomBlock: the plain partial sums of x and x^2 over the current block sit in a shared-memory
// slot of kEssMomSlot(E) floats, [2][E], and are folded into the compensated sums in device memory
// (v.mom: sum, compensation, sum of squares, compensation) when the block is full and when the
// chain leaves the launch.  A partial of 16 terms has relative error ~1e-6, well inside what the
// compensated sum keeps.  An even stride, so that coordinate pairs move as 8-byte words (two
// wavefronts per warp access, the minimum for 8-byte words).
template <int E>
constexpr int kEssMomSlot = 2 * E + 2;
constexpr int kEssMomBlock = 16;

// The compensated (Kahan) update of kahan_add for a coordinate pair, in packed single-precision
// instructions: x - c and (t - s) - y are taken as fma(c, -1, x) and fma(y, -1, t - s) (exact
// negations), each one correctly rounded operation.
__device__ __forceinline__ void kahan_add2(float2& sum, float2& comp, float2 x) {
  const float2 neg1 = make_float2(-1.f, -1.f);
  const float2 y = __ffma2_rn(comp, neg1, x);
  const float2 t = __fadd2_rn(sum, y);
  comp = __ffma2_rn(y, neg1, __ffma2_rn(sum, neg1, t));
  sum = t;
}

// Single-precision GP-logit: the lanes hold only the sign-folded coordinates xs = -s x and
// ns = -s nu (exact; bit e of smask marks the coordinates whose sign is flipped), so the
// likelihood is one multiply-add per coordinate (ess_loglik_gp32), the accepted state is
// xs' = xs cos + ns sin (exactly -s x'), and x is recovered exactly for the emitted samples.
// FULL: d = E * G (no ragged lanes).
// PF (32-lane groups, FULL, E a multiple of 4): the direction of sample t + 1 is copied into the
// group's shared-memory row `pf` (cp.async, 16 bytes per copy, L2 only) when sample t starts,
// so that its ring row is on chip when t + 1 starts.  Only samples below gen_hi, whose
// directions were generated before this launch, are copied.
// MOMC (moments-only jobs): the lane's partial sums over the current block of samples are held
// in its shared-memory slot mslot (kEssMomSlot) and folded into the compensated sums in device
// memory every kEssMomBlock samples and when the chain leaves the launch.
// Loop form: every pass evaluates one angle (one FSM state); the state that follows is set up
// in the branch the decision takes -- after DONE the next sample's INIT (threshold, initial
// angle, bracket), after a rejection the SHRINK (bracket end, new angle) -- so a state costs
// one decision branch.  A launch that ends after a rejection leaves the chain in SHRINK with
// the rejected angle, as the state machine's SHRINK expects it.
template <int G, int E, bool FULL, bool PF = false, bool MOMC = false>
__device__ __forceinline__ void ess_advance_chain_gp(const EssView<float>& v, int64_t c, int budget, int lane,
                                                     float* pf = nullptr, float* mslot = nullptr) {
  static_assert(!PF || (G == 32 && FULL && E % 4 == 0), "prefetch needs full 32-lane rows");
  const int d = FULL ? E * G : v.tg.d;
  int mom_pending = 0;  // samples in the current block of partial sums (MOMC)
  // the block's partial sums into the compensated sums in device memory, the partials cleared
  auto mom_flush = [&]() {
    if constexpr (MOMC && E % 2 == 0) {
      float* m0 = v.mom + (size_t)c * d + lane;
#pragma unroll
      for (int e = 0; e < E; e += 2) {
        float2* sp = reinterpret_cast<float2*>(mslot + e);
        const size_t k0 = (size_t)e * G, k1 = k0 + G;
        float2 s1 = make_float2(m0[k0], m0[k1]);
        float2 c1 = make_float2(m0[v.mom_stride + k0], m0[v.mom_stride + k1]);
        float2 s2 = make_float2(m0[2 * v.mom_stride + k0], m0[2 * v.mom_stride + k1]);
        float2 c2 = make_float2(m0[3 * v.mom_stride + k0], m0[3 * v.mom_stride + k1]);
        kahan_add2(s1, c1, sp[0]);
        kahan_add2(s2, c2, sp[E / 2]);
        m0[k0] = s1.x; m0[k1] = s1.y;
        m0[v.mom_stride + k0] = c1.x; m0[v.mom_stride + k1] = c1.y;
        m0[2 * v.mom_stride + k0] = s2.x; m0[2 * v.mom_stride + k1] = s2.y;
        m0[3 * v.mom_stride + k0] = c2.x; m0[3 * v.mom_stride + k1] = c2.y;
        sp[0] = make_float2(0.f, 0.f);
        sp[E / 2] = make_float2(0.f, 0.f);
      }
    }
  };
  if constexpr (MOMC) {
#pragma unroll
    for (int e = 0; e < 2 * E; ++e) mslot[e] = 0.f;
  }
  const int D = (d + 3) / 4;  // Philox blocks of z (four normals each)
  const unsigned gmask = group_mask<G>();
  float xs[E], ns[E];
  uint32_t smask = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = e * G + lane;
    float x = 0.f;
    if (FULL || k < d) {
      x = v.x[(size_t)c * d + k];
      if (v.tg.vec[k] > 0.f) smask |= 1u << e;
    }
    xs[e] = flip_sign(x, smask, e);
    ns[e] = 0.f;
  }
  float ell = v.ell[c], logy = v.logy[c], th = v.th[c], thmin = v.thmin[c], thmax = v.thmax[c];
  int t = v.t[c], st = v.k[c], s = v.s[c];
  const int hi = v.gen_hi[c];
  const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
  int slot = t % v.W;  // ring slot of sample t, advanced with t
  int pf_t = -1;  // sample whose direction is in pf (copy issued)
  // the chain's rows: direction ring (sign-folded, ess_ring_folded), samples, loop counts
  const float* ring_c = v.nu + (size_t)c * v.W * v.dstride;
  float* out_c = v.out ? v.out + (size_t)c * v.n * d : nullptr;
  int* counts_c = v.counts + (size_t)c * v.n;
  auto load_nu = [&]() {
    if constexpr (PF) {
      if (pf_t == t) {
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncwarp();
#pragma unroll
        for (int e = 0; e < E; ++e) ns[e] = pf[e * G + lane];
        return;
      }
    }
    const float* src = ring_c + (size_t)slot * v.dstride;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = e * G + lane;
      if (FULL || k < d) ns[e] = src[k];
    }
  };
  UniformLaneCache<G> pc;
  int b = 0;     // states evaluated in this launch
  int lim2 = 0;  // shrink offsets below lim2 need neither a cache refill nor a budget check
  // INIT of sample t, the (b+1)-th state of this launch
  auto init = [&]() {
    load_nu();
    if constexpr (PF) {
      if (t + 1 < hi && b + 1 < budget) {
        __syncwarp();  // every lane has read pf
        const int nslot = slot + 1 == v.W ? 0 : slot + 1;
        const float* src = ring_c + (size_t)nslot * v.dstride;
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(pf);
#pragma unroll
        for (int j = 0; j < E / 4; ++j) {
          const int q = (j * G + lane) * 4;
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 4u * (uint32_t)q), "l"(src + q)
                       : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        pf_t = t + 1;
      }
    }
    const float2 u = pc.init_ab(key, t, D, lane, gmask);
    logy = ess_threshold<float>(ell, Conv<float>::log_of(u.x));
    th = float(kTwoPi) * u.y;
    thmin = th - float(kTwoPi);
    thmax = th;
    s = 0;
    lim2 = min(pc.lim, budget - b);
  };
  // SHRINK at offset off = 1 + s < lim2: the bracket end moves to the rejected angle th and a new
  // angle is drawn inside
  auto shrink = [&](int off) {
    if (th < 0.f) thmin = th; else thmax = th;
    th = thmin + (thmax - thmin) * pc.shrink_a(key, t, D, off, lane, gmask);
    ++s;
  };
  // Before the shrink at offset off >= lim2: the launch's budget is spent (returns false) or the
  // cache window ends (refilled).  b and off grow together through a sample's shrinks, so
  // b == budget exactly when off reaches budget - b + off, the bound lim2 folds in; one
  // comparison per SHRINK state then covers both.
  auto refill = [&](int off) {
    if (b == budget) return false;
    pc.refill(key, t, D, off, lane);
    lim2 = min(pc.lim, budget - b + off);
    return true;
  };
  int err = 0;
  bool run = t < v.n && budget > 0;
  if (run) {
    if (st == ESS_INIT) {
      run = t < hi;  // else the direction is not generated yet
      if (run) init();
    } else {
      load_nu();
      refill(1 + s);
      shrink(1 + s);
    }
  }
  while (run) {
    float sn, cs;
    ess_sincos<float>(th, sn, cs);
    const float ellp = ess_loglik_gp32<G, E, FULL>(xs, ns, cs * kLog2ef, sn * kLog2ef, lane, d, gmask);
    ++b;
    const bool accept = ellp > logy;
    if (accept || s >= kMaxShrinks) {
      if (accept) {
        if constexpr (E % 2 == 0) {
          const float2 c2 = make_float2(cs, cs), s2 = make_float2(sn, sn);
#pragma unroll
          for (int e = 0; e < E; e += 2) {
            const float2 r = __ffma2_rn(make_float2(xs[e], xs[e + 1]), c2,
                                        __fmul2_rn(make_float2(ns[e], ns[e + 1]), s2));
            xs[e] = r.x;
            xs[e + 1] = r.y;
          }
        } else {
#pragma unroll
          for (int e = 0; e < E; ++e) xs[e] = fmaf(xs[e], cs, ns[e] * sn);
        }
        ell = ellp;
      } else {
        // a NaN likelihood (non-finite coordinates) is never above the threshold: such a
        // sample ends here, at the shrink cap
        err |= ellp == ellp ? ERR_SHRINK_CAP : ERR_SHRINK_CAP | ERR_NONFINITE;
      }
      float x[E];
#pragma unroll
      for (int e = 0; e < E; ++e) x[e] = flip_sign(xs[e], smask, e);
      if (out_c) {
        float* dst = out_c + (size_t)t * d;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int k = e * G + lane;
          if (FULL || k < d) dst[k] = x[e];
        }
      } else if constexpr (MOMC && E % 2 == 0) {
        // the pair (e, e + 1) of each sum as one 8-byte word of the slot: into the block's
        // partial sums, which join the compensated sums every kEssMomBlock samples
#pragma unroll
        for (int e = 0; e < E; e += 2) {
          const float2 xv = make_float2(x[e], x[e + 1]);
          float2* sp = reinterpret_cast<float2*>(mslot + e);
          sp[0] = __fadd2_rn(sp[0], xv);
          sp[E / 2] = __ffma2_rn(xv, xv, sp[E / 2]);
        }
        if (++mom_pending == kEssMomBlock) {
          mom_flush();
          mom_pending = 0;
        }
      } else {
        ess_emit<float, G, E, FULL>(v, c, t, lane, x, MOMC ? mslot : nullptr);
      }
      if (lane == 0) counts_c[t] = s;
      ++t;
      if (++slot == v.W) slot = 0;
      st = ESS_INIT;
      if (t == v.n) {
        if (lane == 0) atomicAdd(v.chains_done, 1);
        break;
      }
      if (b == budget || t >= hi) break;
      init();
    } else {
      st = ESS_SHRINK;
      const int off = 1 + s;
      if (off >= lim2 && !refill(off)) break;
      shrink(off);
    }
  }
  if constexpr (PF) {
    if (pf_t >= 0) asm volatile("cp.async.wait_all;" ::: "memory");  // pf is reused by the next chain
    __syncwarp();
  }
  if constexpr (MOMC) {
    if (mom_pending) mom_flush();
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = e * G + lane;
    if (FULL || k < d) v.x[(size_t)c * d + k] = flip_sign(xs[e], smask, e);
  }
  if (lane == 0) {
    v.ell[c] = ell; v.logy[c] = logy; v.th[c] = th; v.thmin[c] = thmin; v.thmax[c] = thmax;
    v.t[c] = t; v.k[c] = st; v.s[c] = s;
    v.steps[c] += b;
    if (v.own_window) {
      v.gen_lo[c] = hi;
      v.gen_hi[c] = min(t + v.W, v.n);
    }
    if (err) atomicOr(v.err, err);
  }
}

// MODE 0: any target (ess_advance_chain_generic).  MODE 1: single-precision GP-logit
// (ess_advance_chain_gp).  MODE 2: MODE 1 with d = E * G.  MODE 3: any target, log-density
// not amortised (the ablation step form).
template <typename T, int G, int E, int MODE>
__device__ __forceinline__ void ess_advance_chain(const EssView<T>& v, int64_t c, int budget, int lane) {
  if constexpr (MODE == 3) ess_advance_chain_generic<T, G, E, false>(v, c, budget, lane);
  else if constexpr (MODE >= 1 && sizeof(T) == 4) ess_advance_chain_gp<G, E, MODE == 2>(v, c, budget, lane);
  else ess_advance_chain_generic<T, G, E>(v, c, budget, lane);
}

// registers per thread allowed by the launch bounds: three 256-thread blocks per SM for FP32
// rows of up to 8 coordinates per lane (16 on the GP-logit path, which keeps two arrays
// instead of three), two otherwise
template <typename T, int G, int E, int MODE>
__host__ __device__ constexpr int ess_min_blocks() {
  if (sizeof(T) == 4 && (MODE == 1 || MODE == 2) && E <= 8) return 4;
  return ((sizeof(T) == 4 && (E <= 8 || ((MODE == 1 || MODE == 2) && E <= 16))) || (sizeof(T) == 8 && E <= 2)) ? 3
                                                                                                           : 2;
}

// MODE 2 with 32-lane groups and E % 4 == 0 prefetches directions through shared memory
// (one row of d floats per warp; at most 256 threads, 8 warps, per block).
template <typename T, int G, int E, int MODE>
constexpr bool kEssPrefetch = sizeof(T) == 4 && MODE == 2 && G == 32 && E % 4 == 0;

// MOMC (with the prefetch form, moments-only jobs): each thread's running sums in a dynamic
// shared-memory slot of kEssMomSlot<E> floats.
template <typename T, int G, int E, int MODE, bool MOMC = false>
__global__ void __launch_bounds__(256, (ess_min_blocks<T, G, E, MODE>()))
ess_fsm_kernel(EssView<T> v, int budget) {
  const int lane = threadIdx.x % G;
  const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  if constexpr (kEssPrefetch<T, G, E, MODE>) {
    __shared__ __align__(16) float pf_rows[8][E * G];
    float* pf = pf_rows[threadIdx.x / 32];
    if constexpr (MOMC) {
      extern __shared__ __align__(16) float ess_mom_smem[];
      float* mslot = ess_mom_smem + (size_t)threadIdx.x * kEssMomSlot<E>;
      for (int64_t c = group; c < v.m; c += ngroups)
        ess_advance_chain_gp<G, E, true, true, true>(v, c, budget, lane, pf, mslot);
    } else {
      for (int64_t c = group; c < v.m; c += ngroups) ess_advance_chain_gp<G, E, true, true>(v, c, budget, lane, pf);
    }
  } else {
    for (int64_t c = group; c < v.m; c += ngroups) ess_advance_chain<T, G, E, MODE>(v, c, budget, lane);
  }
}

// ---- fused launches over several jobs (serving) --------------------------------------------------
// Job k owns the work items [off[k], off[k+1]) of the flattened range; a block or chain
// group finds its job by binary search.
__device__ __forceinline__ int find_job(const int64_t* off, int njobs, int64_t item) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename T>
__global__ void __launch_bounds__(256) ess_nu_gen_multi_kernel(const EssView<T>* views, const int64_t* off,
                                                               int njobs) {
  const int64_t item = blockIdx.x;
  const int k = find_job(off, njobs, item);
  const EssView<T> v = views[k];
  const int64_t local = item - off[k];
  const int64_t nbx = (v.m + 63) / 64;
  const int64_t per_z = nbx * v.W;
  const int bz = (int)(local / per_z);
  const int by = (int)((local % per_z) / nbx);
  const int64_t bx = local % nbx;
  ess_nu_gen_tile<T>(v, bx, by, bz);
}

template <typename T, int G, int E>
__global__ void __launch_bounds__(256) ess_fsm_multi_kernel(const EssView<T>* views, const int64_t* off,
                                                            int njobs, int64_t total, int budget) {
  const int lane = threadIdx.x % G;
  const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  if (item >= total) return;
  const int k = find_job(off, njobs, item);
  const EssView<T> v = views[k];
  if constexpr (kEssGpFast<T, E>) {
    if (ess_ring_folded(v)) {
      ess_advance_chain<T, G, E, 1>(v, item - off[k], budget, lane);
      return;
    }
  }
  ess_advance_chain<T, G, E, 0>(v, item - off[k], budget, lane);
}

// ------------------------------------------------------------------------------------------
// Synchronised program (Alg. 6, vmap(sample)): for every sample, INIT for all chains, then the
// loop body for all chains still below their threshold, every iteration a grid-wide step, until
// no chain is left in the loop; then the next sample.  Chain state lives in device memory
// between visits.  Three forms run the same visits in the same order per chain, so they give the
// same samples as each other and as the FSM kernels:
//   sweep  (ess_sync_kernel): every group walks all its chains each iteration, skipping those
//          already done -- the masked loop of vmap with the masked work skipped;
//   list   (ess_sync_list_kernel): the chains still in the loop are kept in a compacted list
//          that every group shares, so an iteration's work is spread over the whole grid and
//          costs only the chains that are left plus the barrier;
//   graph  (ess_cg_* kernels in a CUDA graph with conditional while nodes): the same list
//          iterations as separate kernel launches, the loop conditions evaluated on the device,
//          no grid barrier.
// The cooperative kernels are launched with every block resident; barrier waits are bounded.

// One visit of chain c at sample t: INIT (first) or SHRINK, the likelihood of the proposal, DONE
// when it clears the threshold (or at the shrink cap).  Returns true while sample t of the chain
// is still open (the chain stays in the loop).  `ld` is the lane's likelihood data
// (ess_sync_lane_data).
template <typename T, int E>
struct EssLaneData {
  T yv[E];         // y (GAUSS_CONJ) or labels (GP_LOGIT) of the lane's coordinates (generic path)
  uint32_t smask;  // GP-logit path: bit e set where the label of coordinate e is +1
};

template <typename T, int G, int E, bool GP>
__device__ __forceinline__ bool ess_sync_visit(const EssView<T>& v, int64_t c, int t, bool first,
                                               const EssLaneData<T, E>& ld, int lane, unsigned gmask, int& err) {
  const int d = v.tg.d;
  const int D = (d + 3) / 4;  // Philox blocks of z (four normals each)
  const T* src = v.nu + ((size_t)c * v.W + (t % v.W)) * v.dstride;
  // GP path: the sign-folded coordinates xs = -s x, ns = -s nu, as in the FSM kernel
  // (ess_advance_chain_gp; the ring already holds ns, ess_ring_folded); otherwise x and nu
  T xa[E], na[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = e * G + lane;
    const T x = k < d ? v.x[(size_t)c * d + k] : T(0);
    const T nu = k < d ? src[k] : T(0);
    if constexpr (GP) {
      xa[e] = flip_sign(x, ld.smask, e);
      na[e] = nu;
    } else {
      xa[e] = x;
      na[e] = nu;
    }
  }
  const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
  T logy, th, thmin, thmax;
  int s;
  if (first) {  // INIT (S1)
    const P4 r = key.block((uint32_t)t, 0, (uint32_t)D);
    logy = ess_threshold<T>(v.ell[c], Conv<T>::log_u(r.w0, r.w1));
    th = T(kTwoPi) * Conv<T>::u(r.w2, r.w3);
    thmin = th - T(kTwoPi);
    thmax = th;
    s = 0;
  } else {      // SHRINK (S2)
    logy = v.logy[c]; th = v.th[c]; thmin = v.thmin[c]; thmax = v.thmax[c]; s = v.s[c];
    if (th < T(0)) thmin = th; else thmax = th;
    const P4 r = key.block((uint32_t)t, 0, (uint32_t)(D + 1 + s));
    th = thmin + (thmax - thmin) * Conv<T>::u(r.w0, r.w1);
    ++s;
  }
  T sn, cs;
  ess_sincos<T>(th, sn, cs);
  T ellp;
  if constexpr (GP) {
    ellp = ess_loglik_gp32<G, E>(xa, na, cs * kLog2ef, sn * kLog2ef, lane, d, gmask);
  } else {
    T xp[E];
#pragma unroll
    for (int e = 0; e < E; ++e) xp[e] = fma(xa[e], cs, na[e] * sn);
    ellp = ess_loglik<T, G, E>(v.tg, xp, lane, ld.yv, gmask);
  }
  if (!(ellp == ellp)) { ellp = neg_inf<T>(); err |= ERR_NONFINITE; }
  const bool accept = ellp > logy;
  if (accept || s >= kMaxShrinks) {  // DONE (S3)
    T x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      // the accepted point x' = x cos + nu sin (GP path: -s x', exactly, then unfolded)
      const T xn = accept ? fma(xa[e], cs, na[e] * sn) : xa[e];
      if constexpr (GP) x[e] = flip_sign(xn, ld.smask, e);
      else x[e] = xn;
      const int k = e * G + lane;
      if (accept && k < d) v.x[(size_t)c * d + k] = x[e];
    }
    if (!accept) err |= ERR_SHRINK_CAP;
    ess_emit<T, G, E>(v, c, t, lane, x);
    if (lane == 0) {
      if (accept) v.ell[c] = ellp;
      v.counts[(size_t)c * v.n + t] = s;
      v.k[c] = ESS_INIT;
      v.t[c] = t + 1;
      v.steps[c] += 1;
      if (t + 1 == v.n) atomicAdd(v.chains_done, 1);
    }
    return false;
  }
  if (lane == 0) {
    v.logy[c] = logy; v.th[c] = th; v.thmin[c] = thmin; v.thmax[c] = thmax; v.s[c] = s;
    v.k[c] = ESS_SHRINK;
    v.steps[c] += 1;
  }
  return true;
}

// the likelihood's per-lane data: y (GAUSS_CONJ) or the labels (GP_LOGIT); the GP-logit path keeps
// only the labels' signs
template <typename T, int G, int E, bool GP>
__device__ __forceinline__ EssLaneData<T, E> ess_sync_lane_data(const EssView<T>& v, int lane) {
  EssLaneData<T, E> ld;
  ld.smask = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = e * G + lane;
    const T y = (k < v.tg.d && v.tg.vec) ? v.tg.vec[k] : T(0);
    if constexpr (GP) {
      if (y > T(0)) ld.smask |= 1u << e;
      ld.yv[e] = T(0);
    } else {
      ld.yv[e] = y;
    }
  }
  return ld;
}

// registers per thread for the synchronised kernels: three 256-thread blocks per SM in single
// precision (85 registers), two in double
template <typename T>
__host__ __device__ constexpr int ess_sync_min_blocks() { return sizeof(T) == 4 ? 3 : 2; }

// Sweep form.  Chains are assigned statically to groups.
template <typename T, int G, int E, bool GP>
__global__ void __launch_bounds__(256, (ess_sync_min_blocks<T>())) ess_sync_kernel(EssView<T> v, int t_begin, int t_end,
                                                       GridBarrier bar, unsigned* active_cnt,
                                                       unsigned long long* iterations) {
  const int lane = threadIdx.x % G;
  const unsigned gmask = group_mask<G>();
  const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  __shared__ unsigned blk_active;
  int iter = 0;
  int err = 0;
  const EssLaneData<T, E> ld = ess_sync_lane_data<T, G, E, GP>(v, lane);

  // With at most 32 chains per group, the group keeps a bit mask of its chains still in the loop
  // (bit j: chain group + j ngroups), so a finished chain costs nothing in later iterations;
  // otherwise it reads each chain's state id.
  const bool use_mask = v.m <= 32 * ngroups;
  for (int t = t_begin; t < t_end; ++t) {
    bool first = true;
    unsigned live = 0;
    while (true) {
      if (threadIdx.x == 0) blk_active = 0;
      __syncthreads();
      unsigned my_active = 0;
      unsigned next = 0;
      int j = 0;
      for (int64_t c = group; c < v.m; c += ngroups, ++j) {
        // masked: already done with sample t
        const bool open = first || (use_mask ? ((live >> j) & 1u) != 0 : v.k[c] == ESS_SHRINK);
        if (open && ess_sync_visit<T, G, E, GP>(v, c, t, first, ld, lane, gmask, err)) {
          my_active = 1;
          if (use_mask) next |= 1u << j;
        }
      }
      live = next;
      if (my_active && lane == 0) atomicAdd(&blk_active, 1u);
      __syncthreads();
      // whether any chain stays in the loop: a flag that blocks with live chains set (a store,
      // not an atomic: only its being non-zero is read)
      const int slot = iter % 3;
      if (threadIdx.x == 0 && blk_active) *(volatile unsigned*)&active_cnt[slot] = 1u;
      if (!grid_sync(bar, v.err)) return;
      const unsigned total = read_after_grid_sync(&active_cnt[slot]);
      if (leader) {
        active_cnt[(iter + 2) % 3] = 0;  // last read one iteration ago, next written in two
        if (!first) *iterations += 1;    // one loop-body iteration of the batched while
      }
      ++iter;
      first = false;
      if (total == 0) break;
    }
  }
  if (err && lane == 0) atomicOr(v.err, err);
}

// One visit of a resident chain: INIT (first) or SHRINK, the proposal's likelihood, DONE -- the
// arithmetic of ess_sync_visit on the shared-memory copies.  sl: the chain's slot (ns, the
// uniforms, the scalars).  Returns true while sample t is still open.
template <int E>
__device__ __forceinline__ bool ess_res_visit(const EssView<float>& v, int64_t c, int t, bool first, float (&xs)[E],
                                              float* sl, uint32_t smask, int lane, int D, int& err) {
  constexpr int G = 32, d = 32 * E;
  float* ua = sl + 32 * E;
  float* sc = ua + 32;
  const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
  float ns[E];
  float logy, th, thmin, thmax;
  int s;
  if (first) {  // INIT: the sample's direction from its ring row, its uniforms, the bracket
    const float* src = v.nu + ((size_t)c * v.W + (t % v.W)) * v.dstride;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      ns[e] = src[e * G + lane];
      sl[e * G + lane] = ns[e];
    }
    const P4 r = key.block((uint32_t)t, 0, (uint32_t)(D + lane));
    const float a = Conv<float>::u(r.w0, r.w1);
    ua[lane] = a;
    const float a0 = __shfl_sync(0xffffffffu, a, 0);
    const float b0 = __shfl_sync(0xffffffffu, Conv<float>::u(r.w2, r.w3), 0);
    logy = ess_threshold<float>(sc[4], Conv<float>::log_of(a0));
    th = float(kTwoPi) * b0;
    thmin = th - float(kTwoPi);
    thmax = th;
    s = 0;
  } else {      // SHRINK
#pragma unroll
    for (int e = 0; e < E; ++e) ns[e] = sl[e * G + lane];
    logy = sc[0]; th = sc[1]; thmin = sc[2]; thmax = sc[3]; s = __float_as_int(sc[5]);
    if (th < 0.f) thmin = th; else thmax = th;
    const int off = 1 + s;
    float u;
    if (off < 32) {
      u = ua[off];
    } else {
      const P4 r = key.block((uint32_t)t, 0, (uint32_t)(D + off));
      u = Conv<float>::u(r.w0, r.w1);
    }
    th = thmin + (thmax - thmin) * u;
    ++s;
  }
  float sn, cs;
  ess_sincos<float>(th, sn, cs);
  float ellp = ess_loglik_gp32<G, E, true>(xs, ns, cs * kLog2ef, sn * kLog2ef, lane, d, 0xffffffffu);
  if (!(ellp == ellp)) { ellp = neg_inf<float>(); err |= ERR_NONFINITE; }
  const bool accept = ellp > logy;
  __syncwarp();  // every lane has read the slot's scalars
  if (accept || s >= kMaxShrinks) {  // DONE
    float x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const float xn = accept ? fmaf(xs[e], cs, ns[e] * sn) : xs[e];
      xs[e] = xn;
      x[e] = flip_sign(xn, smask, e);
    }
    if (!accept) err |= ERR_SHRINK_CAP;
    ess_emit<float, G, E, true>(v, c, t, lane, x);
    if (lane == 0) {
      if (accept) sc[4] = ellp;
      v.counts[(size_t)c * v.n + t] = s;
      if (t + 1 == v.n) atomicAdd(v.chains_done, 1);
    }
    return false;
  }
  if (lane == 0) {
    sc[0] = logy; sc[1] = th; sc[2] = thmin; sc[3] = thmax; sc[5] = __int_as_float(s);
  }
  return true;
}

// Resident form of the sweep (single-precision GP-logit, 32-lane groups, full rows, d = 32 E):
// each group keeps its chains on chip for the whole launch -- the sign-folded state xs of every
// chain in registers (xs[slot][E]), the current sample's sign-folded direction ns, the sample's
// Philox uniforms (lane l: draw D + l, the uniform a; lane 0 also b) and the bracket in shared
// memory -- so a loop-body visit reads no device memory; the direction of sample t is read from
// its ring row once, at its INIT.  Same visits in the same order as the sweep (same samples, loop
// counts and iteration counts); the state goes back to device memory when the launch ends.
// Slots: chain group + j ngroups for j < kEssResSlots; a launch needs m <= kEssResSlots ngroups.
constexpr int kEssResSlots = 8;
constexpr int kEssResScalars = 8;  // per slot: logy, th, thmin, thmax, ell, s, pad, visits

template <int E>
__host__ __device__ constexpr size_t ess_res_slot_floats() { return (size_t)32 * E + 32 + kEssResScalars; }

template <int E>
__global__ void __launch_bounds__(256, 2) ess_sync_resident_kernel(EssView<float> v, int t_begin, int t_end,
                                                                   GridBarrier bar, unsigned* active_cnt,
                                                                   unsigned long long* iterations) {
  constexpr int G = 32, d = 32 * E;
  extern __shared__ __align__(16) float res_smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  const int D = (d + 3) / 4;
  float* wbase = res_smem + (size_t)warp * kEssResSlots * ess_res_slot_floats<E>();
  __shared__ unsigned blk_active;
  int iter = 0, err = 0;
  uint32_t smask = 0;
#pragma unroll
  for (int e = 0; e < E; ++e)
    if (v.tg.vec[e * G + lane] > 0.f) smask |= 1u << e;
  float xs[kEssResSlots][E];
#pragma unroll
  for (int j = 0; j < kEssResSlots; ++j) {
    const int64_t c = group + (int64_t)j * ngroups;
    float* sl = wbase + (size_t)j * ess_res_slot_floats<E>();
    if (lane == 0) sl[32 * E + 32 + 7] = __int_as_float(0);
#pragma unroll
    for (int e = 0; e < E; ++e) xs[j][e] = c < v.m ? flip_sign(v.x[(size_t)c * d + e * G + lane], smask, e) : 0.f;
    if (lane == 0 && c < v.m) sl[32 * E + 32 + 4] = v.ell[c];
  }
  __syncwarp();
  for (int t = t_begin; t < t_end; ++t) {
    bool first = true;
    unsigned live = 0;
    while (true) {
      if (threadIdx.x == 0) blk_active = 0;
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kEssResSlots; ++j) {
        const int64_t c = group + (int64_t)j * ngroups;
        if (c < v.m && (first || ((live >> j) & 1u))) {
          float* sl = wbase + (size_t)j * ess_res_slot_floats<E>();
          if (lane == 0) sl[32 * E + 39] = __int_as_float(__float_as_int(sl[32 * E + 39]) + 1);
          if (ess_res_visit<E>(v, c, t, first, xs[j], sl, smask, lane, D, err)) live |= 1u << j;
          else live &= ~(1u << j);
        }
      }
      if (live && lane == 0) atomicAdd(&blk_active, 1u);
      __syncthreads();
      const int slot = iter % 3;
      if (threadIdx.x == 0 && blk_active) *(volatile unsigned*)&active_cnt[slot] = 1u;
      if (!grid_sync(bar, v.err)) return;
      const unsigned total = read_after_grid_sync(&active_cnt[slot]);
      if (leader) {
        active_cnt[(iter + 2) % 3] = 0;
        if (!first) *iterations += 1;
      }
      ++iter;
      first = false;
      if (total == 0) break;
    }
  }
  // every chain finished samples t_begin .. t_end - 1: its state back to device memory
#pragma unroll
  for (int j = 0; j < kEssResSlots; ++j) {
    const int64_t c = group + (int64_t)j * ngroups;
    if (c < v.m) {
      const float* sl = wbase + (size_t)j * ess_res_slot_floats<E>();
#pragma unroll
      for (int e = 0; e < E; ++e) v.x[(size_t)c * d + e * G + lane] = flip_sign(xs[j][e], smask, e);
      if (lane == 0) {
        v.ell[c] = sl[32 * E + 32 + 4];
        v.t[c] = t_end;
        v.k[c] = ESS_INIT;
        v.steps[c] += (long long)__float_as_int(sl[32 * E + 39]);
      }
    }
  }
  if (err && lane == 0) atomicOr(v.err, err);
}

// List form.  Iteration `it` (counted over the whole launch) appends the chains that stay in the
// loop to list it % 2 with counter it % 3; after the barrier every group reads that counter and
// takes list entries i = group, group + ngroups, ...  The leader clears counter (it + 2) % 3,
// whose last reads happened before this barrier and whose next appends come after the next one.
// lists: [2][m] chain indices.
template <typename T, int G, int E, bool GP>
__global__ void __launch_bounds__(256, (ess_sync_min_blocks<T>())) ess_sync_list_kernel(EssView<T> v, int t_begin, int t_end,
                                                            GridBarrier bar, unsigned* cnt, int* lists,
                                                            unsigned long long* iterations) {
  const int lane = threadIdx.x % G;
  const unsigned gmask = group_mask<G>();
  const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  int it = 0;
  int err = 0;
  const EssLaneData<T, E> ld = ess_sync_lane_data<T, G, E, GP>(v, lane);
  for (int t = t_begin; t < t_end; ++t) {
    // INIT of every chain
    int* out = lists + (size_t)(it & 1) * v.m;
    for (int64_t c = group; c < v.m; c += ngroups) {
      if (ess_sync_visit<T, G, E, GP>(v, c, t, true, ld, lane, gmask, err) && lane == 0)
        out[atomicAdd(&cnt[it % 3], 1u)] = (int)c;
    }
    while (true) {
      if (!grid_sync(bar, v.err)) return;
      const unsigned n_act = read_after_grid_sync(&cnt[it % 3]);
      const int* in = lists + (size_t)(it & 1) * v.m;
      if (leader) cnt[(it + 2) % 3] = 0;
      ++it;
      if (n_act == 0) break;
      if (leader) *iterations += 1;  // one loop-body iteration of the batched while
      out = lists + (size_t)(it & 1) * v.m;
      for (int64_t i = group; i < (int64_t)n_act; i += ngroups) {
        const int64_t c = in[i];
        if (ess_sync_visit<T, G, E, GP>(v, c, t, false, ld, lane, gmask, err) && lane == 0)
          out[atomicAdd(&cnt[it % 3], 1u)] = (int)c;
      }
    }
  }
  if (err && lane == 0) atomicOr(v.err, err);
}

// Graph form: device-side state of the loops.  The kernels below run one after another in a
// graph (no barrier inside a launch).  The last block of the INIT and iteration kernels to finish
// (counted in blocks_done) evaluates the inner while condition; ess_cg_next_kernel the outer one.
struct EssCgState {
  int t;                // current sample
  int t_end;            // samples of this graph launch end here
  int phase;            // list / counter the next iteration reads
  unsigned blocks_done; // blocks of the running kernel that have finished
  unsigned cnt[2];      // appended chains per list
};

// Run by the last block of a kernel to finish: after INIT (init = 1) the list just written is the
// first iteration's input; after an iteration it becomes the next one's, the consumed list is
// cleared, and one loop-body iteration is counted.  The inner loop continues while the input list
// is not empty.
__device__ __forceinline__ void ess_cg_finish(EssCgState* st, bool init, cudaGraphConditionalHandle inner,
                                              unsigned long long* iterations) {
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();  // this block's appends before its count
    last = atomicAdd(&st->blocks_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();    // every block's appends are visible from here
  st->blocks_done = 0;
  const int p = st->phase;
  if (init) {
    cudaGraphSetConditional(inner, *(volatile unsigned*)&st->cnt[p] > 0 ? 1u : 0u);
    return;
  }
  *iterations += 1;
  st->cnt[p] = 0;
  st->phase = p ^ 1;
  cudaGraphSetConditional(inner, *(volatile unsigned*)&st->cnt[p ^ 1] > 0 ? 1u : 0u);
}

// INIT of every chain at sample st->t; the chains that stay in the loop go to list st->phase.
template <typename T, int G, int E, bool GP>
__global__ void __launch_bounds__(256, (ess_sync_min_blocks<T>())) ess_cg_init_kernel(EssView<T> v, EssCgState* st, int* lists,
                                                          cudaGraphConditionalHandle inner,
                                                          unsigned long long* iterations) {
  const int lane = threadIdx.x % G;
  const unsigned gmask = group_mask<G>();
  const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const int t = st->t, p = st->phase;
  int err = 0;
  const EssLaneData<T, E> ld = ess_sync_lane_data<T, G, E, GP>(v, lane);
  int* out = lists + (size_t)p * v.m;
  for (int64_t c = group; c < v.m; c += ngroups)
    if (ess_sync_visit<T, G, E, GP>(v, c, t, true, ld, lane, gmask, err) && lane == 0)
      out[atomicAdd(&st->cnt[p], 1u)] = (int)c;
  if (err && lane == 0) atomicOr(v.err, err);
  ess_cg_finish(st, true, inner, iterations);
}

// One loop-body iteration over list st->phase; the chains that stay go to the other list.
template <typename T, int G, int E, bool GP>
__global__ void __launch_bounds__(256, (ess_sync_min_blocks<T>())) ess_cg_iter_kernel(EssView<T> v, EssCgState* st, int* lists,
                                                          cudaGraphConditionalHandle inner,
                                                          unsigned long long* iterations) {
  const int lane = threadIdx.x % G;
  const unsigned gmask = group_mask<G>();
  const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const int t = st->t, p = st->phase;
  const int64_t n_act = st->cnt[p];
  int err = 0;
  const EssLaneData<T, E> ld = ess_sync_lane_data<T, G, E, GP>(v, lane);
  const int* in = lists + (size_t)p * v.m;
  int* out = lists + (size_t)(p ^ 1) * v.m;
  for (int64_t i = group; i < n_act; i += ngroups) {
    const int64_t c = in[i];
    if (ess_sync_visit<T, G, E, GP>(v, c, t, false, ld, lane, gmask, err) && lane == 0)
      out[atomicAdd(&st->cnt[p ^ 1], 1u)] = (int)c;
  }
  if (err && lane == 0) atomicOr(v.err, err);
  ess_cg_finish(st, false, inner, iterations);
}

// After a sample: the next one, while samples remain; its INIT writes list st->phase, cleared here.
static __global__ void ess_cg_next_kernel(EssCgState* st, cudaGraphConditionalHandle outer) {
  st->cnt[st->phase] = 0;
  st->t += 1;
  cudaGraphSetConditional(outer, st->t < st->t_end ? 1u : 0u);
}

static __global__ void ess_cg_begin_kernel(EssCgState* st, int t_begin, int t_end) {
  st->t = t_begin;
  st->t_end = t_end;
  st->phase = 0;
  st->blocks_done = 0;
  st->cnt[0] = st->cnt[1] = 0;
}

// log f(x) of every chain's starting point
template <typename T>
__global__ void ess_init_kernel(EssView<T> v) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= v.m) return;
  const int d = v.tg.d;
  T acc = T(0);
  for (int k = 0; k < d; ++k) {
    const T xk = v.x[(size_t)c * d + k];
    if (v.tg.kind == TGT_GP_LOGIT) acc += softplus<T>(-v.tg.vec[k] * xk);
    else if (v.tg.kind == TGT_GAUSS_CONJ) { const T r = v.tg.vec[k] - xk; acc = fma(r, r, acc); }
  }
  T ell = T(0);
  if (v.tg.kind == TGT_GP_LOGIT) ell = -acc;
  else if (v.tg.kind == TGT_GAUSS_CONJ) ell = -acc / (T(2) * v.tg.s2);
  if (!(ell == ell)) { ell = neg_inf<T>(); atomicOr(v.err, ERR_NONFINITE); }
  v.ell[c] = ell;
}

template <typename T>
__global__ void moments_kernel(const T* samples, const int* t, int64_t m, int n, int d, T* out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * d) return;
  const int64_t c = idx / d;
  const int k = (int)(idx % d);
  T s = 0, cs = 0, s2 = 0, c2 = 0;
  const int tc = t[c];
  const T* p = samples + (size_t)c * n * d + k;
  int i = 0;
  for (; i + 8 <= tc; i += 8) {  // eight loads in flight, the sums still taken in sample order
    T x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = p[(size_t)(i + u) * d];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      kahan_add(s, cs, x[u]);
      kahan_add(s2, c2, x[u] * x[u]);
    }
  }
  for (; i < tc; ++i) {
    const T x = p[(size_t)i * d];
    kahan_add(s, cs, x);
    kahan_add(s2, c2, x * x);
  }
  const size_t md = (size_t)m * d;
  out[idx] = s; out[md + idx] = cs; out[2 * md + idx] = s2; out[3 * md + idx] = c2;
}

template <typename T>
cudaError_t launch_moments_from_samples(const T* samples, const int* t, int64_t m, int n, int d, T* out,
                                        cudaStream_t st) {
  const int64_t total = m * d;
  moments_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(samples, t, m, n, d, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}
#if FSMC_ESS_HAS(4)
template cudaError_t launch_moments_from_samples<float>(const float*, const int*, int64_t, int, int, float*,
                                                        cudaStream_t);
#endif

// The sums of x and x^2 ([4][m d] running sums with their compensations) as doubles, [2][m d].
template <typename T>
__global__ void moments_to_double_kernel(const T* mom, int64_t md, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= md) return;
  out[i] = (double)mom[i];
  out[md + i] = (double)mom[2 * md + i];
}

template <typename T>
cudaError_t launch_moments_to_double(const T* mom, int64_t md, double* out, cudaStream_t st) {
  moments_to_double_kernel<T><<<(unsigned)((md + 255) / 256), 256, 0, st>>>(mom, md, out);
  return cudaGetLastError();
}
#if FSMC_ESS_HAS(4)
template cudaError_t launch_moments_to_double<float>(const float*, int64_t, double*, cudaStream_t);
#endif
#if FSMC_ESS_HAS(4)
template cudaError_t launch_moments_to_double<double>(const double*, int64_t, double*, cudaStream_t);
#endif
#if FSMC_ESS_HAS(4)
template cudaError_t launch_moments_from_samples<double>(const double*, const int*, int64_t, int, int, double*,
                                                         cudaStream_t);
#endif

// Refill window of the next pipelined round.  It runs while the FSM kernel of the current
// round advances t, and may read either the old or the new t: the directions it asks for are
// those of samples hi_cur .. t + W - 1, whose ring slots belong to samples below t, which the
// running FSM kernel no longer reads.
template <typename T>
__global__ void ess_window_kernel(EssView<T> v, const int* hi_cur) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= v.m) return;
  const int lo = hi_cur[c];
  const int t = *(volatile const int*)&v.t[c];
  v.gen_lo[c] = lo;
  v.gen_hi[c] = max(lo, min(t + v.W, v.n));
}

template <typename T>
cudaError_t launch_ess_window(const EssView<T>& v, const int* hi_cur, cudaStream_t st) {
  ess_window_kernel<T><<<(unsigned)((v.m + 255) / 256), 256, 0, st>>>(v, hi_cur);
  return cudaGetLastError();
}
#if FSMC_ESS_HAS(4)
template cudaError_t launch_ess_window<float>(const EssView<float>&, const int*, cudaStream_t);
#endif
#if FSMC_ESS_HAS(4)
template cudaError_t launch_ess_window<double>(const EssView<double>&, const int*, cudaStream_t);
#endif

static __global__ void fill_int_kernel(int* p, int64_t n, int value) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = value;
}

template <typename T>
__global__ void from_double_kernel(const double* src, int64_t n, T* dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (T)src[i];
}

template <typename T>
cudaError_t launch_from_double(const double* src, int64_t n, T* dst, cudaStream_t st) {
  from_double_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, n, dst);
  return cudaGetLastError();
}
#if FSMC_ESS_HAS(4)
template cudaError_t launch_from_double<float>(const double*, int64_t, float*, cudaStream_t);
#endif
#if FSMC_ESS_HAS(4)
template cudaError_t launch_from_double<double>(const double*, int64_t, double*, cudaStream_t);
#endif

#if FSMC_ESS_HAS(4)
cudaError_t launch_fill_int(int* p, int64_t n, int value, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  fill_int_kernel<<<(unsigned)blocks, 256, 0, st>>>(p, n, value);
  return cudaGetLastError();
}
#endif

template <typename T>
cudaError_t launch_ess_init(const EssView<T>& v, cudaStream_t st) {
  ess_init_kernel<T><<<(unsigned)((v.m + 127) / 128), 128, 0, st>>>(v);
  return cudaGetLastError();
}
#if FSMC_ESS_HAS(4)
template cudaError_t launch_ess_init<float>(const EssView<float>&, cudaStream_t);
#endif
#if FSMC_ESS_HAS(4)
template cudaError_t launch_ess_init<double>(const EssView<double>&, cudaStream_t);
#endif

// ------------------------------------------------------------------------------------------
// host launchers
template <typename T>
cudaError_t launch_ess_nu_gen(const EssView<T>& v, cudaStream_t st) {
  dim3 grid((unsigned)((v.m + 63) / 64), (unsigned)v.W, (unsigned)((v.tg.d + 255) / 256));
  ess_nu_gen_kernel<T><<<grid, 256, 0, st>>>(v);
  return cudaGetLastError();
}

template <typename T, int G, int E>
static cudaError_t fsm_launch(const EssView<T>& v, int budget, int threads, cudaStream_t st) {
  const int64_t groups_per_block = threads / G;
  const int64_t blocks = (v.m + groups_per_block - 1) / groups_per_block;
  if (v.step_form == 2) {
    ess_fsm_kernel<T, G, E, 3><<<(unsigned)blocks, threads, 0, st>>>(v, budget);
    return cudaGetLastError();
  }
  if constexpr (kEssGpFast<T, E>) {
    if (ess_ring_folded(v)) {
      if (v.tg.d == E * G) {
        const size_t momb = (size_t)threads * kEssMomSlot<E> * sizeof(float);
        if (kEssPrefetch<T, G, E, 2> && !v.out && momb <= 48 * 1024)
          ess_fsm_kernel<T, G, E, 2, true><<<(unsigned)blocks, threads, momb, st>>>(v, budget);
        else
          ess_fsm_kernel<T, G, E, 2><<<(unsigned)blocks, threads, 0, st>>>(v, budget);
      } else {
        ess_fsm_kernel<T, G, E, 1><<<(unsigned)blocks, threads, 0, st>>>(v, budget);
      }
      return cudaGetLastError();
    }
  }
  ess_fsm_kernel<T, G, E, 0><<<(unsigned)blocks, threads, 0, st>>>(v, budget);
  return cudaGetLastError();
}

template <typename T, int G, int E>
static cudaError_t sync_launch(const EssView<T>& v, int t0, int t1, GridBarrier bar,
                               unsigned* active_cnt, unsigned long long* iters, int threads, int form,
                               int* lists, cudaStream_t st) {
  if (form == 4) {  // resident sweep: single-precision GP-logit, 32 lanes, d = 32 E, E <= 8
    if constexpr (sizeof(T) == 4 && G == 32 && E <= 8) {
      if (!ess_ring_folded(v) || v.tg.d != 32 * E) return cudaErrorInvalidValue;
      auto kern = ess_sync_resident_kernel<E>;
      const size_t smem = (size_t)8 * kEssResSlots * ess_res_slot_floats<E>() * sizeof(float);
      cudaError_t e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
      if (e != cudaSuccess) return e;
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      const int64_t need = (v.m + 8 * kEssResSlots - 1) / (8 * kEssResSlots);  // blocks for m chains
      if (per_sm < 1 || need > (int64_t)per_sm * sms) return cudaErrorInvalidValue;
      const int64_t blocks = std::min<int64_t>((int64_t)per_sm * sms, (v.m + 7) / 8);
      EssView<float> vv = v;
      void* args[] = {(void*)&vv, (void*)&t0, (void*)&t1, (void*)&bar, (void*)&active_cnt, (void*)&iters};
      return cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)blocks), dim3(256), args, smem, st);
    } else {
      return cudaErrorInvalidValue;
    }
  }
  void* kern = form == 2 ? (void*)ess_sync_list_kernel<T, G, E, false> : (void*)ess_sync_kernel<T, G, E, false>;
  if constexpr (kEssGpFast<T, E>) {
    if (ess_ring_folded(v))
      kern = form == 2 ? (void*)ess_sync_list_kernel<T, G, E, true> : (void*)ess_sync_kernel<T, G, E, true>;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t groups_per_block = threads / G;
  int64_t blocks = std::min<int64_t>((int64_t)per_sm * sms, (v.m + groups_per_block - 1) / groups_per_block);
  if (blocks < 1) blocks = 1;
  EssView<T> vv = v;
  if (form == 2) {
    void* args[] = {(void*)&vv, (void*)&t0, (void*)&t1, (void*)&bar, (void*)&active_cnt, (void*)&lists,
                    (void*)&iters};
    return cudaLaunchCooperativeKernel(kern, dim3((unsigned)blocks), dim3(threads), args, 0, st);
  }
  void* args[] = {(void*)&vv, (void*)&t0, (void*)&t1, (void*)&bar, (void*)&active_cnt, (void*)&iters};
  return cudaLaunchCooperativeKernel(kern, dim3((unsigned)blocks), dim3(threads), args, 0, st);
}

// The graph form of the synchronised program for samples [t_begin, t_end) of a launch:
//   while (t < t_end) {              -- outer conditional node, condition set by ess_cg_next_kernel
//     init                           -- INIT of every chain; its last block: inner condition =
//                                       list not empty
//     while (list not empty) {       -- inner conditional node
//       iter                         -- one loop-body iteration over the list; its last block
//                                       updates the condition
//     }
//     next                           -- t += 1, outer condition = t < t_end
//   }
// The sample range is read from the EssCgState that ess_cg_begin_kernel writes before each launch,
// so one executable graph serves every chunk of samples of the job.
template <typename T, int G, int E>
static cudaError_t sync_graph_build(const EssView<T>& v, int threads, EssCgState* cg, int* lists,
                                    unsigned long long* iters, cudaGraphExec_t* out) {
  void* kinit = (void*)ess_cg_init_kernel<T, G, E, false>;
  void* kiter = (void*)ess_cg_iter_kernel<T, G, E, false>;
  if constexpr (kEssGpFast<T, E>) {
    if (ess_ring_folded(v)) {
      kinit = (void*)ess_cg_init_kernel<T, G, E, true>;
      kiter = (void*)ess_cg_iter_kernel<T, G, E, true>;
    }
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kinit, threads, 0);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t groups_per_block = threads / G;
  int64_t blocks = std::min<int64_t>((int64_t)std::max(per_sm, 1) * sms, (v.m + groups_per_block - 1) / groups_per_block);
  if (blocks < 1) blocks = 1;

  cudaGraph_t g = nullptr;
  if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return e;
  EssView<T> vv = v;
  auto kernel_node = [&](cudaGraph_t graph, const cudaGraphNode_t* dep, void* fn, dim3 grid, dim3 block,
                         void** args, cudaGraphNode_t* node) {
    cudaKernelNodeParams kp{};
    kp.func = fn;
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    kp.extra = nullptr;
    return cudaGraphAddKernelNode(node, graph, dep, dep ? 1 : 0, &kp);
  };
  auto while_node = [&](cudaGraph_t graph, const cudaGraphNode_t* dep, cudaGraphConditionalHandle h,
                        cudaGraphNode_t* node, cudaGraph_t* body) {
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaError_t r = cudaGraphAddNode(node, graph, dep, nullptr, dep ? 1 : 0, &np);
    if (r == cudaSuccess) *body = np.conditional.phGraph_out[0];
    return r;
  };
  cudaGraphConditionalHandle h_out = 0, h_in = 0;
  cudaGraphNode_t n_out, n_init, n_in, n_next, n_iter;
  cudaGraph_t outer = nullptr, inner = nullptr;
  e = cudaGraphConditionalHandleCreate(&h_out, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) e = while_node(g, nullptr, h_out, &n_out, &outer);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h_in, outer, 0, cudaGraphCondAssignDefault);
  void* a_loop[] = {(void*)&vv, (void*)&cg, (void*)&lists, (void*)&h_in, (void*)&iters};
  void* a_next[] = {(void*)&cg, (void*)&h_out};
  if (e == cudaSuccess) e = kernel_node(outer, nullptr, kinit, dim3((unsigned)blocks), dim3(threads), a_loop, &n_init);
  if (e == cudaSuccess) e = while_node(outer, &n_init, h_in, &n_in, &inner);
  if (e == cudaSuccess) e = kernel_node(outer, &n_in, (void*)ess_cg_next_kernel, dim3(1), dim3(1), a_next, &n_next);
  // after the first iterations few chains are left: one block per SM keeps the launches short
  const int64_t iter_blocks = std::min<int64_t>(blocks, sms);
  if (e == cudaSuccess) e = kernel_node(inner, nullptr, kiter, dim3((unsigned)iter_blocks), dim3(threads), a_loop, &n_iter);
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return e;
}

#define FSMC_ESS_DISPATCH(FN, ...)                                              \
  do {                                                                          \
    const int d = v.tg.d;                                                       \
    if (G == 1) {                                                               \
      if (d <= 2) return FN<T, 1, 2>(__VA_ARGS__);                              \
      if (d <= 4) return FN<T, 1, 4>(__VA_ARGS__);                              \
      if (d <= 8) return FN<T, 1, 8>(__VA_ARGS__);                              \
      if (d <= 16) return FN<T, 1, 16>(__VA_ARGS__);                            \
      if (d <= 32) return FN<T, 1, 32>(__VA_ARGS__);                            \
    } else if (G == 8) {                                                        \
      if (d <= 64) return FN<T, 8, 8>(__VA_ARGS__);                             \
      if (d <= 128) return FN<T, 8, 16>(__VA_ARGS__);                           \
      if (d <= 256) return FN<T, 8, 32>(__VA_ARGS__);                           \
    } else if (G == 16) {                                                       \
      if (d <= 64) return FN<T, 16, 4>(__VA_ARGS__);                            \
      if (d <= 128) return FN<T, 16, 8>(__VA_ARGS__);                           \
      if (d <= 256) return FN<T, 16, 16>(__VA_ARGS__);                          \
      if (d <= 512) return FN<T, 16, 32>(__VA_ARGS__);                          \
    } else if (G == 32) {                                                       \
      if (d <= 32) return FN<T, 32, 1>(__VA_ARGS__);                            \
      if (d <= 64) return FN<T, 32, 2>(__VA_ARGS__);                            \
      if (d <= 128) return FN<T, 32, 4>(__VA_ARGS__);                           \
      if (d <= 256) return FN<T, 32, 8>(__VA_ARGS__);                           \
      if (d <= 512) return FN<T, 32, 16>(__VA_ARGS__);                          \
      if (d <= 1024) return FN<T, 32, 32>(__VA_ARGS__);                         \
    }                                                                           \
    return cudaErrorInvalidValue;                                               \
  } while (0)

template <typename T>
cudaError_t launch_ess_fsm(const EssView<T>& v, int G, int budget, int threads, cudaStream_t st) {
  FSMC_ESS_DISPATCH(fsm_launch, v, budget, threads, st);
}

template <typename T, int G, int E>
static cudaError_t fsm_multi_launch(const EssView<T>& v, const EssView<T>* views, const int64_t* off,
                                    int njobs, int64_t total, int budget, int threads, cudaStream_t st) {
  (void)v;
  const int64_t groups_per_block = threads / G;
  const int64_t blocks = (total + groups_per_block - 1) / groups_per_block;
  ess_fsm_multi_kernel<T, G, E><<<(unsigned)blocks, threads, 0, st>>>(views, off, njobs, total, budget);
  return cudaGetLastError();
}

// `v` is any job of the group (it selects G and E from its d); all jobs share them.
template <typename T>
cudaError_t launch_ess_fsm_multi(const EssView<T>& v, int G, const EssView<T>* views, const int64_t* off,
                                 int njobs, int64_t total, int budget, int threads, cudaStream_t st) {
  FSMC_ESS_DISPATCH(fsm_multi_launch, v, views, off, njobs, total, budget, threads, st);
}

template <typename T>
cudaError_t launch_ess_nu_gen_multi(const EssView<T>* views, const int64_t* off, int njobs,
                                    int64_t total_tiles, cudaStream_t st) {
  if (total_tiles <= 0) return cudaSuccess;
  ess_nu_gen_multi_kernel<T><<<(unsigned)total_tiles, 256, 0, st>>>(views, off, njobs);
  return cudaGetLastError();
}

// shape of the group an ESS job belongs to: jobs with equal (lanes, E) share a fused launch
#if FSMC_ESS_HAS(4)
int ess_group_E(int G, int d) {
  if (G == 1) return d <= 2 ? 2 : d <= 4 ? 4 : d <= 8 ? 8 : d <= 16 ? 16 : 32;
  if (G == 8) return d <= 64 ? 8 : d <= 128 ? 16 : 32;
  if (G == 16) return d <= 64 ? 4 : d <= 128 ? 8 : d <= 256 ? 16 : 32;
  return d <= 32 ? 1 : d <= 64 ? 2 : d <= 128 ? 4 : d <= 256 ? 8 : d <= 512 ? 16 : 32;
}
#endif

template <typename T>
cudaError_t launch_ess_sync(const EssView<T>& v, int G, int t0, int t1, GridBarrier bar,
                            unsigned* active_cnt, unsigned long long* iters, int threads, int form,
                            int* lists, cudaStream_t st) {
  FSMC_ESS_DISPATCH(sync_launch, v, t0, t1, bar, active_cnt, iters, threads, form, lists, st);
}

template <typename T>
cudaError_t build_ess_sync_graph(const EssView<T>& v, int G, int threads, void* cg_state, int* lists,
                                 unsigned long long* iters, cudaGraphExec_t* out) {
  EssCgState* cg = (EssCgState*)cg_state;
  FSMC_ESS_DISPATCH(sync_graph_build, v, threads, cg, lists, iters, out);
}

#if FSMC_ESS_HAS(3)
cudaError_t launch_ess_sync_graph(cudaGraphExec_t exec, void* cg_state, int t0, int t1, cudaStream_t st) {
  ess_cg_begin_kernel<<<1, 1, 0, st>>>((EssCgState*)cg_state, t0, t1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaGraphLaunch(exec, st);
}
#endif

#if FSMC_ESS_HAS(2)
template cudaError_t launch_ess_fsm_multi<float>(const EssView<float>&, int, const EssView<float>*,
                                                 const int64_t*, int, int64_t, int, int, cudaStream_t);
#endif
#if FSMC_ESS_HAS(2)
template cudaError_t launch_ess_fsm_multi<double>(const EssView<double>&, int, const EssView<double>*,
                                                  const int64_t*, int, int64_t, int, int, cudaStream_t);
#endif
#if FSMC_ESS_HAS(4)
template cudaError_t launch_ess_nu_gen_multi<float>(const EssView<float>*, const int64_t*, int, int64_t,
                                                    cudaStream_t);
#endif
#if FSMC_ESS_HAS(4)
template cudaError_t launch_ess_nu_gen_multi<double>(const EssView<double>*, const int64_t*, int, int64_t,
                                                     cudaStream_t);
#endif
#if FSMC_ESS_HAS(4)
template cudaError_t launch_ess_nu_gen<float>(const EssView<float>&, cudaStream_t);
#endif
#if FSMC_ESS_HAS(4)
template cudaError_t launch_ess_nu_gen<double>(const EssView<double>&, cudaStream_t);
#endif
#if FSMC_ESS_HAS(1)
template cudaError_t launch_ess_fsm<float>(const EssView<float>&, int, int, int, cudaStream_t);
#endif
#if FSMC_ESS_HAS(2)
template cudaError_t launch_ess_fsm<double>(const EssView<double>&, int, int, int, cudaStream_t);
#endif
#if FSMC_ESS_HAS(3)
template cudaError_t launch_ess_sync<float>(const EssView<float>&, int, int, int, GridBarrier,
                                            unsigned*, unsigned long long*, int, int, int*, cudaStream_t);
#endif
#if FSMC_ESS_HAS(3)
template cudaError_t launch_ess_sync<double>(const EssView<double>&, int, int, int, GridBarrier,
                                             unsigned*, unsigned long long*, int, int, int*, cudaStream_t);
#endif
#if FSMC_ESS_HAS(3)
template cudaError_t build_ess_sync_graph<float>(const EssView<float>&, int, int, void*, int*,
                                                 unsigned long long*, cudaGraphExec_t*);
#endif
#if FSMC_ESS_HAS(3)
template cudaError_t build_ess_sync_graph<double>(const EssView<double>&, int, int, void*, int*,
                                                  unsigned long long*, cudaGraphExec_t*);
#endif

}  // namespace fsmc
