// Device building blocks shared by the fsmc kernels: counter-based RNG, uniform and
// normal conversions, chain-group reductions, a bounded grid barrier, and the
// structure-of-arrays job view the kernels read and write.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fsmc {

// ---- error bits written to a job's device error word ---------------------------------
enum : int {
  ERR_SHRINK_CAP = 1,     // an ESS bracket shrank kMaxShrinks times without acceptance
  ERR_BARRIER_TIMEOUT = 2,// a bounded grid-barrier wait expired
  ERR_NONFINITE = 4,      // a non-finite log-density was treated as -inf
};
constexpr int kMaxShrinks = 10000;
constexpr unsigned kBarrierSpinLimit = 1u << 24;  // ~1-2 s of nanosleep(64) polls

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) -----------------------------------
struct P4 { uint32_t w0, w1, w2, w3; };

// Each round takes one 32x32 -> 64-bit product per multiplier (high and low halves together)
// and the round keys are the seed key plus multiples of the Weyl constants.
__device__ __forceinline__ P4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t rk0 = k0 + (uint32_t)r * 0x9E3779B9u;
    const uint32_t rk1 = k1 + (uint32_t)r * 0xBB67AE85u;
    const unsigned long long p0 = (unsigned long long)c0 * 0xD2511F53u;
    const unsigned long long p1 = (unsigned long long)c2 * 0xCD9E8D57u;
    c0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk0;
    c1 = (uint32_t)p1;
    c2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk1;
    c3 = (uint32_t)p0;
  }
  return P4{c0, c1, c2, c3};
}

// Key = (chain, seed_lo); counter = (draw, sample, tag, seed_hi).
struct Key {
  uint32_t chain, seed_lo, seed_hi;
  __device__ __forceinline__ P4 block(uint32_t sample, uint32_t tag, uint32_t draw) const {
    return philox(draw, sample, tag, seed_hi, chain, seed_lo);
  }
};

// Hardware base-2 exponential and logarithm and square root (PTX ex2.approx,
// lg2.approx, sqrt.approx; single precision, relative error ~2^-22).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---- conversions ----------------------------------------------------------------------------
// Uniform in (0,1): u = ((hi:lo >> 12) + 1/2) 2^-52, exact in double.  1 - u is the same map of
// the complemented words, which gives log u accurately near 1 in single precision.
template <typename T> struct Conv;

template <> struct Conv<double> {
  static __device__ __forceinline__ double u(uint32_t hi, uint32_t lo) {
    unsigned long long v = (((unsigned long long)hi << 32) | lo) >> 12;
    return ((double)v + 0.5) * 0x1p-52;
  }
  static __device__ __forceinline__ double log_u(uint32_t hi, uint32_t lo) { return log(u(hi, lo)); }
  // one-word uniform (w + 1/2) 2^-32, exact
  static __device__ __forceinline__ double u32(uint32_t w) { return ((double)w + 0.5) * 0x1p-32; }
  // Box-Muller pair: r = sqrt(-2 ln u32(a)), phi = 2 pi u32(b)
  static __device__ __forceinline__ void bm(uint32_t a, uint32_t b, double& z0, double& z1) {
    const double r = sqrt(-2.0 * log(u32(a)));
    double s, c;
    sincospi(2.0 * u32(b), &s, &c);
    z0 = r * c;
    z1 = r * s;
  }
  // four normals per block: pairs from (w0, w1) and (w2, w3)
  static __device__ __forceinline__ void normal_quad(const P4& b, double (&z)[4]) {
    bm(b.w0, b.w1, z[0], z[1]);
    bm(b.w2, b.w3, z[2], z[3]);
  }
};

template <> struct Conv<float> {
  // single-precision rounding of the same 52-bit uniform (relative error <= 2^-23)
  static __device__ __forceinline__ float u(uint32_t hi, uint32_t lo) {
    return fmaf((float)hi, 0x1p-32f, fmaf((float)(lo >> 12), 0x1p-52f, 0x1p-53f));
  }
  // log u = ln 2 log2 u with lg2.approx: absolute error ~1e-7, which moves a comparison of log u
  // with a log acceptance ratio, or a slice threshold log f + log u, by far less than the FP32
  // rounding of the log-densities involved
  static __device__ __forceinline__ float log_u(uint32_t hi, uint32_t lo) { return log_of(u(hi, lo)); }
  // log of a uniform already converted (the same bits as log_u of its words)
  static __device__ __forceinline__ float log_of(float u) { return lg2_approx(u) * 0.693147180559945309417f; }
  // single-precision rounding of the one-word uniform (w + 1/2) 2^-32
  static __device__ __forceinline__ float u32(uint32_t w) { return fmaf((float)w, 0x1p-32f, 0x1p-33f); }
  // Box-Muller with the hardware approximations: the radius r = sqrt(-2 ln 2 log2 u) from
  // lg2.approx and sqrt.approx (relative error ~2^-22 each), and the angle phi = 2 pi u written
  // as psi + pi with psi in [-pi, pi), where __sincosf is accurate to ~5e-7
  // (cos phi = -cos psi, sin phi = -sin psi).
  static __device__ __forceinline__ void bm(uint32_t a, uint32_t b, float& z0, float& z1) {
    const float r = sqrt_approx(fmaxf(lg2_approx(u32(a)) * -1.38629436111989061883f, 0.f));
    const float psi = fmaf(6.28318530717958647692f, u32(b), -3.14159265358979323846f);
    float s, c;
    __sincosf(psi, &s, &c);
    z0 = -r * c;
    z1 = -r * s;
  }
  // four normals per block: pairs from (w0, w1) and (w2, w3)
  static __device__ __forceinline__ void normal_quad(const P4& b, float (&z)[4]) {
    bm(b.w0, b.w1, z[0], z[1]);
    bm(b.w2, b.w3, z[2], z[3]);
  }
};

// ---- chain-group reductions -------------------------------------------------------------------
// A chain is owned by G consecutive lanes (G = 1 chain-per-thread, G = 16 two chains per warp,
// G = 32 chain-per-warp).  Butterfly sums give every lane of the group the same bits.  `mask`
// names the lanes of the calling group (group_mask<G>()): groups of one warp may be at
// different points of their loops, so a sub-warp group never names the other group's lanes.
template <int G>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (G >= 32) return 0xffffffffu;
  else return ((1u << G) - 1u) << ((threadIdx.x & 31u) & ~(unsigned)(G - 1));
}

template <int G, typename T>
__device__ __forceinline__ T group_sum(T v, unsigned mask = 0xffffffffu) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

// N independent group sums with their shuffles interleaved (each result has group_sum's bits).
template <int G, int N, typename T>
__device__ __forceinline__ void group_sum_n(T (&v)[N], unsigned mask = 0xffffffffu) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
    for (int n = 0; n < N; ++n) v[n] += __shfl_xor_sync(mask, v[n], o);
}


// ---- balanced FSM launch over a resident grid ------------------------------------------------
// An FSM launch runs every unit (a chain, or a group of chains that share a block) for `budget`
// states.  With one unit per worker (warp or block) and more units than workers that can be
// resident (P), a latency-bound launch takes ceil(G / P) waves of time for G / P waves of work
// (NUTS on logistic regression, 4096 chains in 512 blocks of eight, 296 resident: 1.73 waves
// in two).  Instead the grid is P resident workers and each runs its share of the units one
// after another, with the workers' times balanced: for G = a P + r, workers below r take a + 1
// units of `budget` states, the others a units of budget + ceil(budget / a) states.  The order of the units is rotated by rot (sched[0]), which
// the last block of each launch advances by the units that took the longer budget, so that
// every unit takes it in turn.  Which states run in which launch changes no chain's samples.
struct BalancedRun {
  int64_t first, count;  // units first .. first + count - 1 (before rotation)
  int budget;            // states per unit
};
__device__ __forceinline__ BalancedRun balanced_run(int64_t G, int64_t P, int64_t w, int budget) {
  if (G <= P) return BalancedRun{w, w < G ? 1 : 0, budget};
  const int64_t a = G / P, r = G % P;
  if (w < r) return BalancedRun{w * (a + 1), a + 1, budget};
  return BalancedRun{r * (a + 1) + (w - r) * a, a, budget + (int)((budget + a - 1) / a)};
}
// After the block's last unit (every thread of the block calls it): the block's arrival on
// sched[1]; the last of the grid's blocks advances the rotation sched[0].  The next launch on the
// stream reads the new value.
__device__ __forceinline__ void balanced_done(int* sched, int64_t G, int64_t P, int rot) {
  __syncthreads();
  if (threadIdx.x == 0 && G > P) {
    __threadfence();
    if (atomicAdd(&sched[1], 1) == (int)gridDim.x - 1) {
      const int64_t a = G / P, r = G % P;
      sched[1] = 0;
      sched[0] = (int)((rot + (P - r) * a) % G);
    }
  }
}

// ---- bounded grid barrier (cooperative launches only) ----------------------------------------
// Counting barrier in two forms; both count arrivals in count[0] (zeroed by the host before
// every launch, kGridBarrierBytes), so that with n = blocks (+ missing) the arrival that sees
// count = old belongs to barrier k = old / n.
//   kBarCount: every block polls count[0] until it reaches (k + 1) n -- the barrier completes with
//              the last arrival itself.
//   kBarFlag:  the last arrival of barrier k (old = (k + 1) n - 1) bumps a release word on its own
//              128-byte line, count[32], which the others poll; polling then never touches the line
//              the arrivals update.
// Measured on B300 (synchronised kernels, ms per job): the ESS and DR kernels (444 and ~1000
// blocks of 256 / 128 threads, a barrier per loop iteration) are 8-10 % faster with kBarCount;
// the NUTS kernel (a barrier per sub-state of every doubling) 35 % faster with kBarFlag.
// Every wait is bounded: after spin_limit polls (default kBarrierSpinLimit) the block records
// ERR_BARRIER_TIMEOUT and returns false, a block that sees the bit set by another gives up at
// once, and a block that finds it set before arriving leaves without arriving; callers then leave
// the kernel.
constexpr size_t kGridBarrierBytes = 256;
enum BarrierForm : int { kBarCount = 0, kBarFlag = 1 };

struct GridBarrier {
  unsigned* count;  // kGridBarrierBytes: arrivals at word 0, the release word at word 32
  unsigned spin_limit = kBarrierSpinLimit;  // polls before a wait gives up
  unsigned missing = 0;  // test hook: arrivals every wait expects beyond the grid's blocks (0 in
                         // production); with missing > 0 no barrier completes and every wait runs out
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int FORM = kBarCount>
__device__ __forceinline__ bool grid_sync(GridBarrier b, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    if (*(volatile int*)err & ERR_BARRIER_TIMEOUT) {
      ok = 0;  // a wait of this run already gave up: leave without arriving
    } else {
      const unsigned n = gridDim.x * gridDim.y * gridDim.z + b.missing;
      volatile unsigned* rel = b.count + 32;
      const unsigned g = FORM == kBarFlag ? *rel : 0u;
      __threadfence();  // the block's writes (ordered before thread 0 by the block barrier) first
      const unsigned old = atomicAdd(b.count, 1u);
      unsigned spins = 0;
      if (FORM == kBarFlag && old % n == n - 1) {
        __threadfence();
        atomicAdd(b.count + 32, 1u);
      } else {
        const unsigned target = (old / n + 1) * n;
        while (FORM == kBarFlag ? *rel == g : (int)(ld_acquire_gpu(b.count) - target) < 0) {
          if (++spins > b.spin_limit || (*(volatile int*)err & ERR_BARRIER_TIMEOUT)) {
            atomicOr(err, ERR_BARRIER_TIMEOUT);
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
    }
  }
  __syncthreads();
  return ok != 0;
}

// A word every block reads right after a grid barrier (a loop's "any chain left" flag or its
// count), read by thread 0 of the block and handed to the others through shared memory.  Read by
// every thread of every block at once, right after many blocks wrote it, the word's line is a hot
// spot: measured on B300 with 444 blocks of 256 threads, ~14 us per loop iteration against ~0.1
// us for one read per block.  Callers pass a block barrier (the next grid_sync) before calling
// it again, so thread 0 never overwrites the shared copy while another thread still reads it.
__device__ __forceinline__ unsigned read_after_grid_sync(const unsigned* p) {
  __shared__ unsigned shared_copy;
  if (threadIdx.x == 0) shared_copy = *(volatile const unsigned*)p;
  __syncthreads();
  return shared_copy;
}

// ---- device-side target view ---------------------------------------------------------------------
enum TargetKind : int {
  TGT_GAUSS_CONJ = 0, TGT_GP_LOGIT = 1, TGT_FUNNEL = 2, TGT_LOGREG = 3, TGT_GAUSS_DIAG = 4, TGT_FLAT = 5,
  TGT_MOG = 6, TGT_GP_REG = 7
};

template <typename T>
struct TargetView {
  int kind;
  int d;
  int n_data;
  const T* L;     // ESS prior Cholesky [d][d] (lower)
  const T* vec;   // y (GAUSS_CONJ), s (GP_LOGIT), mu (GAUSS_DIAG), y (LOGREG), log w_k (MOG), y (GP_REG)
  const T* vec2;  // sigma (GAUSS_DIAG)
  const T* X;     // LOGREG design matrix [n_data][d]; MOG means mu_k [n_data][d]; GP_REG squared
                  // distances D [n_data][n_data]
  const T* XT;    // LOGREG design matrix transposed, [d][n_pad] with zero rows >= n_data
  int n_pad;      // n_data rounded up to a multiple of 4
  T s2;           // GAUSS_CONJ noise variance
  // MOG: S^-1 = c_par P + c_perp (I - P) with P = 1 1^T / d, so for v = x - mu_k
  // v^T S^-1 v = (1^T v)^2 c_par / d + |v - (1^T v / d) 1|^2 c_perp
  T c_par;        // 1 / (1 + (d - 1) rho): the principal eigenvalue's inverse
  T c_perp;       // 1 / (1 - rho)
};

template <typename T>
__device__ __forceinline__ T softplus(T t) {
  // log(1 + e^t) without overflow.  Single precision uses the hardware exp2/log2
  // approximations: the absolute error per term stays below ~2e-7.
  if constexpr (sizeof(T) == 4) {
    return fmaxf(t, 0.f) + __logf(1.f + __expf(-fabsf(t)));
  } else {
    return t > 0.0 ? t + log1p(exp(-t)) : log1p(exp(t));
  }
}

template <typename T>
__device__ __forceinline__ T neg_inf() { return -(T)INFINITY; }

}  // namespace fsmc
