// Slice sampling (Neal 2003) on a random line through x as a finite state machine.
//
// Fig. 2 ("Slice Sampling") has INIT-E, EXPAND (the stepping-out loop body), INIT-S, SHRINK
// (the shrinkage loop body) and DONE: two while loops in sequence.  One FSM step is the bundled
// and amortised step: it makes exactly one log-density evaluation -- at the left end while
// stepping out to the left, at the right end while stepping out to the right, or at the current
// proposal while shrinking -- and the cheap states (INIT-E, INIT-S, DONE) run inline between
// evaluations.  A sample takes as many steps as it makes evaluations (N_ij).
//
// Stepping out is Neal's procedure with the limit m: the initial interval [L, R] = [-w V, w - w V]
// (along the line, x at 0) is extended by w at most J = floor(m V') times to the left, then at
// most K = m - 1 - J times to the right, each end while it lies inside the slice
// (log pi > log y).  Shrinkage draws theta ~ U(L, R); a proposal outside the slice replaces the
// end on its side of 0.  The direction is u = z / |z|, z ~ N(0, I_d).
//
// Random numbers of sample t (tag 0): draws 0..D-1 the normals z (D = ceil(d/4)); draw D words
// 0-1 the threshold's uniform, words 2-3 V; draw D+1 words 0-1 V'; draw D+2+p proposal p.
#include <algorithm>
#include <cmath>
#include "fsmc_device.cuh"
#include "fsmc_kernels.h"
#include "target_logp.cuh"

namespace fsmc {

enum SliceState : int { SL_START = 0, SL_LEFT = 1, SL_RIGHT = 2, SL_PROP = 3, SL_DONE = 4 };

template <typename T, int E>
struct SliceChain {
  T x[E], u[E];
  T lp, logy, L, R, th;
  int k, J, K, s, nev, t;
};

// log y = log pi(x) + log U.  Single precision keeps the threshold at least one ulp below
// log pi(x): otherwise log U ~ -1e-8 rounds away, and the shrinking interval, whose limit x is
// then not inside the slice, would never accept.
template <typename T>
__device__ __forceinline__ T slice_threshold(T lp, T log_u) {
  T logy = lp + log_u;
  if constexpr (sizeof(T) == 4) {
    if (!(logy < lp) && lp > -INFINITY) logy = nextafterf(lp, -INFINITY);
  }
  return logy;
}

// The random numbers a sample's INIT-E needs -- blocks 0..D-1 (the normals z), D (threshold and
// V) and D+1 (V') of its stream -- drawn ahead of time, one block per FSM step, while the chain
// is still busy with the previous sample: INIT-E then runs in the few threads of a warp whose
// chains just finished a sample, and only the blocks not yet drawn are left for it.  The values
// are those the blocks give whenever they are drawn.
template <typename T, int E>
struct SlicePrefetch {
  T z[E];
  uint32_t w[6];  // block D words 0-3, block D+1 words 0-1
  int q;          // blocks drawn so far
};

template <typename T, int E>
__device__ __forceinline__ void slice_draw_block(const Key& key, int t, int D, SlicePrefetch<T, E>& pf) {
  const P4 b = key.block((uint32_t)t, 0, (uint32_t)pf.q);
  if (pf.q < D) {
    T z[4];
    Conv<T>::normal_quad(b, z);
#pragma unroll
    for (int qq = 0; qq < (E + 3) / 4; ++qq)
      if (qq == pf.q) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (4 * qq + i < E) pf.z[4 * qq + i] = z[i];
      }
  } else if (pf.q == D) {
    pf.w[0] = b.w0; pf.w[1] = b.w1; pf.w[2] = b.w2; pf.w[3] = b.w3;
  } else {
    pf.w[4] = b.w0; pf.w[5] = b.w1;
  }
  ++pf.q;
}

// INIT-S / the next SHRINK proposal: theta ~ U(L, R) from draw D + 2 + s.
template <typename T, int E>
__device__ __forceinline__ void slice_propose(const SliceView<T>& v, const Key& key, SliceChain<T, E>& c) {
  const int D = (v.tg.d + 3) / 4;
  const P4 b = key.block((uint32_t)c.t, 0, (uint32_t)(D + 2 + c.s));
  c.th = c.L + (c.R - c.L) * Conv<T>::u(b.w0, b.w1);
  c.k = SL_PROP;
}

// After the left end: step out to the right while its budget lasts, else start shrinking.
template <typename T, int E>
__device__ __forceinline__ void slice_after_left(const SliceView<T>& v, const Key& key, SliceChain<T, E>& c) {
  if (c.K > 0) c.k = SL_RIGHT;
  else slice_propose<T, E>(v, key, c);
}

// INIT-E: direction, threshold, initial interval and the stepping-out budgets of sample c.t, from
// the prefetched blocks of that sample (the missing ones drawn here); pf then starts on c.t + 1.
template <typename T, int E>
__device__ __forceinline__ void slice_begin(const SliceView<T>& v, const Key& key, SliceChain<T, E>& c,
                                            SlicePrefetch<T, E>& pf) {
  const int d = v.tg.d;
  const int D = (d + 3) / 4;
  while (pf.q < D + 2) slice_draw_block<T, E>(key, c.t, D, pf);
  T ss = T(0);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    c.u[e] = e < d ? pf.z[e] : T(0);
    ss = fma(c.u[e], c.u[e], ss);
  }
  const T rn = T(1) / sqrt(ss);
#pragma unroll
  for (int e = 0; e < E; ++e) c.u[e] *= rn;
  c.logy = slice_threshold<T>(c.lp, Conv<T>::log_u(pf.w[0], pf.w[1]));
  c.L = -v.w * Conv<T>::u(pf.w[2], pf.w[3]);
  c.R = c.L + v.w;
  c.J = min((int)floor(T(v.mlim) * Conv<T>::u(pf.w[4], pf.w[5])), v.mlim - 1);
  c.K = v.mlim - 1 - c.J;
  c.s = 0;
  c.nev = 0;
  pf.q = 0;
  if (c.J > 0) c.k = SL_LEFT;
  else slice_after_left<T, E>(v, key, c);
}

// One FSM step: the log-density at the point the state names, then the state's decision.
// Returns true when the sample is finished (x, lp hold it; after the shrink cap x is kept).
template <typename T, int E>
__device__ __forceinline__ bool slice_step(const SliceView<T>& v, const Key& key, SliceChain<T, E>& c, int& err) {
  const T th = c.k == SL_LEFT ? c.L : c.k == SL_RIGHT ? c.R : c.th;
  T xp[E];
#pragma unroll
  for (int e = 0; e < E; ++e) xp[e] = fma(th, c.u[e], c.x[e]);
  T lpp = full_logp<T, E>(v.tg, xp);
  if (!(lpp == lpp)) { lpp = neg_inf<T>(); err |= ERR_NONFINITE; }
  c.nev += 1;
  const bool inside = lpp > c.logy;
  if (c.k == SL_LEFT) {
    if (inside) {
      c.L -= v.w;
      if (--c.J > 0) return false;
    }
    slice_after_left<T, E>(v, key, c);
    return false;
  }
  if (c.k == SL_RIGHT) {
    if (inside) {
      c.R += v.w;
      if (--c.K > 0) return false;
    }
    slice_propose<T, E>(v, key, c);
    return false;
  }
  c.s += 1;
  if (inside) {
#pragma unroll
    for (int e = 0; e < E; ++e) c.x[e] = xp[e];
    c.lp = lpp;
    return true;
  }
  if (th < T(0)) c.L = th; else c.R = th;
  if (c.s >= kMaxShrinks) {  // keep x
    err |= ERR_SHRINK_CAP;
    return true;
  }
  slice_propose<T, E>(v, key, c);
  return false;
}

// The FSM kernel's form of slice_step (same samples): the state decisions as one instruction
// stream with one place that draws the next shrink proposal's Philox block; in the per-state form
// a warp whose chains sit in different states draws it at up to three places.
template <typename T, int E>
__device__ __forceinline__ bool slice_step_fsm(const SliceView<T>& v, const Key& key, SliceChain<T, E>& c, int& err) {
  const T th = c.k == SL_LEFT ? c.L : c.k == SL_RIGHT ? c.R : c.th;
  T xp[E];
#pragma unroll
  for (int e = 0; e < E; ++e) xp[e] = fma(th, c.u[e], c.x[e]);
  T lpp = full_logp<T, E>(v.tg, xp);
  if (!(lpp == lpp)) { lpp = neg_inf<T>(); err |= ERR_NONFINITE; }
  c.nev += 1;
  const bool inside = lpp > c.logy;
  bool prop = false, fin = false;
  if (c.k != SL_PROP) {  // stepping out: the left end while J lasts, then the right end while K lasts
    const bool left = c.k == SL_LEFT;
    if (inside) {
      if (left) { c.L -= v.w; --c.J; } else { c.R += v.w; --c.K; }
    }
    if (!(inside && (left ? c.J : c.K) > 0)) {
      if (left && c.K > 0) c.k = SL_RIGHT;
      else prop = true;
    }
  } else {
    c.s += 1;
    if (inside) {
#pragma unroll
      for (int e = 0; e < E; ++e) c.x[e] = xp[e];
      c.lp = lpp;
      fin = true;
    } else {
      if (th < T(0)) c.L = th; else c.R = th;
      if (c.s >= kMaxShrinks) {  // keep x
        err |= ERR_SHRINK_CAP;
        fin = true;
      } else {
        prop = true;
      }
    }
  }
  if (prop) slice_propose<T, E>(v, key, c);
  return fin;
}

template <typename T, int E>
__device__ __forceinline__ void slice_load(const SliceView<T>& v, int64_t c, SliceChain<T, E>& s) {
  const int d = v.tg.d;
#pragma unroll
  for (int e = 0; e < E; ++e) s.x[e] = e < d ? v.x[(size_t)c * d + e] : T(0);
  s.lp = v.lp[c];
  s.t = v.t[c];
  s.k = v.k[c];
  if (s.k != SL_START && s.k != SL_DONE) {
#pragma unroll
    for (int e = 0; e < E; ++e) s.u[e] = e < d ? v.u[(size_t)c * d + e] : T(0);
    s.logy = v.logy[c]; s.L = v.L[c]; s.R = v.R[c]; s.th = v.th[c];
    s.J = v.J[c]; s.K = v.K[c]; s.s = v.s[c]; s.nev = v.nev[c];
  }
}

template <typename T, int E>
__device__ __forceinline__ void slice_store(const SliceView<T>& v, int64_t c, const SliceChain<T, E>& s) {
  const int d = v.tg.d;
#pragma unroll
  for (int e = 0; e < E; ++e)
    if (e < d) v.x[(size_t)c * d + e] = s.x[e];
  v.lp[c] = s.lp;
  v.t[c] = s.t;
  v.k[c] = s.k;
  if (s.k != SL_START && s.k != SL_DONE) {
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (e < d) v.u[(size_t)c * d + e] = s.u[e];
    v.logy[c] = s.logy; v.L[c] = s.L; v.R[c] = s.R; v.th[c] = s.th;
    v.J[c] = s.J; v.K[c] = s.K; v.s[c] = s.s; v.nev[c] = s.nev;
  }
}

template <typename T, int E>
__device__ __forceinline__ void slice_finish(const SliceView<T>& v, int64_t c, SliceChain<T, E>& s,
                                             const MomSmem<T, E>& ms = MomSmem<T, E>{nullptr}) {
  chain_emit<T, E>(v, v.tg.d, c, s.t, s.x, ms);
  v.counts[(size_t)c * v.n + s.t] = s.nev;
  v.aux[(size_t)c * v.n + s.t] = s.s;
  s.t += 1;
  if (s.t == v.n) atomicAdd(v.chains_done, 1);
}

// FSM kernel: chain-per-thread, every chain advances `budget` evaluations.
// MOMC: a moments-only job whose chains keep their running sums in dynamic shared memory
// during the launch (MomSmem); the other instantiation updates device memory per sample.
template <typename T, int E, bool MOMC = false>
__global__ void __launch_bounds__(256) slice_fsm_kernel(SliceView<T> v, int budget) {
  extern __shared__ __align__(16) unsigned char slice_mom_smem[];
  const MomSmem<T, E> ms{MOMC ? reinterpret_cast<T*>(slice_mom_smem) + (size_t)threadIdx.x * MomSmem<T, E>::kSlot : nullptr};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < v.m; c += stride) {
    SliceChain<T, E> s;
    slice_load<T, E>(v, c, s);
    if (s.t >= v.n) continue;
    if constexpr (MOMC) mom_smem_load<T, E>(v, v.tg.d, c, ms);
    const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
    const int D = (v.tg.d + 3) / 4;
    int err = 0, steps = 0;
    SlicePrefetch<T, E> pf;
    pf.q = 0;  // for sample t if it has not started, else for t + 1
    if (s.k == SL_START) slice_begin<T, E>(v, key, s, pf);
    for (int b = 0; b < budget; ++b) {
      ++steps;
      if (pf.q < D + 2 && s.t + 1 < v.n) slice_draw_block<T, E>(key, s.t + 1, D, pf);
      if (slice_step_fsm<T, E>(v, key, s, err)) {
        slice_finish<T, E>(v, c, s, ms);
        if (s.t == v.n) { s.k = SL_DONE; break; }
        slice_begin<T, E>(v, key, s, pf);
      }
    }
    slice_store<T, E>(v, c, s);
    v.steps[c] += steps;
    if (err) atomicOr(v.err, err);
    if constexpr (MOMC) mom_smem_store<T, E>(v, v.tg.d, c, ms);
  }
}

// Synchronised kernel (Alg. 6 with two loops in sequence): for every sample, INIT-E for all
// chains; then the left stepping-out loop, the right one and the shrink loop, each iterated with a
// grid barrier until no chain is left in it (chains that left a loop wait, masked).
template <typename T, int E>
__global__ void __launch_bounds__(256) slice_sync_kernel(SliceView<T> v, int t_begin, int t_end,
                                                         GridBarrier bar, unsigned* active_cnt,
                                                         unsigned long long* iterations) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t c_first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  __shared__ unsigned blk_active;
  int iter = 0, err = 0;
  if (stride >= v.m) {
    // At most one chain per thread (the grid covers the job when it fits): the chain's state
    // stays in the thread's registers for the whole launch instead of a device-memory load and
    // store around every loop iteration; same steps in the same order.
    const int64_t c = c_first;
    const bool has = c < v.m;
    SliceChain<T, E> s;
    if (has) slice_load<T, E>(v, c, s);
    const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
    long long steps = 0;
    for (int t = t_begin; t < t_end; ++t) {
      if (has) {
        SlicePrefetch<T, E> pf;
        pf.q = 0;
        slice_begin<T, E>(v, key, s, pf);
      }
      for (int phase = SL_LEFT; phase <= SL_PROP; ++phase) {
        while (true) {
          if (threadIdx.x == 0) blk_active = 0;
          __syncthreads();
          unsigned mine = 0;
          if (has && s.k == phase) {
            ++steps;
            if (slice_step<T, E>(v, key, s, err)) {
              slice_finish<T, E>(v, c, s);
              s.k = SL_DONE;
            }
            if (s.k == phase) mine = 1;
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
    }
    if (has) {
      slice_store<T, E>(v, c, s);
      v.steps[c] += steps;
    }
    if (err) atomicOr(v.err, err);
    return;
  }
  for (int t = t_begin; t < t_end; ++t) {
    for (int64_t c = c_first; c < v.m; c += stride) {
      SliceChain<T, E> s;
      slice_load<T, E>(v, c, s);
      const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
      SlicePrefetch<T, E> pf;
      pf.q = 0;
      slice_begin<T, E>(v, key, s, pf);
      slice_store<T, E>(v, c, s);
    }
    for (int phase = SL_LEFT; phase <= SL_PROP; ++phase) {
      while (true) {
        if (threadIdx.x == 0) blk_active = 0;
        __syncthreads();
        unsigned mine = 0;
        for (int64_t c = c_first; c < v.m; c += stride) {
          if (v.k[c] != phase) continue;  // masked: not in this loop (yet, or any more)
          SliceChain<T, E> s;
          slice_load<T, E>(v, c, s);
          const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
          v.steps[c] += 1;
          if (slice_step<T, E>(v, key, s, err)) {
            slice_finish<T, E>(v, c, s);
            s.k = SL_DONE;
          }
          slice_store<T, E>(v, c, s);
          if (s.k == phase) mine = 1;
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
  }
  if (err) atomicOr(v.err, err);
}

template <typename T, int E>
__global__ void slice_init_kernel(SliceView<T> v) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= v.m) return;
  T x[E];
#pragma unroll
  for (int e = 0; e < E; ++e) x[e] = e < v.tg.d ? v.x[(size_t)c * v.tg.d + e] : T(0);
  T lp = full_logp<T, E>(v.tg, x);
  if (!(lp == lp)) { lp = neg_inf<T>(); atomicOr(v.err, ERR_NONFINITE); }
  v.lp[c] = lp;
  v.k[c] = SL_START;
}

// ---- a chain per warp (32 < d <= 1024) -----------------------------------------------------------
// Lane l holds coordinates k = e 32 + l of x and of the direction u; the density and |z| are warp
// sums, and the chain's scalars (threshold, interval, budgets, counts) are the same in every lane.
// The random numbers are the chain-per-thread sampler's: coordinate k's normal is element k mod 4
// of block floor(k / 4) (each lane draws the Box-Muller pair that holds its coordinate), the
// threshold and V from block D, V' from block D + 1, proposal p from block D + 2 + p.
template <typename T, int E>
__device__ __forceinline__ void slicew_begin(const SliceView<T>& v, const Key& key, SliceChain<T, E>& c,
                                             int lane) {
  const int d = v.tg.d;
  const int D = (d + 3) / 4;
  T ss = T(0);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int kk = e * 32 + lane;
    c.u[e] = T(0);
    if (kk < d) {
      const P4 r = key.block((uint32_t)c.t, 0, (uint32_t)(kk >> 2));
      T z0, z1;
      if ((kk & 3) < 2) Conv<T>::bm(r.w0, r.w1, z0, z1);
      else Conv<T>::bm(r.w2, r.w3, z0, z1);
      c.u[e] = (kk & 1) ? z1 : z0;
    }
    ss = fma(c.u[e], c.u[e], ss);
  }
  const T rn = T(1) / sqrt(group_sum<32>(ss));
#pragma unroll
  for (int e = 0; e < E; ++e) c.u[e] *= rn;
  const P4 b = key.block((uint32_t)c.t, 0, (uint32_t)D);
  const P4 b1 = key.block((uint32_t)c.t, 0, (uint32_t)(D + 1));
  c.logy = slice_threshold<T>(c.lp, Conv<T>::log_u(b.w0, b.w1));
  c.L = -v.w * Conv<T>::u(b.w2, b.w3);
  c.R = c.L + v.w;
  c.J = min((int)floor(T(v.mlim) * Conv<T>::u(b1.w0, b1.w1)), v.mlim - 1);
  c.K = v.mlim - 1 - c.J;
  c.s = 0;
  c.nev = 0;
  if (c.J > 0) c.k = SL_LEFT;
  else slice_after_left<T, E>(v, key, c);
}

template <typename T, int E>
__device__ __forceinline__ bool slicew_step(const SliceView<T>& v, const Key& key, SliceChain<T, E>& c, int lane,
                                            int& err) {
  const T th = c.k == SL_LEFT ? c.L : c.k == SL_RIGHT ? c.R : c.th;
  T xp[E];
#pragma unroll
  for (int e = 0; e < E; ++e) xp[e] = fma(th, c.u[e], c.x[e]);
  T lpp = warp_logp<T, E>(v.tg, xp, lane);
  if (!(lpp == lpp)) { lpp = neg_inf<T>(); err |= ERR_NONFINITE; }
  c.nev += 1;
  const bool inside = lpp > c.logy;
  if (c.k == SL_LEFT) {
    if (inside) {
      c.L -= v.w;
      if (--c.J > 0) return false;
    }
    slice_after_left<T, E>(v, key, c);
    return false;
  }
  if (c.k == SL_RIGHT) {
    if (inside) {
      c.R += v.w;
      if (--c.K > 0) return false;
    }
    slice_propose<T, E>(v, key, c);
    return false;
  }
  c.s += 1;
  if (inside) {
#pragma unroll
    for (int e = 0; e < E; ++e) c.x[e] = xp[e];
    c.lp = lpp;
    return true;
  }
  if (th < T(0)) c.L = th; else c.R = th;
  if (c.s >= kMaxShrinks) {  // keep x
    err |= ERR_SHRINK_CAP;
    return true;
  }
  slice_propose<T, E>(v, key, c);
  return false;
}

template <typename T, int E>
__device__ __forceinline__ void slicew_load(const SliceView<T>& v, int64_t c, SliceChain<T, E>& s, int lane) {
  const int d = v.tg.d;
#pragma unroll
  for (int e = 0; e < E; ++e) s.x[e] = e * 32 + lane < d ? v.x[(size_t)c * d + e * 32 + lane] : T(0);
  s.lp = v.lp[c];
  s.t = v.t[c];
  s.k = v.k[c];
  if (s.k != SL_START && s.k != SL_DONE) {
#pragma unroll
    for (int e = 0; e < E; ++e) s.u[e] = e * 32 + lane < d ? v.u[(size_t)c * d + e * 32 + lane] : T(0);
    s.logy = v.logy[c]; s.L = v.L[c]; s.R = v.R[c]; s.th = v.th[c];
    s.J = v.J[c]; s.K = v.K[c]; s.s = v.s[c]; s.nev = v.nev[c];
  }
}

// every lane writes its coordinates, lane 0 the scalars (after the lanes have read them)
template <typename T, int E>
__device__ __forceinline__ void slicew_store(const SliceView<T>& v, int64_t c, const SliceChain<T, E>& s, int lane) {
  const int d = v.tg.d;
  __syncwarp();
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int k = e * 32 + lane;
    if (k < d) {
      v.x[(size_t)c * d + k] = s.x[e];
      if (s.k != SL_START && s.k != SL_DONE) v.u[(size_t)c * d + k] = s.u[e];
    }
  }
  if (lane == 0) {
    v.lp[c] = s.lp;
    v.t[c] = s.t;
    v.k[c] = s.k;
    if (s.k != SL_START && s.k != SL_DONE) {
      v.logy[c] = s.logy; v.L[c] = s.L; v.R[c] = s.R; v.th[c] = s.th;
      v.J[c] = s.J; v.K[c] = s.K; v.s[c] = s.s; v.nev[c] = s.nev;
    }
  }
  __syncwarp();
}

template <typename T, int E>
__device__ __forceinline__ void slicew_finish(const SliceView<T>& v, int64_t c, SliceChain<T, E>& s, int lane) {
  warp_chain_emit<T, E>(v, v.tg.d, c, s.t, s.x, lane);
  if (lane == 0) {
    v.counts[(size_t)c * v.n + s.t] = s.nev;
    v.aux[(size_t)c * v.n + s.t] = s.s;
  }
  s.t += 1;
  if (s.t == v.n && lane == 0) atomicAdd(v.chains_done, 1);
}

// FSM kernel, a chain per warp, every chain advances `budget` evaluations.
template <typename T, int E>
__global__ void __launch_bounds__(128) slice_fsm_warp_kernel(SliceView<T> v, int budget) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < v.m; c += nwarps) {
    SliceChain<T, E> s;
    slicew_load<T, E>(v, c, s, lane);
    if (s.t >= v.n) continue;
    const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
    int err = 0, steps = 0;
    if (s.k == SL_START) slicew_begin<T, E>(v, key, s, lane);
    for (int b = 0; b < budget; ++b) {
      ++steps;
      if (slicew_step<T, E>(v, key, s, lane, err)) {
        slicew_finish<T, E>(v, c, s, lane);
        if (s.t == v.n) { s.k = SL_DONE; break; }
        slicew_begin<T, E>(v, key, s, lane);
      }
    }
    slicew_store<T, E>(v, c, s, lane);
    if (lane == 0) {
      v.steps[c] += steps;
      if (err) atomicOr(v.err, err);
    }
  }
}

// Synchronised kernel, a chain per warp: as slice_sync_kernel.
template <typename T, int E>
__global__ void __launch_bounds__(128) slice_sync_warp_kernel(SliceView<T> v, int t_begin, int t_end,
                                                              GridBarrier bar, unsigned* active_cnt,
                                                              unsigned long long* iterations) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t c_first = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  __shared__ unsigned blk_active;
  int iter = 0, err = 0;
  for (int t = t_begin; t < t_end; ++t) {
    for (int64_t c = c_first; c < v.m; c += nwarps) {
      SliceChain<T, E> s;
      slicew_load<T, E>(v, c, s, lane);
      const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
      slicew_begin<T, E>(v, key, s, lane);
      slicew_store<T, E>(v, c, s, lane);
    }
    for (int phase = SL_LEFT; phase <= SL_PROP; ++phase) {
      while (true) {
        if (threadIdx.x == 0) blk_active = 0;
        __syncthreads();
        unsigned mine = 0;
        for (int64_t c = c_first; c < v.m; c += nwarps) {
          if (v.k[c] != phase) continue;  // masked: not in this loop (yet, or any more)
          SliceChain<T, E> s;
          slicew_load<T, E>(v, c, s, lane);
          const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
          if (slicew_step<T, E>(v, key, s, lane, err)) {
            slicew_finish<T, E>(v, c, s, lane);
            s.k = SL_DONE;
          }
          slicew_store<T, E>(v, c, s, lane);
          if (lane == 0) v.steps[c] += 1;
          if (s.k == phase) mine = 1;
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
    }
  }
  if (err && lane == 0) atomicOr(v.err, err);
}

template <typename T, int E>
__global__ void slice_init_warp_kernel(SliceView<T> v) {
  const int lane = threadIdx.x & 31;
  const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= v.m) return;
  T x[E];
#pragma unroll
  for (int e = 0; e < E; ++e) x[e] = e * 32 + lane < v.tg.d ? v.x[(size_t)c * v.tg.d + e * 32 + lane] : T(0);
  T lp = warp_logp<T, E>(v.tg, x, lane);
  if (!(lp == lp)) { lp = neg_inf<T>(); if (lane == 0) atomicOr(v.err, ERR_NONFINITE); }
  if (lane == 0) {
    v.lp[c] = lp;
    v.k[c] = SL_START;
  }
}

template <typename T, int E>
static cudaError_t fsm_warp_launch(const SliceView<T>& v, int budget, int threads, cudaStream_t st) {
  const int64_t blocks = (v.m * 32 + threads - 1) / threads;
  slice_fsm_warp_kernel<T, E><<<(unsigned)blocks, threads, 0, st>>>(v, budget);
  return cudaGetLastError();
}

template <typename T, int E>
static cudaError_t sync_warp_launch(const SliceView<T>& v, int t0, int t1, GridBarrier bar, unsigned* active_cnt,
                                    unsigned long long* iters, int threads, cudaStream_t st) {
  auto kern = slice_sync_warp_kernel<T, E>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = std::min<int64_t>((int64_t)per_sm * sms, (v.m * 32 + threads - 1) / threads);
  if (blocks < 1) blocks = 1;
  SliceView<T> vv = v;
  void* args[] = {(void*)&vv, (void*)&t0, (void*)&t1, (void*)&bar, (void*)&active_cnt, (void*)&iters};
  return cudaLaunchCooperativeKernel((void*)kern, dim3((unsigned)blocks), dim3(threads), args, 0, st);
}

template <typename T, int E>
static cudaError_t init_warp_launch(const SliceView<T>& v, cudaStream_t st) {
  slice_init_warp_kernel<T, E><<<(unsigned)((v.m * 32 + 127) / 128), 128, 0, st>>>(v);
  return cudaGetLastError();
}

#define FSMC_SLICE_WARP_DISPATCH(FN, ...)                    \
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
static cudaError_t fsm_launch(const SliceView<T>& v, int budget, int threads, cudaStream_t st) {
  const int64_t blocks = (v.m + threads - 1) / threads;
  const size_t smem = mom_smem_bytes<T, E>(v, threads);
  if (smem) slice_fsm_kernel<T, E, true><<<(unsigned)blocks, threads, smem, st>>>(v, budget);
  else slice_fsm_kernel<T, E><<<(unsigned)blocks, threads, 0, st>>>(v, budget);
  return cudaGetLastError();
}

template <typename T, int E>
static cudaError_t sync_launch(const SliceView<T>& v, int t0, int t1, GridBarrier bar, unsigned* active_cnt,
                               unsigned long long* iters, int threads, cudaStream_t st) {
  auto kern = slice_sync_kernel<T, E>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = std::min<int64_t>((int64_t)per_sm * sms, (v.m + threads - 1) / threads);
  if (blocks < 1) blocks = 1;
  SliceView<T> vv = v;
  void* args[] = {(void*)&vv, (void*)&t0, (void*)&t1, (void*)&bar, (void*)&active_cnt, (void*)&iters};
  return cudaLaunchCooperativeKernel((void*)kern, dim3((unsigned)blocks), dim3(threads), args, 0, st);
}

template <typename T, int E>
static cudaError_t init_launch(const SliceView<T>& v, cudaStream_t st) {
  slice_init_kernel<T, E><<<(unsigned)((v.m + 127) / 128), 128, 0, st>>>(v);
  return cudaGetLastError();
}

#define FSMC_SLICE_DISPATCH(FN, ...)                         \
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
cudaError_t launch_slice_fsm(const SliceView<T>& v, int budget, int threads, cudaStream_t st) {
  if (v.lanes == 32) FSMC_SLICE_WARP_DISPATCH(fsm_warp_launch, v, budget, threads, st);
  FSMC_SLICE_DISPATCH(fsm_launch, v, budget, threads, st);
}
template <typename T>
cudaError_t launch_slice_sync(const SliceView<T>& v, int t0, int t1, GridBarrier bar, unsigned* active_cnt,
                              unsigned long long* iters, int threads, cudaStream_t st) {
  if (v.lanes == 32) FSMC_SLICE_WARP_DISPATCH(sync_warp_launch, v, t0, t1, bar, active_cnt, iters, threads, st);
  FSMC_SLICE_DISPATCH(sync_launch, v, t0, t1, bar, active_cnt, iters, threads, st);
}
template <typename T>
cudaError_t launch_slice_init(const SliceView<T>& v, cudaStream_t st) {
  if (v.lanes == 32) FSMC_SLICE_WARP_DISPATCH(init_warp_launch, v, st);
  FSMC_SLICE_DISPATCH(init_launch, v, st);
}

template cudaError_t launch_slice_fsm<float>(const SliceView<float>&, int, int, cudaStream_t);
template cudaError_t launch_slice_fsm<double>(const SliceView<double>&, int, int, cudaStream_t);
template cudaError_t launch_slice_sync<float>(const SliceView<float>&, int, int, GridBarrier, unsigned*,
                                              unsigned long long*, int, cudaStream_t);
template cudaError_t launch_slice_sync<double>(const SliceView<double>&, int, int, GridBarrier, unsigned*,
                                               unsigned long long*, int, cudaStream_t);
template cudaError_t launch_slice_init<float>(const SliceView<float>&, cudaStream_t);
template cudaError_t launch_slice_init<double>(const SliceView<double>&, cudaStream_t);

}  // namespace fsmc
