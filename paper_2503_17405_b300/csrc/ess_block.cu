// Elliptical slice sampling (Alg. 8) for targets whose likelihood is one dense linear-algebra
// problem per evaluation: GP regression's marginal likelihood (Sec. 7.2), where f(x) needs the
// Cholesky factorisation of an n x n covariance built from the hyperparameters x = (sigma, tau,
// lambda).  This is the expensive-log-density regime of Sec. 4 in which the FSM's speed-up E(m)
// approaches R(m): the step is the likelihood.
//
// Layout: one chain per CTA of WPC = 1, 2 or 4 warps (a CTA's shared memory is one chain's
// matrix, and the SM packs as many as fit; WPC grows when there are too few chains to fill the
// SMs).  The threads run the chain's cheap FSM logic redundantly (INIT, SHRINK, DONE; identical
// values in every thread) and evaluate the likelihood together: the lower triangle of the
// covariance, packed by rows in shared memory with y appended as an extra row, is factorised
// C = L diag(d) L^T left-looking, column by column; for column j every row below it takes a dot
// product of length j, the threads taking rows, so the work is balanced, with two barriers per
// column.  The y row comes out as the forward substitution L^-1 y, so log det C = sum log d_j
// and y^T C^-1 y = sum (L^-1 y)_j^2 / d_j.
// The FSM kernel takes chains from an atomic counter, each for `budget` steps; one step is one
// likelihood evaluation (bundled and amortised, as in ess.cu).
#include <algorithm>
#include "ess_common.cuh"
#include "fsmc_device.cuh"
#include "fsmc_kernels.h"

namespace fsmc {

constexpr int kBlkE = 4;  // registers per chain vector (d <= 4)

template <typename T>
__device__ __forceinline__ T blk_exp(T a) { if constexpr (sizeof(T) == 4) return expf(a); else return exp(a); }
template <typename T>
__device__ __forceinline__ T blk_log(T a) { if constexpr (sizeof(T) == 4) return logf(a); else return log(a); }

// Row i of the packed lower triangle (length i + 1) starts at off(i) in shared memory, with gaps
// so that off(i + 1) = off(i) + 17 (mod 32): the threads of a warp read the same column k of 32
// consecutive rows, which then fall in 32 different banks (17 is odd).  Rows r .. n-1 that do
// not fit live in a per-CTA scratch block in device memory (L2-resident: a few hundred KB per
// resident CTA), contiguous; the y row, v, the pivots d, the running sums s and the row offsets
// stay in shared memory.
__host__ __device__ __forceinline__ int row_gap(int i) { return (17 - (i + 1)) & 31; }
__host__ __device__ __forceinline__ size_t gpreg_rows_elems(int r) {
  size_t off = 0;
  for (int i = 0; i < r; ++i) off += (size_t)(i + 1) + row_gap(i);
  return off;
}

constexpr size_t kGpRegSmemBudget = 220 * 1024;

// Shared-memory bytes with the first r rows in shared memory: the rows, the y row, v, d, s (n
// elements each) and the n + 1 row offsets.
template <typename T>
__host__ __device__ __forceinline__ size_t gpreg_smem_bytes_r(int n, int r) {
  return (gpreg_rows_elems(r) + 4 * (size_t)n) * sizeof(T) + ((size_t)n + 1) * sizeof(int);
}

// Rows kept in shared memory: all of them when they fit the budget.
template <typename T>
__host__ __device__ __forceinline__ int gpreg_rows_in_smem(int n) {
  int r = n;
  while (r > 0 && gpreg_smem_bytes_r<T>(n, r) > kGpRegSmemBudget) --r;
  return r;
}

template <typename T>
__host__ __device__ __forceinline__ size_t gpreg_smem_bytes(int n) {
  return gpreg_smem_bytes_r<T>(n, gpreg_rows_in_smem<T>(n));
}

template <int WPC>
__device__ __forceinline__ void cta_sync() {
  if constexpr (WPC == 1) __syncwarp(); else __syncthreads();
}

// log N(y; 0, C), C_ij = tau^2 exp(-lambda^2 D_ij) + sigma^2 delta_ij (x = (sigma, tau, lambda)),
// -inf when a pivot is not positive.  Column j of the left-looking LDL^T:
//   v_k = L_jk d_k (k < j),  d_j = C_jj - s_j,  L_ij = (C_ij - sum_k L_ik v_k) / d_j,
// for the rows i > j and the y row (whose entries become (L^-1 y)_j / d_j; the numerator is
// (L^-1 y)_j), where s_i = sum_{k<j} L_ik^2 d_k is kept per row by the thread that computes L_ij
// (so d_j needs no reduction).  Storage: M[i][j] = L_ij, d and s in their own arrays.  Every
// thread returns the same value.
// Dot product sum_{k<j} r[k] v[k] subtracted from r[j] (4 accumulators).
template <typename T>
__device__ __forceinline__ T row_residual(const T* r, const T* V, int j) {
  T a0 = r[j], a1 = T(0), a2 = T(0), a3 = T(0);
  int k = 0;
  for (; k + 4 <= j; k += 4) {
    a0 = fma(-r[k], V[k], a0);
    a1 = fma(-r[k + 1], V[k + 1], a1);
    a2 = fma(-r[k + 2], V[k + 2], a2);
    a3 = fma(-r[k + 3], V[k + 3], a3);
  }
  for (; k < j; ++k) a0 = fma(-r[k], V[k], a0);
  return (a0 + a1) + (a2 + a3);
}

// Offset of scratch row i (i >= r) in the CTA's scratch block: rows r .. i-1 before it.
__device__ __forceinline__ size_t spill_off(int i, int r) {
  return (size_t)i * (i + 1) / 2 - (size_t)r * (r + 1) / 2;
}

// M: the shared rows (row i < r at M + off[i]; the y row at M + off[n], followed by v, d, s);
// G: this CTA's scratch block (rows r .. n-1).  Shared and scratch rows are read by separate
// loops so that the shared ones stay shared-memory loads.
template <typename T, int WPC>
__device__ T gpreg_loglik_cta(const TargetView<T>& tg, const T (&x)[kBlkE], T* M, const int* off, T* G, int r,
                              T* red) {
  constexpr int NT = 32 * WPC;
  const int n = tg.n_data, tid = threadIdx.x;
  const T s2 = x[0] * x[0], t2 = x[1] * x[1], l2 = x[2] * x[2];
  T* ry = M + off[n];      // the y row
  T* V = ry + n;           // v of the current column
  T* Dp = V + n;           // pivots d
  T* S = Dp + n;           // s_i
  for (int i = 0; i < n; ++i) {
    const T* Dr = tg.X + (size_t)i * n;
    if (i < r) {
      T* ri = M + off[i];
      for (int j = tid; j <= i; j += NT) ri[j] = t2 * blk_exp<T>(-l2 * Dr[j]) + (i == j ? s2 : T(0));
    } else {
      T* ri = G + spill_off(i, r);
      for (int j = tid; j <= i; j += NT) ri[j] = t2 * blk_exp<T>(-l2 * Dr[j]) + (i == j ? s2 : T(0));
    }
  }
  for (int j = tid; j < n; j += NT) {
    ry[j] = tg.vec[j];
    S[j] = T(0);
  }
  if (r < n) __threadfence_block();  // scratch rows written by one thread are read by others
  cta_sync<WPC>();
  T quad = T(0);
  bool pd = true;
  for (int j = 0; j < n; ++j) {
    T dj;
    if (j < r) {  // the same values in every thread
      const T* rj = M + off[j];
      dj = rj[j] - S[j];
      for (int k = tid; k < j; k += NT) V[k] = rj[k] * Dp[k];
    } else {
      const T* rj = G + spill_off(j, r);
      dj = rj[j] - S[j];
      for (int k = tid; k < j; k += NT) V[k] = rj[k] * Dp[k];
    }
    if (!(dj > T(0))) { pd = false; break; }
    const T inv = T(1) / dj;
    if (tid == 0) Dp[j] = dj;
    cta_sync<WPC>();  // V complete
    for (int i = j + 1 + tid; i <= n; i += NT) {
      if (i < r || i == n) {
        T* ri = i < n ? M + off[i] : ry;
        const T cij = row_residual<T>(ri, V, j);
        const T lij = cij * inv;
        ri[j] = lij;
        if (i < n) S[i] = fma(lij, cij, S[i]);  // += L_ij^2 d_j
        else quad = fma(cij, lij, quad);
      } else {
        T* ri = G + spill_off(i, r);
        const T cij = row_residual<T>(ri, V, j);
        const T lij = cij * inv;
        ri[j] = lij;
        S[i] = fma(lij, cij, S[i]);
      }
    }
    if (r < n) __threadfence_block();
    cta_sync<WPC>();  // every thread has read V and the rows before V is rewritten
  }
  if (!pd) {
    cta_sync<WPC>();
    return neg_inf<T>();
  }
  T logdet = T(0);
  for (int j = tid; j < n; j += NT) logdet += blk_log<T>(Dp[j]);
  logdet = group_sum<32>(logdet);
  quad = group_sum<32>(quad);
  if constexpr (WPC > 1) {
    const int w = tid >> 5;
    if ((tid & 31) == 0) { red[w] = logdet; red[WPC + w] = quad; }
    __syncthreads();
    logdet = T(0);
    quad = T(0);
    for (int q = 0; q < WPC; ++q) { logdet += red[q]; quad += red[WPC + q]; }
  }
  cta_sync<WPC>();  // the matrix and red are free for the next evaluation
  return T(-0.5) * quad - T(0.5) * logdet - T(0.5) * T(n) * T(1.8378770664093454836);  // log(2 pi)
}

// Per-chain ESS state, the same in every thread of the CTA.
template <typename T>
struct BlkChain {
  T x[kBlkE], nu[kBlkE];
  T ell, logy, th, thmin, thmax;
  int t, k, s;
};

template <typename T>
__device__ __forceinline__ void blk_load(const EssBlockView<T>& v, int64_t c, BlkChain<T>& s) {
  const int d = v.tg.d;
#pragma unroll
  for (int e = 0; e < kBlkE; ++e) {
    s.x[e] = e < d ? v.x[(size_t)c * d + e] : T(0);
    s.nu[e] = e < d ? v.nu[(size_t)c * d + e] : T(0);
  }
  s.ell = v.ell[c]; s.logy = v.logy[c]; s.th = v.th[c]; s.thmin = v.thmin[c]; s.thmax = v.thmax[c];
  s.t = v.t[c]; s.k = v.k[c]; s.s = v.s[c];
}

template <typename T>
__device__ __forceinline__ void blk_store(const EssBlockView<T>& v, int64_t c, const BlkChain<T>& s) {
  if (threadIdx.x != 0) return;
  const int d = v.tg.d;
#pragma unroll
  for (int e = 0; e < kBlkE; ++e)
    if (e < d) {
      v.x[(size_t)c * d + e] = s.x[e];
      v.nu[(size_t)c * d + e] = s.nu[e];
    }
  v.ell[c] = s.ell; v.logy[c] = s.logy; v.th[c] = s.th; v.thmin[c] = s.thmin; v.thmax[c] = s.thmax;
  v.t[c] = s.t; v.k[c] = s.k; v.s[c] = s.s;
}

// One FSM step of chain c: INIT (new ellipse, threshold, first angle) or SHRINK (narrow the
// bracket, next angle), the likelihood at the proposal, and DONE when it clears the threshold.
// Returns true while the chain stays in SHRINK.
// The CTA's covariance storage (see gpreg_loglik_cta).
template <typename T>
struct BlkMat {
  T* M;
  const int* off;
  T* G;
  int r;
};

template <typename T, int WPC>
__device__ bool blk_step(const EssBlockView<T>& v, int64_t c, BlkChain<T>& s, const BlkMat<T>& mt, T* red, int& err) {
  const int d = v.tg.d;
  const bool lead = threadIdx.x == 0;
  const Key key{(uint32_t)(v.chain0 + c), v.seed_lo, v.seed_hi};
  if (s.k == ESS_INIT) {
    // nu = L z, z from draw 0 (D = 1 block of four normals for d <= 4)
    T z[4];
    Conv<T>::normal_quad(key.block((uint32_t)s.t, 0, 0), z);
#pragma unroll
    for (int r = 0; r < kBlkE; ++r) {
      T acc = T(0);
#pragma unroll
      for (int q = 0; q <= r; ++q)
        if (r < d) acc = fma(v.tg.L[r * d + q], z[q], acc);
      s.nu[r] = r < d ? acc : T(0);
    }
    const P4 b = key.block((uint32_t)s.t, 0, 1);
    s.logy = ess_threshold<T>(s.ell, Conv<T>::log_u(b.w0, b.w1));
    s.th = T(kTwoPi) * Conv<T>::u(b.w2, b.w3);
    s.thmin = s.th - T(kTwoPi);
    s.thmax = s.th;
    s.s = 0;
  } else {
    if (s.th < T(0)) s.thmin = s.th; else s.thmax = s.th;
    const P4 b = key.block((uint32_t)s.t, 0, (uint32_t)(2 + s.s));
    s.th = s.thmin + (s.thmax - s.thmin) * Conv<T>::u(b.w0, b.w1);
    ++s.s;
  }
  T sn, cs, xp[kBlkE];
  ess_sincos<T>(s.th, sn, cs);
#pragma unroll
  for (int e = 0; e < kBlkE; ++e) xp[e] = fma(s.x[e], cs, s.nu[e] * sn);
  T ellp = gpreg_loglik_cta<T, WPC>(v.tg, xp, mt.M, mt.off, mt.G, mt.r, red);
  if (!(ellp == ellp)) { ellp = neg_inf<T>(); err |= ERR_NONFINITE; }
  const bool accept = ellp > s.logy;
  if (accept || s.s >= kMaxShrinks) {
    if (accept) {
#pragma unroll
      for (int e = 0; e < kBlkE; ++e) s.x[e] = xp[e];
      s.ell = ellp;
    } else {
      err |= ERR_SHRINK_CAP;
    }
    if (lead) {
      if (v.out) {
#pragma unroll
        for (int e = 0; e < kBlkE; ++e)
          if (e < d) v.out[((size_t)c * v.n + s.t) * d + e] = s.x[e];
      } else {
#pragma unroll
        for (int e = 0; e < kBlkE; ++e) {
          if (e >= d) continue;
          const size_t o = (size_t)c * d + e, st = v.mom_stride;
          T* mo = v.mom;
          T y = s.x[e] - mo[o + st]; T tt = mo[o] + y; mo[o + st] = (tt - mo[o]) - y; mo[o] = tt;
          const T x2 = s.x[e] * s.x[e];
          y = x2 - mo[o + 3 * st]; tt = mo[o + 2 * st] + y; mo[o + 3 * st] = (tt - mo[o + 2 * st]) - y;
          mo[o + 2 * st] = tt;
        }
      }
      v.counts[(size_t)c * v.n + s.t] = s.s;
    }
    ++s.t;
    if (s.t == v.n && lead) atomicAdd(v.chains_done, 1);
    s.k = ESS_INIT;
    return false;
  }
  s.k = ESS_SHRINK;
  return true;
}

// This CTA's matrix: the first r rows, then the y row, v, d and s in shared memory, then the
// row offsets (n + 1 ints); rows r .. n-1 in the CTA's scratch block.
template <typename T, int WPC>
__device__ __forceinline__ BlkMat<T> blk_layout(const EssBlockView<T>& v, unsigned char* raw) {
  const int n = v.tg.n_data;
  const int r = v.rows_smem;
  int* off = (int*)(raw + (gpreg_rows_elems(r) + 4 * (size_t)n) * sizeof(T));
  if (threadIdx.x == 0) {
    int o = 0;
    for (int i = 0; i < r; ++i) { off[i] = o; o += i + 1 + row_gap(i); }
    for (int i = r; i < n; ++i) off[i] = 0;  // scratch rows: spill_off
    off[n] = o;
  }
  cta_sync<WPC>();
  return BlkMat<T>{(T*)raw, off, v.spill ? v.spill + (size_t)blockIdx.x * v.spill_stride : nullptr, r};
}

template <typename T, int WPC>
__global__ void __launch_bounds__(32 * WPC) ess_block_fsm_kernel(EssBlockView<T> v, int budget) {
  extern __shared__ __align__(16) unsigned char blk_smem[];
  __shared__ T red[2 * WPC];
  __shared__ unsigned cur;
  const BlkMat<T> mt = blk_layout<T, WPC>(v, blk_smem);
  int err = 0;
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(v.work, 1u);
    cta_sync<WPC>();
    const int64_t c = cur;
    cta_sync<WPC>();
    if (c >= v.m) break;
    BlkChain<T> s;
    blk_load<T>(v, c, s);
    int steps = 0;
    for (int b = 0; b < budget && s.t < v.n; ++b) {
      blk_step<T, WPC>(v, c, s, mt, red, err);
      ++steps;
    }
    blk_store<T>(v, c, s);
    if (threadIdx.x == 0) v.steps[c] += steps;
  }
  if (err && threadIdx.x == 0) atomicOr(v.err, err);
}

// Synchronised kernel (Alg. 6): for every sample, INIT for all chains, then SHRINK iterations
// over the chains still shrinking, a grid barrier after each.  CTAs take chains in a fixed
// grid-stride order; a CTA with no chain left in the loop waits at the barrier.
template <typename T, int WPC>
__global__ void __launch_bounds__(32 * WPC) ess_block_sync_kernel(EssBlockView<T> v, int t_begin, int t_end,
                                                                  GridBarrier bar, unsigned* active_cnt,
                                                                  unsigned long long* iterations) {
  extern __shared__ __align__(16) unsigned char blk_smem[];
  __shared__ T red[2 * WPC];
  const BlkMat<T> mt = blk_layout<T, WPC>(v, blk_smem);
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  int iter = 0, err = 0;
  for (int t = t_begin; t < t_end; ++t) {
    for (bool first = true;; first = false) {
      unsigned mine = 0;
      for (int64_t c = blockIdx.x; c < v.m; c += gridDim.x) {
        if (!first && v.k[c] != ESS_SHRINK) continue;  // masked: this chain has its sample
        cta_sync<WPC>();  // every thread has read k[c] before thread 0 may store it
        BlkChain<T> s;
        blk_load<T>(v, c, s);
        const bool more = blk_step<T, WPC>(v, c, s, mt, red, err);
        blk_store<T>(v, c, s);
        if (threadIdx.x == 0) v.steps[c] += 1;
        mine += more ? 1u : 0u;
      }
      const int slot = iter % 3;
      if (threadIdx.x == 0 && mine) atomicAdd(&active_cnt[slot], mine);
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
  if (err && threadIdx.x == 0) atomicOr(v.err, err);
}

// log f(x0) of every chain, one CTA per chain.
template <typename T, int WPC>
__global__ void __launch_bounds__(32 * WPC) ess_block_init_kernel(EssBlockView<T> v) {
  extern __shared__ __align__(16) unsigned char blk_smem[];
  __shared__ T red[2 * WPC];
  const BlkMat<T> mt = blk_layout<T, WPC>(v, blk_smem);
  const int d = v.tg.d;
  for (int64_t c = blockIdx.x; c < v.m; c += gridDim.x) {
    T x[kBlkE];
#pragma unroll
    for (int e = 0; e < kBlkE; ++e) x[e] = e < d ? v.x[(size_t)c * d + e] : T(0);
    T ell = gpreg_loglik_cta<T, WPC>(v.tg, x, mt.M, mt.off, mt.G, mt.r, red);
    if (threadIdx.x == 0) {
      if (!(ell == ell)) { ell = neg_inf<T>(); atomicOr(v.err, ERR_NONFINITE); }
      v.ell[c] = ell;
      v.k[c] = ESS_INIT;
    }
  }
}

// ------------------------------------------------------------------------------------------
template <typename K>
static cudaError_t blk_prepare(K kern, int threads, size_t smem, int* per_sm, int* sms) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  int dev = 0;
  cudaGetDevice(&dev);
  e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  return *per_sm > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

// Warps per chain: enough that the chains fill ~16 warps per SM, at most 4.
static int blk_wpc(int64_t m, int sms) {
  const int64_t want = (int64_t)sms * 16;
  return m >= want ? 1 : m * 2 >= want ? 2 : 4;
}
int ess_block_auto_wpc(int64_t m, int sms) { return blk_wpc(m, sms); }

template <typename T, int WPC>
static cudaError_t fsm_launch(const EssBlockView<T>& v, int budget, cudaStream_t st) {
  auto kern = ess_block_fsm_kernel<T, WPC>;
  const size_t smem = gpreg_smem_bytes_r<T>(v.tg.n_data, v.rows_smem);
  int per_sm = 0, sms = 0;
  cudaError_t e = blk_prepare(kern, 32 * WPC, smem, &per_sm, &sms);
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::min<int64_t>(std::min<int64_t>((int64_t)per_sm * sms, v.m), v.max_ctas);
  e = cudaMemsetAsync(v.work, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)blocks, 32 * WPC, smem, st>>>(v, budget);
  return cudaGetLastError();
}

template <typename T, int WPC>
static cudaError_t sync_launch(const EssBlockView<T>& v, int t0, int t1, GridBarrier bar, unsigned* active_cnt,
                               unsigned long long* iters, cudaStream_t st) {
  auto kern = ess_block_sync_kernel<T, WPC>;
  const size_t smem = gpreg_smem_bytes_r<T>(v.tg.n_data, v.rows_smem);
  int per_sm = 0, sms = 0;
  cudaError_t e = blk_prepare(kern, 32 * WPC, smem, &per_sm, &sms);
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::min<int64_t>(std::min<int64_t>((int64_t)per_sm * sms, v.m), v.max_ctas);
  EssBlockView<T> vv = v;
  void* args[] = {(void*)&vv, (void*)&t0, (void*)&t1, (void*)&bar, (void*)&active_cnt, (void*)&iters};
  return cudaLaunchCooperativeKernel((void*)kern, dim3((unsigned)blocks), dim3(32 * WPC), args, smem, st);
}

template <typename T, int WPC>
static cudaError_t init_launch(const EssBlockView<T>& v, cudaStream_t st) {
  auto kern = ess_block_init_kernel<T, WPC>;
  const size_t smem = gpreg_smem_bytes_r<T>(v.tg.n_data, v.rows_smem);
  int per_sm = 0, sms = 0;
  cudaError_t e = blk_prepare(kern, 32 * WPC, smem, &per_sm, &sms);
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::min<int64_t>(std::min<int64_t>((int64_t)per_sm * sms, v.m), v.max_ctas);
  kern<<<(unsigned)blocks, 32 * WPC, smem, st>>>(v);
  return cudaGetLastError();
}

#define FSMC_BLK_DISPATCH(FN, ...)                    \
  do {                                                \
    int dev = 0, sms = 0;                             \
    cudaGetDevice(&dev);                              \
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev); \
    switch (v.wpc ? v.wpc : blk_wpc(v.m, sms)) {      \
      case 1: return FN<T, 1>(__VA_ARGS__);           \
      case 2: return FN<T, 2>(__VA_ARGS__);           \
      default: return FN<T, 4>(__VA_ARGS__);          \
    }                                                 \
  } while (0)

template <typename T>
cudaError_t launch_ess_block_fsm(const EssBlockView<T>& v, int budget, cudaStream_t st) {
  FSMC_BLK_DISPATCH(fsm_launch, v, budget, st);
}

template <typename T>
cudaError_t launch_ess_block_sync(const EssBlockView<T>& v, int t0, int t1, GridBarrier bar, unsigned* active_cnt,
                                  unsigned long long* iters, cudaStream_t st) {
  FSMC_BLK_DISPATCH(sync_launch, v, t0, t1, bar, active_cnt, iters, st);
}

template <typename T>
cudaError_t launch_ess_block_init(const EssBlockView<T>& v, cudaStream_t st) {
  FSMC_BLK_DISPATCH(init_launch, v, st);
}

// Rows of an n-point covariance kept in shared memory, and the scratch elements per CTA for the
// rest (0 when all fit).
template <typename T>
int gpreg_smem_rows(int n) { return gpreg_rows_in_smem<T>(n); }
template <typename T>
size_t gpreg_spill_elems(int n) {
  const int r = gpreg_rows_in_smem<T>(n);
  size_t e = 0;
  for (int i = r; i < n; ++i) e += (size_t)(i + 1);
  return e;
}
template int gpreg_smem_rows<float>(int);
template int gpreg_smem_rows<double>(int);
template size_t gpreg_spill_elems<float>(int);
template size_t gpreg_spill_elems<double>(int);

template cudaError_t launch_ess_block_fsm<float>(const EssBlockView<float>&, int, cudaStream_t);
template cudaError_t launch_ess_block_fsm<double>(const EssBlockView<double>&, int, cudaStream_t);
template cudaError_t launch_ess_block_sync<float>(const EssBlockView<float>&, int, int, GridBarrier, unsigned*,
                                                  unsigned long long*, cudaStream_t);
template cudaError_t launch_ess_block_sync<double>(const EssBlockView<double>&, int, int, GridBarrier, unsigned*,
                                                   unsigned long long*, cudaStream_t);
template cudaError_t launch_ess_block_init<float>(const EssBlockView<float>&, cudaStream_t);
template cudaError_t launch_ess_block_init<double>(const EssBlockView<double>&, cudaStream_t);

}  // namespace fsmc
