// Run statistics of Sec. 4 reduced on the device: over the samples i < t_min that every chain
// has completed, the sum of the loop-body counts N_ij and the sum over i of max_j N_ij, from
// which R(m) = mean_i max_j N_ij / mean_ij N_ij (Sec. 4.2); also t_min, the samples and FSM
// states summed over chains, and the synchronised kernel's iteration counter and the error
// word, so that the host reads one 64-byte record instead of the [m][n] count array.
#include <algorithm>
#include <climits>

#include "fsmc_kernels.h"

namespace fsmc {

__global__ void stats_reset_kernel(DevStats* o) {
  o->tmin = LLONG_MAX;
  o->samples_done = 0;
  o->fsm_steps = 0;
  o->sum_all = 0;
  o->sum_max = 0;
  o->iters = 0;
  o->err = 0;
  o->pad = 0;
}

// t_min, sum_j t_j and sum_j steps_j (a warp combines its chains before the atomics)
__global__ void stats_chains_kernel(const int* t, const long long* steps, int64_t m, DevStats* o) {
  long long tmin = LLONG_MAX, tsum = 0, ssum = 0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < m; c += (int64_t)gridDim.x * blockDim.x) {
    const long long tc = t[c];
    tmin = tc < tmin ? tc : tmin;
    tsum += tc;
    ssum += steps[c];
  }
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) {
    const long long a = __shfl_xor_sync(0xffffffffu, tmin, o2);
    tmin = a < tmin ? a : tmin;
    tsum += __shfl_xor_sync(0xffffffffu, tsum, o2);
    ssum += __shfl_xor_sync(0xffffffffu, ssum, o2);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&o->tmin, tmin);
    atomicAdd((unsigned long long*)&o->samples_done, (unsigned long long)tsum);
    atomicAdd((unsigned long long*)&o->fsm_steps, (unsigned long long)ssum);
  }
}

// Column maxima and the total over samples i < t_min.  Block (32, 8): threadIdx.x picks the
// sample i = 32 blockIdx.x + threadIdx.x (a warp reads 32 consecutive counts of one chain), and
// the 8 rows of the block with the blockIdx.y slices stride over the chains.
__global__ void stats_columns_kernel(const int* counts, int64_t m, int n, const DevStats* o,
                                     unsigned* colmax, unsigned long long* sum_all) {
  __shared__ unsigned smax[8][33];
  __shared__ unsigned long long ssum[8][33];
  const long long tmin = o->tmin;
  const int i = blockIdx.x * 32 + threadIdx.x;
  unsigned mx = 0;
  unsigned long long sm = 0;
  if (i < tmin) {
    for (int64_t c = (int64_t)blockIdx.y * 8 + threadIdx.y; c < m; c += (int64_t)gridDim.y * 8) {
      const unsigned v = (unsigned)counts[(size_t)c * n + i];
      mx = v > mx ? v : mx;
      sm += v;
    }
  }
  smax[threadIdx.y][threadIdx.x] = mx;
  ssum[threadIdx.y][threadIdx.x] = sm;
  __syncthreads();
  if (threadIdx.y == 0) {
#pragma unroll
    for (int r = 1; r < 8; ++r) {
      const unsigned a = smax[r][threadIdx.x];
      mx = a > mx ? a : mx;
      sm += ssum[r][threadIdx.x];
    }
    if (i < tmin) atomicMax(&colmax[i], mx);
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o2);
    if (threadIdx.x == 0 && sm) atomicAdd(sum_all, sm);
  }
}

// sum over i < t_min of max_j N_ij, and the scalars the record carries beside the sums
__global__ void stats_final_kernel(const unsigned* colmax, int n, const unsigned long long* iters,
                                   const int* err, DevStats* o) {
  __shared__ unsigned long long part[32];
  const long long tmin = o->tmin;
  const int lim = tmin < n ? (int)tmin : n;
  unsigned long long s = 0;
  for (int i = threadIdx.x; i < lim; i += blockDim.x) s += colmax[i];
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o2);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += part[w];
    o->sum_max = tot;
    o->iters = (long long)*iters;
    o->err = *err;
  }
}

cudaError_t launch_job_stats(const int* counts, const int* t, const long long* steps, int64_t m, int n,
                             const unsigned long long* iters, const int* err, unsigned* colmax,
                             DevStats* out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(colmax, 0, (size_t)n * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  stats_reset_kernel<<<1, 1, 0, st>>>(out);
  const int cb = (int)std::min<int64_t>((m + 255) / 256, 1184);
  stats_chains_kernel<<<cb < 1 ? 1 : cb, 256, 0, st>>>(t, steps, m, out);
  // about 2048 blocks of 256 threads over the (sample tile, chain slice) grid
  const int gx = (n + 31) / 32;
  int64_t gy = std::max<int64_t>(1, 2048 / gx);
  gy = std::min<int64_t>(gy, (m + 7) / 8);
  gy = std::min<int64_t>(gy, 65535);
  stats_columns_kernel<<<dim3(gx, (unsigned)gy), dim3(32, 8), 0, st>>>(counts, m, n, out, colmax,
                                                                       (unsigned long long*)&out->sum_all);
  stats_final_kernel<<<1, 1024, 0, st>>>(colmax, n, iters, err, out);
  return cudaGetLastError();
}

}  // namespace fsmc
