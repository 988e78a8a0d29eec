// Ellipse directions nu = L z on the 5th-generation tensor cores (tcgen05), d <= 256, FP32 jobs.
//
// The contraction behind ESS's INIT state is dense: for every (chain, sample) column the
// lower-triangular prior factor L (d x d) multiplies a fresh standard-normal z.  Here:
//  * L is split once into two FP16 parts, L = L_hi + L_lo (11 + 11 significant bits), laid out
//    in the tensor cores' K-major shared-memory layout and copied into shared memory once per
//    CTA with a bulk TMA copy; it stays resident while the CTA walks over column tiles;
//  * for each tile of 64 columns, all 256 threads draw z from Philox (Box-Muller, the same
//    conversion as the SIMT path) straight into shared memory, split into z_hi + z_lo;
//  * one elected thread issues tcgen05.mma (kind::f16, FP32 accumulation in tensor memory):
//    L_hi z_hi + L_hi z_lo + L_lo z_hi per 16-wide k-step (the dropped L_lo z_lo term is
//    ~2^-22 relative), for row tile 0 (rows 0..127, k < 128) and row tile 1 (rows 128..255);
//  * the accumulators are read back with tcgen05.ld and stored to the chains' direction rings.
// The columns of one refill are compacted first (a prefix sum over the chains' refill counts and
// a (chain, sample) list), so every tile holds 64 columns that are actually needed: chains
// consume different numbers of directions per round, and tiles over fixed chain blocks and ring
// offsets were on average about half empty.
// Every wait on an mbarrier is bounded; on expiry the kernel records ERR_BARRIER_TIMEOUT,
// waits (bounded) for its outstanding MMAs, frees its tensor memory and returns.
#include <cuda_fp16.h>
#include <algorithm>

#include "ess_common.cuh"
#include "fsmc_device.cuh"
#include "fsmc_kernels.h"

namespace fsmc {

namespace {

constexpr int TC_PRODUCER_WARPS = 16;
constexpr int TC_THREADS = (TC_PRODUCER_WARPS + 2) * 32;  // + the MMA warp and the column-list warp
constexpr int TC_N = 64;          // columns per tile
constexpr int TC_TMEM_COLS = 256; // two accumulator buffers of (row tile 0, row tile 1) x 64 columns
constexpr int TC_KC = 64;         // k per staged chunk
constexpr int TC_STAGE = TC_N * TC_KC * 2;  // bytes of one FP16 part of a z chunk (8 KB)
constexpr unsigned kWaitLimit = 1u << 20;  // polls of at most ~1 us each

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// bounded wait for the phase with the given parity to complete; gives up early once another
// warp has recorded a failure in *fail (when fail is not null)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, volatile int* fail) {
  const uint32_t a = smem_u32(bar);
  for (unsigned it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    // the thread is suspended until the phase completes or about 1 us has passed
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(1000u)
        : "memory");
    if (done) return true;
    if (fail && (it & 15) == 15 && *fail) return false;
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// warp-uniform forms: every lane polls, and the warp proceeds only if every lane saw the phase
// complete; the failure flag is read once (lane 0) for the whole warp
__device__ __forceinline__ bool warp_wait(uint64_t* bar, unsigned parity, volatile int* fail) {
  return __all_sync(0xffffffffu, mbar_wait(bar, parity, fail));
}
__device__ __forceinline__ bool warp_failed(volatile int* fail) {
  return __shfl_sync(0xffffffffu, *fail, 0) != 0;
}

// tensor-core shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, swizzle mode 0 (none)
}

// instruction descriptor, kind::f16: A, B = F16, D = F32, both K-major
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

struct TcLayout {
  int K0, K1;          // k extent of row tile 0 / 1 (K1 = 0: no row tile 1)
  int kpad;            // k extent of z (multiple of TC_KC)
  int a_bytes;         // whole A image
};

__host__ __device__ inline TcLayout tc_layout(int d) {
  TcLayout L;
  L.kpad = (d + TC_KC - 1) / TC_KC * TC_KC;
  L.K0 = L.kpad < 128 ? L.kpad : 128;
  L.K1 = d > 128 ? L.kpad : 0;
  L.a_bytes = 128 * L.K0 * 2 * 2 + 128 * L.K1 * 2 * 2;
  return L;
}

// byte offset of element (m, k) in a K-major no-swizzle image with k extent K
__host__ __device__ inline int kmajor_off(int m, int k, int K) {
  return (m >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (m & 7) * 16 + (k & 7) * 2;
}

}  // namespace

// Builds the FP16 hi/lo image of L in the tensor cores' layout:
// [row tile 0 hi][row tile 0 lo][row tile 1 hi][row tile 1 lo].
__global__ void ess_tc_build_a_kernel(const float* L, int d, unsigned char* img) {
  const TcLayout lay = tc_layout(d);
  const int total = 128 * lay.K0 + 128 * lay.K1;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int rt, m, k, K;
    if (idx < 128 * lay.K0) { rt = 0; K = lay.K0; m = idx / K; k = idx % K; }
    else { rt = 1; K = lay.K1; m = (idx - 128 * lay.K0) / K; k = (idx - 128 * lay.K0) % K; }
    const int row = rt * 128 + m;
    const float v = (row < d && k < d && k <= row) ? L[(size_t)row * d + k] : 0.f;
    const __half hi = __float2half_rn(v);
    const __half lo = __float2half_rn(v - __half2float(hi));
    const int base = rt == 0 ? 0 : 128 * lay.K0 * 4;
    const int part = 128 * K * 2;
    *reinterpret_cast<__half*>(img + base + kmajor_off(m, k, K)) = hi;
    *reinterpret_cast<__half*>(img + base + part + kmajor_off(m, k, K)) = lo;
  }
}

// Shared-memory layout after the A image and the two z stages.
struct TcBars {
  uint64_t a;              // L image loaded (TMA transaction count)
  uint64_t full[2];        // z stage written (one arrival per producer warp)
  uint64_t empty[2];       // z stage consumed (tcgen05.commit)
  uint64_t acc_full[2];    // accumulator buffer complete (tcgen05.commit)
  uint64_t acc_empty[2];   // accumulator buffer read out (one arrival per producer warp)
  uint64_t cols_full[2];   // column list of a tile written (MMA warp)
  uint64_t cols_empty[2];  // column list no longer read (one arrival per producer warp)
  uint64_t drain;          // teardown: every issued MMA has completed
  uint32_t tmem;
  int fail;
};
struct TcCols {
  float* dst[2][TC_N];     // ring row of each column, null: no column
  int sample[2][TC_N];
  int chain[2][TC_N];
};

__host__ __device__ inline int tc_smem_bytes(int d) {
  return tc_layout(d).a_bytes + 2 * 2 * TC_STAGE + (int)sizeof(TcBars) + (int)sizeof(TcCols);
}

// Warp-specialised pipeline over tiles of 64 refill columns:
//  * warps 0..15 (producers, two groups of eight, one per shared-memory stage) write z chunks,
//    and read out the accumulators of the previous tile (after their first chunk of the next
//    one, so the last MMAs of a tile overlap with the next tile's first chunks);
//  * warp 16 issues the tcgen05 MMAs (one elected lane) into one of two tensor-memory
//    accumulator buffers;
//  * warp 17 loads the column lists of coming tiles into a double-buffered table.
// Every handoff is an mbarrier; every wait is bounded and also ends when another warp has
// recorded a failure.
__global__ void __launch_bounds__(TC_THREADS, 1) ess_nu_gen_tc_kernel(EssView<float> v, const unsigned char* a_img) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int d = v.tg.d;
  const TcLayout lay = tc_layout(d);
  unsigned char* sA = sm;
  unsigned char* sB = sm + lay.a_bytes;  // 2 stages x (hi, lo)
  TcBars* bars = reinterpret_cast<TcBars*>(sB + 2 * 2 * TC_STAGE);
  TcCols* cols = reinterpret_cast<TcCols*>(bars + 1);
  volatile int* fail = &bars->fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool mma_warp = warp == TC_PRODUCER_WARPS;
  const bool cols_warp = warp == TC_PRODUCER_WARPS + 1;
  const int D = (d + 3) / 4;  // Philox blocks of z (four normals each)
  const bool fold = ess_ring_folded(v);
  const int nchunks = lay.kpad / TC_KC;
  const long long total = v.col_base[v.m];
  const long long ntiles = (total + TC_N - 1) / TC_N;
  if (blockIdx.x == 0 && tid == 0 && total > 0) atomicAdd(v.gen_cols, (unsigned long long)total);

  if (tid == 0) {
    bars->fail = 0;
    mbar_init(&bars->a, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bars->full[i], TC_PRODUCER_WARPS / 2);  // the stage's producer group
      mbar_init(&bars->empty[i], 1);
      mbar_init(&bars->acc_full[i], 1);
      mbar_init(&bars->acc_empty[i], TC_PRODUCER_WARPS);
      mbar_init(&bars->cols_full[i], 1);
      mbar_init(&bars->cols_empty[i], TC_PRODUCER_WARPS);
    }
    mbar_init(&bars->drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (mma_warp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&bars->tmem)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = bars->tmem;

  const long long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (cols_warp) {
    // ---------------------------------------------------------------- column-list warp
    // column list of local tile i (tile blockIdx.x + i * gridDim.x) into buffer i & 1, once the
    // producers have read out tile i-2 (the buffer's previous user)
    for (long long i = 0; i < my_tiles && !warp_failed(fail); ++i) {
      const int bb = (int)(i & 1);
      if (i >= 2 && !warp_wait(&bars->cols_empty[bb], (unsigned)(((i >> 1) - 1) & 1), fail)) {
        *fail = 1;
        break;
      }
      const long long tile = blockIdx.x + i * gridDim.x;
#pragma unroll
      for (int r = 0; r < TC_N / 32; ++r) {
        const int n = lane + 32 * r;
        const long long jc = tile * TC_N + n;
        int c = -1, smp = -1;
        if (jc < total) {
          const int2 e = v.colmap[jc];
          c = e.x;
          smp = e.y;
        }
        cols->chain[bb][n] = c;
        cols->sample[bb][n] = smp;
        cols->dst[bb][n] = smp >= 0 ? v.nu + ((size_t)c * v.W + smp % v.W) * v.dstride : nullptr;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->cols_full[bb]);
    }
  } else if (mma_warp) {
    // ---------------------------------------------------------------- MMA warp
    if (lane == 0) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bars->a)),
                   "r"(lay.a_bytes)
                   : "memory");
      for (int off = 0; off < lay.a_bytes; off += 48 * 1024) {
        const int n = min(48 * 1024, lay.a_bytes - off);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(sA + off)),
            "l"(a_img + off), "r"(n), "r"(smem_u32(&bars->a))
            : "memory");
      }
    }
    if (!warp_wait(&bars->a, 0, fail)) *fail = 1;
    const uint32_t idesc = idesc_f16(128, TC_N);
    const uint32_t sA_u = smem_u32(sA), sB_u = smem_u32(sB);
    const uint32_t a_rt0 = sA_u, a_rt1 = sA_u + 128 * lay.K0 * 4;
    long long chunk_ctr = 0;
    bool issued = false;
    for (long long i = 0; i < my_tiles && !warp_failed(fail); ++i) {
      const int bb = (int)(i & 1);
      const uint32_t acc = tmem + (uint32_t)(bb * 2 * TC_N);
      if (i >= 2 && !warp_wait(&bars->acc_empty[bb], (unsigned)(((i >> 1) - 1) & 1), fail)) {
        *fail = 1;
        break;
      }
      for (int kc = 0; kc < nchunks && !warp_failed(fail); ++kc, ++chunk_ctr) {
        const int s = (int)(chunk_ctr & 1);
        if (!warp_wait(&bars->full[s], (unsigned)((chunk_ctr >> 1) & 1), fail)) {
          *fail = 1;
          break;
        }
        if (lane == 0) {
          {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t bh = sB_u + s * 2 * TC_STAGE, bl = bh + TC_STAGE;
#pragma unroll
            for (int ks = 0; ks < TC_KC / 16; ++ks) {
              const int kglob = kc * TC_KC + ks * 16;
              const uint64_t dbh = sdesc(bh + ks * 256, 128, (TC_KC / 8) * 128);
              const uint64_t dbl = sdesc(bl + ks * 256, 128, (TC_KC / 8) * 128);
              if (kglob < lay.K0) {
                const uint32_t ah = a_rt0 + (kglob / 8) * 128, al = ah + 128 * lay.K0 * 2;
                const uint32_t sbo = (lay.K0 / 8) * 128;
                mma_f16(acc, sdesc(ah, 128, sbo), dbh, idesc, kglob > 0);
                mma_f16(acc, sdesc(ah, 128, sbo), dbl, idesc, 1);
                mma_f16(acc, sdesc(al, 128, sbo), dbh, idesc, 1);
              }
              if (lay.K1) {
                const uint32_t ah = a_rt1 + (kglob / 8) * 128, al = ah + 128 * lay.K1 * 2;
                const uint32_t sbo = (lay.K1 / 8) * 128;
                mma_f16(acc + TC_N, sdesc(ah, 128, sbo), dbh, idesc, kglob > 0);
                mma_f16(acc + TC_N, sdesc(ah, 128, sbo), dbl, idesc, 1);
                mma_f16(acc + TC_N, sdesc(al, 128, sbo), dbh, idesc, 1);
              }
            }
            issued = true;
            mma_commit(&bars->empty[s]);
            if (kc == nchunks - 1) mma_commit(&bars->acc_full[bb]);
          }
        }
        __syncwarp();
      }
    }
    // teardown: every issued MMA must have completed before tensor memory is freed
    if (lane == 0 && issued) {
      mma_commit(&bars->drain);
      mbar_wait(&bars->drain, 0, nullptr);
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- producer warps
    // Two groups of eight warps; group g fills the chunks that land in stage g, so each group
    // has a whole chunk time of slack and every thread draws four independent Philox blocks
    // per chunk.  z roles: this lane's column and k half are the same for every chunk; a warp
    // fills two core matrices (8 columns x 8 k, 128 contiguous bytes each) per pass.
    constexpr int kGroupWarps = TC_PRODUCER_WARPS / 2;
    const int grp = warp / kGroupWarps, gw = warp % kGroupWarps;
    const int zn = (((2 * gw + (lane >> 4)) & 7) << 3) + ((lane >> 1) & 7);  // column 0..63
    const int zkh = lane & 1;
    constexpr int kPasses = 64 / (2 * kGroupWarps);  // core-matrix pairs per warp per chunk
    // accumulators of local tile i -> the chains' direction rings
    // (warp w: row tile (w >> 2) & 1, tensor-memory lane quadrant w & 3, column half w >> 3)
    // this thread's epilogue row (the same for every tile) and the sign folded into it
    // (ess_ring_folded), read once
    const int ep_row = ((warp >> 2) & 1) * 128 + (warp & 3) * 32 + lane;
    const uint32_t sgn = fold && ep_row < d && v.tg.vec[ep_row] > 0.f ? 0x80000000u : 0u;
    auto epilogue = [&](long long i) {
      const int bb = (int)(i & 1);
      if (!warp_wait(&bars->acc_full[bb], (unsigned)((i >> 1) & 1), fail)) { *fail = 1; return; }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int rt = (warp >> 2) & 1;
      if (rt == 0 || lay.K1) {
        const int row = ep_row;
        const int jbeg = (warp >> 3) * (TC_N / 2);
        // both 16-column loads in flight before the single wait
        uint32_t r[TC_N / 2];
        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) +
                               (uint32_t)(bb * 2 * TC_N + rt * TC_N + jbeg);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t* q = r + 16 * h;
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
              "[%16];"
              : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
                "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]),
                "=r"(q[15])
              : "r"(taddr + 16 * h));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < d) {
#pragma unroll
          for (int jj = 0; jj < TC_N / 2; ++jj) {
            float* dst = cols->dst[bb][jbeg + jj];
            if (dst) dst[row] = __uint_as_float(r[jj] ^ sgn);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&bars->acc_empty[bb]);
        mbar_arrive(&bars->cols_empty[bb]);
      }
    };
    long long chunk_ctr = 0;
    long long i = 0;
    for (; i < my_tiles && !warp_failed(fail); ++i) {
      const int bb = (int)(i & 1);
      if (!warp_wait(&bars->cols_full[bb], (unsigned)((i >> 1) & 1), fail)) { *fail = 1; break; }
      const int z_smp = cols->sample[bb][zn];
      const Key zkey{(uint32_t)(v.chain0 + cols->chain[bb][zn]), v.seed_lo, v.seed_hi};
      bool broke = false, drained = i == 0;  // drained: tile i-1 has been read out
      for (int kc = 0; kc < nchunks; ++kc, ++chunk_ctr) {
        const int s = (int)(chunk_ctr & 1);
        if (s != grp) continue;  // the other group's stage
        if (warp_failed(fail) ||
            (chunk_ctr >= 2 && !warp_wait(&bars->empty[s], (unsigned)(((chunk_ctr >> 1) - 1) & 1), fail))) {
          *fail = 1;
          broke = true;
          break;
        }
        unsigned char* zhi = sB + s * 2 * TC_STAGE;
        unsigned char* zlo = zhi + TC_STAGE;
        const bool whole = (kc + 1) * TC_KC <= d;  // no coordinate of the chunk lies beyond d
        // all Philox blocks of the chunk first (independent, so their rounds interleave), then
        // Box-Muller, the FP16 hi/lo split and the stores
        P4 blk[kPasses];
#pragma unroll
        for (int it = 0; it < kPasses; ++it) {
          const int kg = (2 * (gw + kGroupWarps * it) + (lane >> 4)) >> 3;
          const int q = kc * (TC_KC / 4) + kg * 2 + zkh;  // Philox draw: normals 4q .. 4q+3
          blk[it] = (z_smp >= 0 && q < D) ? zkey.block((uint32_t)z_smp, 0, (uint32_t)q) : P4{0u, 0u, 0u, 0u};
        }
#pragma unroll
        for (int it = 0; it < kPasses; ++it) {
          const int kg = (2 * (gw + kGroupWarps * it) + (lane >> 4)) >> 3;
          const int q = kc * (TC_KC / 4) + kg * 2 + zkh;
          float z[4] = {0.f, 0.f, 0.f, 0.f};
          if (z_smp >= 0 && q < D) {
            Conv<float>::normal_quad(blk[it], z);
            if (!whole) {
#pragma unroll
              for (int e = 0; e < 4; ++e)
                if (4 * q + e >= d) z[e] = 0.f;
            }
          }
          const __half2 h01 = __float22half2_rn(make_float2(z[0], z[1]));
          const __half2 h23 = __float22half2_rn(make_float2(z[2], z[3]));
          const float2 b01 = __half22float2(h01), b23 = __half22float2(h23);
          const __half2 l01 = __float22half2_rn(make_float2(z[0] - b01.x, z[1] - b01.y));
          const __half2 l23 = __float22half2_rn(make_float2(z[2] - b23.x, z[3] - b23.y));
          const int off = (zn >> 3) * (TC_KC / 8) * 128 + kg * 128 + (zn & 7) * 16 + zkh * 8;
          *reinterpret_cast<uint2*>(zhi + off) =
              make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
          *reinterpret_cast<uint2*>(zlo + off) =
              make_uint2(*reinterpret_cast<const uint32_t*>(&l01), *reinterpret_cast<const uint32_t*>(&l23));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->full[s]);
        if (!drained) {  // after this group's first chunk of tile i
          epilogue(i - 1);
          drained = true;
        }
      }
      if (broke) break;
      if (!drained) epilogue(i - 1);  // the group had no chunk in this tile
    }
    if (i == my_tiles && my_tiles > 0 && !warp_failed(fail)) epilogue(my_tiles - 1);
  }
  if (*fail && tid == 0) atomicOr(v.err, ERR_BARRIER_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (mma_warp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// Refill counts -> exclusive prefix sum col_base[0..m] (one block, chains in passes of
// 1024 x 8, each thread a run of 8 consecutive chains).
__global__ void __launch_bounds__(1024) ess_col_scan_kernel(const int* gen_lo, const int* gen_hi, int64_t m,
                                                            long long* base) {
  constexpr int SEG = 8;
  __shared__ long long warp_tot[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  long long run = 0;
  for (int64_t p0 = 0; p0 < m; p0 += 1024 * SEG) {
    int cnt[SEG];
    long long local = 0;
#pragma unroll
    for (int s = 0; s < SEG; ++s) {
      const int64_t c = p0 + (int64_t)tid * SEG + s;
      cnt[s] = c < m ? max(0, gen_hi[c] - gen_lo[c]) : 0;
      local += cnt[s];
    }
    long long incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      long long wt = warp_tot[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, wt, o);
        if (lane >= o) wt += y;
      }
      warp_tot[lane] = wt;  // inclusive over warps
    }
    __syncthreads();
    long long excl = run + (warp > 0 ? warp_tot[warp - 1] : 0) + incl - local;
#pragma unroll
    for (int s = 0; s < SEG; ++s) {
      const int64_t c = p0 + (int64_t)tid * SEG + s;
      if (c < m) base[c] = excl;
      excl += cnt[s];
    }
    run += warp_tot[31];
    __syncthreads();
  }
  if (tid == 0) base[m] = run;
}

// (chain, sample) of every refill column, in chain order
__global__ void ess_col_fill_kernel(const int* gen_lo, const int* gen_hi, const long long* base, int64_t m,
                                    int2* colmap) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m) return;
  const int lo = gen_lo[c], cnt = gen_hi[c] - lo;
  const long long b = base[c];
  for (int k = 0; k < cnt; ++k) colmap[b + k] = make_int2((int)c, lo + k);
}

size_t ess_tc_image_bytes(int d) { return (size_t)tc_layout(d).a_bytes; }

cudaError_t launch_ess_tc_build(const float* L, int d, unsigned char* img, cudaStream_t st) {
  const TcLayout lay = tc_layout(d);
  const int total = 128 * lay.K0 + 128 * lay.K1;
  ess_tc_build_a_kernel<<<(total + 255) / 256, 256, 0, st>>>(L, d, img);
  return cudaGetLastError();
}

cudaError_t launch_ess_tc_cols(const EssView<float>& v, cudaStream_t st) {
  if (!v.colmap || !v.col_base) return cudaErrorInvalidValue;  // the generator walks the compacted list
  ess_col_scan_kernel<<<1, 1024, 0, st>>>(v.gen_lo, v.gen_hi, v.m, v.col_base);
  ess_col_fill_kernel<<<(unsigned)((v.m + 255) / 256), 256, 0, st>>>(v.gen_lo, v.gen_hi, v.col_base, v.m,
                                                                     v.colmap);
  return cudaGetLastError();
}

cudaError_t launch_ess_tc_gen(const EssView<float>& v, const unsigned char* img, int sms, cudaStream_t st) {
  if (!v.colmap || !v.col_base) return cudaErrorInvalidValue;
  const int smem = tc_smem_bytes(v.tg.d);
  cudaError_t e = cudaFuncSetAttribute(ess_nu_gen_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const long long ntiles = ((long long)v.m * v.W + TC_N - 1) / TC_N;
  const int grid = (int)std::max(1LL, std::min<long long>(ntiles, sms));
  ess_nu_gen_tc_kernel<<<grid, TC_THREADS, smem, st>>>(v, img);
  return cudaGetLastError();
}

cudaError_t launch_ess_nu_gen_tc(const EssView<float>& v, const unsigned char* img, int sms, cudaStream_t st) {
  cudaError_t e = launch_ess_tc_cols(v, st);
  if (e != cudaSuccess) return e;
  return launch_ess_tc_gen(v, img, sms, st);
}

}  // namespace fsmc
