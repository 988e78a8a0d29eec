// Allocation-free elliptical slice sampling run (fsmc_ess_run_static in include/fsmc.h).
//
// Everything the FSM run needs beyond the caller's inputs and outputs -- each chain's
// state and its ring of pre-generated ellipse directions -- lives in one file-scope
// device array of fixed size.  The host code here never allocates device memory: it
// resolves the array's device address once per device with cudaGetSymbolAddress and
// launches the same generator and FSM step kernels as fsmc_job_run.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "engine_internal.h"
#include "fsmc_device.cuh"
#include "fsmc_kernels.h"

using namespace fsmc;

namespace {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;  // 32 MiB per device
constexpr int kMaxDevices = 64;
// Lower bound on a chain's scratch bytes at any d >= 1 and W >= 2: its state (x, t, k, s, the two
// window bounds, ell, logy, three angles, steps: at least 52 bytes) plus two 32-float ring rows.
constexpr size_t kMinChainBytes = 48;

// Shared by every call on a device.  Host code must not take its address directly: in
// host code this name denotes a host-side shadow, not device memory.
__device__ __align__(256) unsigned char g_ess_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_dev[kMaxDevices] = {};

size_t al(size_t v) { return (v + 255) / 256 * 256; }

struct ScratchLayout {
  size_t x, t, k, s, gen, ell, logy, th, steps, misc, nu, total;
};

ScratchLayout layout_for(int64_t m, int d, int W, int dstride) {
  ScratchLayout L{};
  size_t o = 0;
  L.x = o; o = al(o + (size_t)m * d * 4);
  L.t = o; o = al(o + (size_t)m * 4);
  L.k = o; o = al(o + (size_t)m * 4);
  L.s = o; o = al(o + (size_t)m * 4);
  L.gen = o; o = al(o + (size_t)2 * m * 4);
  L.ell = o; o = al(o + (size_t)m * 4);
  L.logy = o; o = al(o + (size_t)m * 4);
  L.th = o; o = al(o + (size_t)3 * m * 4);
  L.steps = o; o = al(o + (size_t)m * 8);
  L.misc = o; o = al(o + 32);  // error word, finished-chain count, generated-column count
  L.nu = o; o = al(o + (size_t)m * W * dstride * 4);
  L.total = o;
  return L;
}

}  // namespace

extern "C" fsmc_status fsmc_ess_run_static(int target_kind, int d, const float* L_dev,
                                           const float* vec_dev, float noise_var, int64_t n_chains,
                                           int64_t n_samples, const float* x0_dev, uint64_t seed,
                                           int lanes_per_chain, float* samples_dev,
                                           int32_t* counts_dev, void* cuda_stream) {
  if (target_kind != FSMC_TGT_GAUSS_CONJ && target_kind != FSMC_TGT_GP_LOGIT && target_kind != FSMC_TGT_FLAT)
    return fsmc_fail(FSMC_EINVAL, "fsmc_ess_run_static: target must be GAUSS_CONJ, GP_LOGIT or FLAT");
  if (d < 1 || d > 1024 || n_chains < 1 || n_samples < 1 || n_samples > (int64_t)1 << 30)
    return fsmc_fail(FSMC_EINVAL, "fsmc_ess_run_static: d in [1, 1024], n_chains >= 1, n_samples >= 1");
  if (lanes_per_chain != 1 && lanes_per_chain != 32)
    return fsmc_fail(FSMC_EINVAL, "fsmc_ess_run_static: lanes_per_chain must be 1 or 32");
  if (lanes_per_chain == 1 && d > 32)
    return fsmc_fail(FSMC_EINVAL, "fsmc_ess_run_static: chain-per-thread needs d <= 32");
  if (!L_dev || !x0_dev || !samples_dev || !counts_dev || (target_kind != FSMC_TGT_FLAT && !vec_dev))
    return fsmc_fail(FSMC_EINVAL, "fsmc_ess_run_static: NULL device pointer");
  if (target_kind == FSMC_TGT_GAUSS_CONJ && !(noise_var > 0))
    return fsmc_fail(FSMC_EINVAL, "fsmc_ess_run_static: noise_var must be > 0");

  // Every chain needs more than kMinChainBytes of scratch whatever W is, so a larger n_chains
  // can never fit; rejecting it here also keeps the layout sums below from overflowing.
  if (n_chains > (int64_t)(kStaticScratchBytes / kMinChainBytes)) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "fsmc_ess_run_static: %lld chains cannot fit the %zu-byte static scratch (at most %zu "
             "chains of any d)",
             (long long)n_chains, kStaticScratchBytes, kStaticScratchBytes / kMinChainBytes);
    return fsmc_fail(FSMC_EINVAL, msg);
  }

  // Ring depth: 16 directions per chain, fewer if that is what makes the run fit.
  const int dstride = (d + 31) / 32 * 32;
  int W = 16;
  ScratchLayout lay = layout_for(n_chains, d, W, dstride);
  while (lay.total > kStaticScratchBytes && W > 2) {
    W /= 2;
    lay = layout_for(n_chains, d, W, dstride);
  }
  if (lay.total > kStaticScratchBytes) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "fsmc_ess_run_static: %lld chains x d=%d need %zu scratch bytes; the static scratch "
             "holds %zu (about %lld chains at this d)",
             (long long)n_chains, d, lay.total, kStaticScratchBytes,
             (long long)(n_chains * (double)kStaticScratchBytes / (double)lay.total));
    return fsmc_fail(FSMC_EINVAL, msg);
  }

  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fsmc_cuda_fail(ce, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fsmc_fail(FSMC_EINVAL, "device ordinal too large");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
      void* p = nullptr;
      ce = cudaGetSymbolAddress(&p, g_ess_scratch);
      if (ce != cudaSuccess) return fsmc_cuda_fail(ce, "cudaGetSymbolAddress(static scratch)");
      g_scratch_dev[dev] = p;
    }
    base = g_scratch_dev[dev];
  }
  char* b = (char*)base;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  EssView<float> v{};
  v.m = n_chains;
  v.n = (int)n_samples;
  v.chain0 = 0;
  v.seed_lo = (uint32_t)seed;
  v.seed_hi = (uint32_t)(seed >> 32);
  v.x = (float*)(b + lay.x);
  v.t = (int*)(b + lay.t);
  v.out = samples_dev;
  v.mom = nullptr;
  v.mom_stride = (size_t)n_chains * d;
  v.counts = counts_dev;
  v.steps = (long long*)(b + lay.steps);
  v.err = (int*)(b + lay.misc);
  v.chains_done = (int*)(b + lay.misc) + 1;
  v.tg = TargetView<float>{};
  v.tg.kind = target_kind;
  v.tg.d = d;
  v.tg.n_data = 0;
  v.tg.L = L_dev;
  v.tg.vec = target_kind == FSMC_TGT_FLAT ? nullptr : vec_dev;
  v.tg.s2 = noise_var;
  v.W = W;
  v.dstride = dstride;
  v.ell = (float*)(b + lay.ell);
  v.logy = (float*)(b + lay.logy);
  v.th = (float*)(b + lay.th);
  v.thmin = v.th + n_chains;
  v.thmax = v.th + 2 * n_chains;
  v.k = (int*)(b + lay.k);
  v.s = (int*)(b + lay.s);
  v.gen_lo = (int*)(b + lay.gen);
  v.gen_hi = v.gen_lo + n_chains;
  v.nu = (float*)(b + lay.nu);
  v.gen_cols = (unsigned long long*)((int*)(b + lay.misc) + 2);
  v.own_window = 1;

#define CKS(expr)                                             \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) return fsmc_cuda_fail(_e, #expr);  \
  } while (0)

  // The array keeps the previous call's contents: reset everything that must start at zero.
  const size_t m = (size_t)n_chains;
  CKS(cudaMemcpyAsync(v.x, x0_dev, m * d * sizeof(float), cudaMemcpyDeviceToDevice, st));
  CKS(cudaMemsetAsync(b + lay.t, 0, m * 4, st));
  CKS(cudaMemsetAsync(b + lay.k, 0, m * 4, st));
  CKS(cudaMemsetAsync(b + lay.s, 0, m * 4, st));
  CKS(cudaMemsetAsync(b + lay.th, 0, 3 * m * 4, st));
  CKS(cudaMemsetAsync(b + lay.logy, 0, m * 4, st));
  CKS(cudaMemsetAsync(b + lay.steps, 0, m * 8, st));
  CKS(cudaMemsetAsync(b + lay.misc, 0, 32, st));
  CKS(cudaMemsetAsync(counts_dev, 0xff, m * (size_t)n_samples * 4, st));
  CKS(launch_fill_int(v.gen_lo, n_chains, 0, st));
  CKS(launch_fill_int(v.gen_hi, n_chains, (int)std::min<int64_t>(W, n_samples), st));
  CKS(launch_ess_init<float>(v, st));

  const int steps_per_launch = 2 * W;
  const int threads = 256;
  // Every round advances each unfinished chain by at least one state (its ring is refilled
  // first), so the run ends; the cap below only guards the host loop.
  const int64_t max_rounds = n_samples * (int64_t)(kMaxShrinks + 1) + 16;
  int64_t rounds = 0;
  while (true) {
    int done = 0;
    CKS(cudaMemcpyAsync(&done, v.chains_done, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKS(cudaStreamSynchronize(st));
    if (done >= n_chains) break;
    if (rounds >= max_rounds) return fsmc_fail(FSMC_ETIMEOUT, "fsmc_ess_run_static: round limit reached");
    for (int r = 0; r < 8; ++r) {
      CKS(launch_ess_nu_gen<float>(v, st));
      CKS(launch_ess_fsm<float>(v, lanes_per_chain, steps_per_launch, threads, st));
    }
    rounds += 8;
  }
  int err = 0;
  CKS(cudaMemcpyAsync(&err, v.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CKS(cudaStreamSynchronize(st));
  if (err & ERR_SHRINK_CAP) return fsmc_fail(FSMC_EDEVICE, "fsmc_ess_run_static: shrink cap reached");
  return FSMC_OK;
#undef CKS
}
