// Host engine behind include/fsmc.h: targets, jobs, device memory, the FSM and synchronised
// run loops (Alg. 7 and Alg. 6 on the device), reads, checkpointing and the serving queue.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fsmc_device.cuh"
#include "fsmc_kernels.h"
#include "engine_internal.h"

using namespace fsmc;

// ---- errors ---------------------------------------------------------------------------------------
static thread_local std::string g_last_error;

fsmc_status fsmc_fail(fsmc_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

fsmc_status fsmc_cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear sticky-free errors so later calls can proceed
  return fsmc_fail(FSMC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(expr)                                                   \
  do {                                                             \
    cudaError_t _e = (expr);                                       \
    if (_e != cudaSuccess) return fsmc_cuda_fail(_e, #expr);       \
  } while (0)

extern "C" const char* fsmc_last_error(void) { return g_last_error.c_str(); }

// ---- engine ---------------------------------------------------------------------------------------
extern "C" fsmc_status fsmc_engine_create(int device, size_t hbm_budget_bytes, fsmc_engine** out) {
  if (!out) return fsmc_fail(FSMC_EINVAL, "out is NULL");
  int count = 0;
  CK(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) return fsmc_fail(FSMC_EINVAL, "no such device");
  CK(cudaSetDevice(device));
  size_t free_b = 0, total_b = 0;
  CK(cudaMemGetInfo(&free_b, &total_b));
  auto* e = new (std::nothrow) fsmc_engine();
  if (!e) return fsmc_fail(FSMC_ENOMEM, "host allocation failed");
  e->device = device;
  e->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)free_b);
  CK(cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, device));
  *out = e;
  return FSMC_OK;
}

static void arena_trim(fsmc_engine* e);

extern "C" void fsmc_engine_destroy(fsmc_engine* e) {
  if (!e) return;
  serving_shutdown(e);
  std::vector<fsmc_job*> jobs;
  std::vector<fsmc_target*> tgts;
  {
    std::lock_guard<std::mutex> g(e->mu);
    jobs = e->jobs;
    tgts = e->targets;
  }
  for (auto* j : jobs) fsmc_job_destroy(j);
  for (auto* t : tgts) fsmc_target_destroy(t);
  arena_trim(e);
  delete e;
}

extern "C" size_t fsmc_engine_bytes_in_use(const fsmc_engine* e) {
  if (!e) return 0;
  std::lock_guard<std::mutex> g(e->mu);
  return e->in_use;
}

// Device blocks of destroyed jobs (arenas and starting points) are kept, at most four, and handed
// to the next job they fit (up to twice its size): back-to-back jobs then skip cudaMalloc and
// cudaFree.
static void arena_trim(fsmc_engine* e) {
  std::lock_guard<std::mutex> g(e->mu);
  for (auto& b : e->spare) cudaFree(b.first);
  e->spare.clear();
}

static cudaError_t arena_take(fsmc_engine* e, size_t bytes, char** out, size_t* got) {
  {
    std::lock_guard<std::mutex> g(e->mu);
    int best = -1;
    for (int i = 0; i < (int)e->spare.size(); ++i) {
      const size_t sz = e->spare[i].second;
      if (sz >= bytes && sz <= 2 * bytes && (best < 0 || sz < e->spare[best].second)) best = i;
    }
    if (best >= 0) {
      *out = e->spare[best].first;
      *got = e->spare[best].second;
      e->spare.erase(e->spare.begin() + best);
      return cudaSuccess;
    }
  }
  cudaError_t ce = cudaMalloc((void**)out, bytes);
  if (ce != cudaSuccess) {  // the cached blocks may be what is missing
    cudaGetLastError();
    arena_trim(e);
    ce = cudaMalloc((void**)out, bytes);
  }
  if (ce == cudaSuccess) *got = bytes;
  return ce;
}

static void arena_give(fsmc_engine* e, char* p, size_t bytes) {
  std::lock_guard<std::mutex> g(e->mu);
  e->spare.emplace_back(p, bytes);
  while (e->spare.size() > 4) {
    cudaFree(e->spare.front().first);
    e->spare.erase(e->spare.begin());
  }
}

bool engine_reserve(fsmc_engine* e, size_t bytes) {
  std::lock_guard<std::mutex> g(e->mu);
  if (e->in_use + bytes > e->budget) return false;
  e->in_use += bytes;
  return true;
}

void engine_release(fsmc_engine* e, size_t bytes) {
  std::lock_guard<std::mutex> g(e->mu);
  e->in_use -= std::min(bytes, e->in_use);
  e->cv.notify_all();  // queued serving jobs may fit now
}

// ---- per-launch profiling -------------------------------------------------------------------------
static cudaEvent_t take_event(fsmc_job* j) {
  if (j->event_next == j->event_pool.size()) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
    j->event_pool.push_back(ev);
  }
  return j->event_pool[j->event_next++];
}

ProfScope::ProfScope(fsmc_job* job, int c, cudaStream_t s) : j(job), cls(c), st(s) {
  if (!j->tun.profile_kernels) return;
  a = take_event(j);
  b = take_event(j);
  if (a && b) cudaEventRecord(a, st);
}

ProfScope::~ProfScope() {
  if (!a || !b) return;
  cudaEventRecord(b, st);
  j->prof_events.push_back({cls, {a, b}});
  j->kernel_launches[cls] += 1;
}

static void prof_collect(fsmc_job* j) {
  for (auto& pe : j->prof_events) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess)
      j->kernel_ms[pe.first] += ms;
  }
  cudaGetLastError();
  j->prof_events.clear();
  j->event_next = 0;
}

static void prof_reset(fsmc_job* j) {
  for (int k = 0; k < 4; ++k) { j->kernel_ms[k] = 0; j->kernel_launches[k] = 0; }
  j->prof_events.clear();
  j->event_next = 0;
}

// ---- targets --------------------------------------------------------------------------------------
static bool target_layout(int kind, int d, int n_data, size_t* n_params, bool* needs_L) {
  *needs_L = false;
  switch (kind) {
    case FSMC_TGT_GAUSS_CONJ: *n_params = (size_t)d * d + d + 1; *needs_L = true; return n_data == 0;
    case FSMC_TGT_GP_LOGIT: *n_params = (size_t)d * d + d; *needs_L = true; return n_data == 0;
    case FSMC_TGT_FLAT: *n_params = (size_t)d * d; *needs_L = true; return n_data == 0;
    case FSMC_TGT_FUNNEL: *n_params = 0; return n_data == 0 && d >= 2;
    case FSMC_TGT_LOGREG: *n_params = (size_t)n_data * d + n_data; return n_data >= 1;
    case FSMC_TGT_GAUSS_DIAG: *n_params = 2 * (size_t)d; return n_data == 0;
    case FSMC_TGT_MOG: *n_params = 1 + (size_t)n_data * (d + 1); return n_data >= 1 && n_data <= 64;
    case FSMC_TGT_GP_REG:
      *n_params = (size_t)d * d + (size_t)n_data * n_data + n_data;
      *needs_L = true;
      return d == 3 && n_data >= 1 && n_data <= kGpRegMaxN32;
  }
  return false;
}

template <typename T>
static fsmc_status upload_target(fsmc_target* t, std::vector<void*>& bufs, TargetView<T>& tv) {
  const int d = t->d;
  const double* p = t->params.data();
  auto up = [&](const double* src, size_t n, const T** dst) -> fsmc_status {
    if (n == 0) { *dst = nullptr; return FSMC_OK; }
    std::vector<T> h(src, src + n);
    void* ptr = nullptr;
    CK(cudaMalloc(&ptr, n * sizeof(T)));
    bufs.push_back(ptr);
    t->bytes += n * sizeof(T);
    CK(cudaMemcpy(ptr, h.data(), n * sizeof(T), cudaMemcpyHostToDevice));
    *dst = (const T*)ptr;
    return FSMC_OK;
  };
  tv = TargetView<T>{};
  tv.kind = t->kind;
  tv.d = d;
  tv.n_data = t->n_data;
  fsmc_status st = FSMC_OK;
  switch (t->kind) {
    case FSMC_TGT_GAUSS_CONJ:
      if ((st = up(p, (size_t)d * d, &tv.L))) return st;
      if ((st = up(p + (size_t)d * d, d, &tv.vec))) return st;
      tv.s2 = (T)p[(size_t)d * d + d];
      break;
    case FSMC_TGT_GP_LOGIT:
      if ((st = up(p, (size_t)d * d, &tv.L))) return st;
      if ((st = up(p + (size_t)d * d, d, &tv.vec))) return st;
      break;
    case FSMC_TGT_FLAT:
      if ((st = up(p, (size_t)d * d, &tv.L))) return st;
      break;
    case FSMC_TGT_LOGREG: {
      if ((st = up(p, (size_t)t->n_data * d, &tv.X))) return st;
      if ((st = up(p + (size_t)t->n_data * d, t->n_data, &tv.vec))) return st;
      // transposed copy for the batched gradient: [d][n_pad], zero rows beyond n_data
      const int n = t->n_data, np = (n + 3) / 4 * 4;
      std::vector<double> xt((size_t)d * np, 0.0);
      for (int i = 0; i < n; ++i)
        for (int k = 0; k < d; ++k) xt[(size_t)k * np + i] = p[(size_t)i * d + k];
      if ((st = up(xt.data(), xt.size(), &tv.XT))) return st;
      tv.n_pad = np;
      break;
    }
    case FSMC_TGT_GAUSS_DIAG:
      if ((st = up(p, d, &tv.vec))) return st;
      if ((st = up(p + d, d, &tv.vec2))) return st;
      break;
    case FSMC_TGT_GP_REG: {
      const size_t n = (size_t)t->n_data;
      if ((st = up(p, (size_t)d * d, &tv.L))) return st;
      if ((st = up(p + (size_t)d * d, n * n, &tv.X))) return st;
      if ((st = up(p + (size_t)d * d + n * n, n, &tv.vec))) return st;
      break;
    }
    case FSMC_TGT_MOG: {
      const int K = t->n_data;
      const double rho = p[0];
      std::vector<double> lw(K);
      for (int k = 0; k < K; ++k) lw[k] = std::log(p[1 + k]);
      if ((st = up(p + 1 + K, (size_t)K * d, &tv.X))) return st;
      if ((st = up(lw.data(), K, &tv.vec))) return st;
      tv.c_par = (T)(1.0 / (1.0 + (d - 1) * rho));
      tv.c_perp = (T)(1.0 / (1.0 - rho));
      break;
    }
    default:
      break;
  }
  return FSMC_OK;
}

extern "C" fsmc_status fsmc_target_create(fsmc_engine* e, fsmc_target_kind kind, int d, int n_data,
                                          const double* params_host, size_t n_params,
                                          fsmc_target** out) {
  if (!e || !out) return fsmc_fail(FSMC_EINVAL, "engine/out is NULL");
  size_t need = 0;
  bool needs_L = false;
  if (d < 1 || d > 1024 || n_data < 0 || !target_layout(kind, d, n_data, &need, &needs_L))
    return fsmc_fail(FSMC_EINVAL, "invalid target kind / d / n_data");
  if (n_params != need) return fsmc_fail(FSMC_EINVAL, "n_params does not match the target layout");
  if (need && !params_host) return fsmc_fail(FSMC_EINVAL, "params_host is NULL");
  if (kind == FSMC_TGT_MOG) {
    const double rho = params_host[0];
    if (!(rho < 1.0) || (d > 1 && !(rho > -1.0 / (d - 1))))
      return fsmc_fail(FSMC_EINVAL, "MOG needs -1/(d-1) < rho < 1");
    for (int k = 0; k < n_data; ++k) {
      const double wk = params_host[1 + k];
      if (!(wk > 0.0) || !std::isfinite(wk)) return fsmc_fail(FSMC_EINVAL, "MOG weights must be positive");
    }
    for (size_t i = 1 + (size_t)n_data; i < need; ++i)
      if (!std::isfinite(params_host[i])) return fsmc_fail(FSMC_EINVAL, "MOG means must be finite");
  }
  if (kind == FSMC_TGT_GP_LOGIT)
    for (int k = 0; k < d; ++k) {
      const double s = params_host[(size_t)d * d + k];
      if (s != 1.0 && s != -1.0) return fsmc_fail(FSMC_EINVAL, "GP_LOGIT labels must be -1 or +1");
    }
  CK(cudaSetDevice(e->device));
  auto* t = new (std::nothrow) fsmc_target();
  if (!t) return fsmc_fail(FSMC_ENOMEM, "host allocation failed");
  t->e = e;
  t->kind = kind;
  t->d = d;
  t->n_data = n_data;
  t->params.assign(params_host, params_host + need);
  fsmc_status st = upload_target<float>(t, t->bufs, t->tv32);
  if (st == FSMC_OK) st = upload_target<double>(t, t->bufs, t->tv64);
  if (st != FSMC_OK) {
    for (void* b : t->bufs) cudaFree(b);
    delete t;
    return st;
  }
  {
    std::lock_guard<std::mutex> g(e->mu);
    e->in_use += t->bytes;
    e->targets.push_back(t);
  }
  *out = t;
  return FSMC_OK;
}

extern "C" void fsmc_target_destroy(fsmc_target* t) {
  if (!t) return;
  fsmc_engine* e = t->e;
  cudaSetDevice(e->device);
  for (void* b : t->bufs) cudaFree(b);
  if (t->tc_img) cudaFree(t->tc_img);
  {
    std::lock_guard<std::mutex> g(e->mu);
    e->in_use -= std::min(t->bytes, e->in_use);
    e->targets.erase(std::remove(e->targets.begin(), e->targets.end(), t), e->targets.end());
  }
  delete t;
}

// ---- jobs -----------------------------------------------------------------------------------------
static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  }
};

// ESS on a target whose likelihood is one dense problem per evaluation: a chain per CTA.
static bool ess_block(const fsmc_job* j) { return j->algo == FSMC_ESS && j->tg->kind == FSMC_TGT_GP_REG; }

// Decides the launch shape when the caller left it open.
static void default_tuning(fsmc_job* j) {
  fsmc_tuning& tu = j->tun;
  if (!tu.step_form) tu.step_form = 1;
  if (ess_block(j)) {
    tu.lanes_per_chain = 32;  // a warp (and CTA) per chain
    tu.ring_slots = 0;
    tu.generator = 0;
    tu.pipelined = 2;
    // a CTA of 1, 2 or 4 warps per chain, more when there are too few chains to fill the SMs
    if (!tu.threads_per_block) tu.threads_per_block = 32 * ess_block_auto_wpc(j->m, j->e->sms);
    if (!tu.steps_per_launch) tu.steps_per_launch = 8;
  } else if (j->algo == FSMC_ESS) {
    if (!tu.lanes_per_chain && tu.sync_form == 4) tu.lanes_per_chain = 32;  // the resident form's layout
    if (!tu.lanes_per_chain) {
      // chain-per-warp when one chain's likelihood is wide (d >= 64) or when there are too
      // few chains to fill the machine one per thread
      const int64_t thread_slots = (int64_t)j->e->sms * 1024;
      tu.lanes_per_chain = (j->d > 32 || j->d >= 64 || j->m * 8 < thread_slots) ? 32 : 1;
    }
    if (!tu.generator) tu.generator = (j->prec == FSMC_FP32 && j->d <= 256) ? 2 : 1;
    // Large jobs on the tensor-core generator take long rounds: each refill launch pays a fixed
    // cost (the L image's copy into every CTA, tensor-memory set-up, pipeline fill and drain)
    // and each FSM launch a tail, so fewer, larger rounds are faster (16384 chains, d = 256:
    // 51.2 ms per job at 64 states per launch and 32 ring slots, 47.5 at 192 / 64, 46.6 at
    // 384 / 128, 44.3 at 512 / 256 with the current step).  The ring grows with them
    // (m x 256 x d x 4 bytes, 4.3 GB at 16384 x 256).  Smaller jobs keep short rounds, which
    // also bound a serving round's length.
    const bool long_rounds = tu.generator == 2 && j->m >= 4096;
    if (!tu.steps_per_launch) tu.steps_per_launch = long_rounds ? 512 : 64;
    if (!tu.ring_slots) tu.ring_slots = long_rounds ? 256 : 32;
    if (!tu.threads_per_block) tu.threads_per_block = 256;
    if (!tu.pipelined) tu.pipelined = 1;
    if (!tu.sync_form) tu.sync_form = 2;
  } else if (j->algo == FSMC_DR || j->algo == FSMC_SLICE) {
    // a chain per thread while its state fits a thread's registers (d <= 32), else a chain per
    // warp (DR), its density's sums taken across the warp
    if (!tu.lanes_per_chain) tu.lanes_per_chain = j->d > 32 ? 32 : 1;
    // long launches: fewer kernel tails (funnel, 65536 chains: DR 48.8 -> 48.0 ms, slice 47.4 ->
    // 45.9 ms per job from 256 to 1024 states per launch)
    if (!tu.steps_per_launch) tu.steps_per_launch = 1024;
    // chain per thread: 256-thread blocks (funnel, 65536 chains, ms per job for 32 / 64 / 128 /
    // 256 threads: DR 45.8 / 45.9 / 45.9 / 44.4, slice 43.9 / 44.1 / 44.0 / 43.6); chain per
    // warp: 128 (the warp kernels' bound)
    if (!tu.threads_per_block) tu.threads_per_block = tu.lanes_per_chain == 1 ? 256 : 128;
  } else {
    if (!tu.lanes_per_chain) tu.lanes_per_chain = 32;
    // leapfrog steps per launch: enough that a launch's tail (its slowest warp) and the launch
    // gaps stay small against its length; cheap log-densities take more
    if (!tu.steps_per_launch) tu.steps_per_launch = j->tg->kind == FSMC_TGT_LOGREG ? 128 : 256;
    if (!tu.threads_per_block) tu.threads_per_block = 128;
  }
}

static fsmc_status job_layout_and_alloc(fsmc_job* j) {
  const size_t es = j->prec == FSMC_FP64 ? 8 : 4;
  const size_t m = (size_t)j->m, n = (size_t)j->n, d = (size_t)j->d;
  Layout L;
  j->o_x = L.take(m * d * es);
  j->o_t = L.take(m * 4);
  j->o_counts = L.take(m * n * 4);
  j->o_steps = L.take(m * 8);
  j->o_err = L.take(4);
  j->o_done = L.take(4);
  j->o_out = j->store ? L.take(m * n * d * es) : 0;
  j->o_mom = L.take(4 * m * d * es);  // running sums (moments-only jobs) or their reduction
  j->o_momd = L.take(2 * m * d * 8);  // the sums as doubles, for the host read
  j->o_bar = L.take(64);
  j->o_gbar = L.take(fsmc::kGridBarrierBytes);
  j->o_iters = L.take(8);
  j->o_stats = L.take(align_up(n * 4, 64) + sizeof(fsmc::DevStats));
  if (ess_block(j)) {
    j->o_ell = L.take(m * es);
    j->o_logy = L.take(m * es);
    j->o_th = L.take(3 * m * es);
    j->o_k = L.take(m * 4);
    j->o_s = L.take(m * 4);
    j->o_nu = L.take(m * d * es);
    j->o_gencols = L.take(8);
    j->o_work = L.take(8);
    // scratch for covariance rows beyond shared memory: one block per CTA that can be resident
    // (shared memory bounds CTAs per SM)
    const size_t spill = es == 8 ? gpreg_spill_elems<double>(j->tg->n_data) : gpreg_spill_elems<float>(j->tg->n_data);
    j->spill_stride = spill;
    j->rows_smem = es == 8 ? gpreg_smem_rows<double>(j->tg->n_data) : gpreg_smem_rows<float>(j->tg->n_data);
    j->spill_ctas = spill ? (int64_t)j->e->sms * 2 : 0;
    j->o_spill = spill ? L.take((size_t)j->spill_ctas * spill * es) : 0;
  } else if (j->algo == FSMC_ESS) {
    j->W = j->tun.ring_slots;
    j->dstride = (int)align_up(d, 32);
    j->o_ell = L.take(m * es);
    j->o_logy = L.take(m * es);
    j->o_th = L.take(3 * m * es);
    j->o_k = L.take(m * 4);
    j->o_s = L.take(m * 4);
    j->o_gen = L.take(2 * m * 4);
    j->o_nu = L.take(m * (size_t)j->W * j->dstride * es);
    j->o_gencols = L.take(8);
    j->o_win = L.take(2 * m * 4);
    j->o_colbase = L.take((m + 1) * 8);
    j->o_colmap = L.take(m * (size_t)j->W * 8);
    j->o_slist = L.take(2 * m * 4 + fsmc::kEssCgStateBytes);
  } else if (j->algo == FSMC_DR) {
    j->o_ell = L.take(m * es);        // log pi(x)
    j->o_y = L.take(3 * m * d * es);  // y1, y2 and (4-state ablation form) the current proposal
    j->o_lpy = L.take(10 * m * es);   // log pi(y1), log pi(y2), current proposal's and its ratio,
                                      // then the kept terms of the later stages' ratios
    j->o_k = L.take(m * 4);
  } else if (j->algo == FSMC_SLICE) {
    j->o_ell = L.take(m * es);        // log pi(x)
    j->o_logy = L.take(m * es);
    j->o_th = L.take(3 * m * es);     // L, R, theta
    j->o_y = L.take(m * d * es);      // direction u
    j->o_k = L.take(5 * m * 4);       // state, J, K, proposals, evaluations
    j->o_aux = L.take(m * n * 4);
  } else {
    nuts_layout(j, L.off);
  }
  j->bytes = L.off;
  if (!engine_reserve(j->e, j->bytes)) {
    char msg[256];
    snprintf(msg, sizeof msg, "job needs %zu device bytes; engine budget %zu, in use %zu",
             j->bytes, j->e->budget, fsmc_engine_bytes_in_use(j->e));
    return fsmc_fail(FSMC_EADMIT, msg);
  }
  cudaError_t ce = arena_take(j->e, j->bytes, &j->dev, &j->arena_bytes);
  if (ce != cudaSuccess) {
    engine_release(j->e, j->bytes);
    j->dev = nullptr;
    cudaGetLastError();
    return fsmc_fail(FSMC_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(ce));
  }
  return FSMC_OK;
}

template <typename T>
static void fill_chains(const fsmc_job* j, ChainsView<T>& v) {
  char* b = j->dev;
  v.m = j->m;
  v.n = (int)j->n;
  v.chain0 = j->chain0;
  v.seed_lo = (uint32_t)j->seed;
  v.seed_hi = (uint32_t)(j->seed >> 32);
  v.x = (T*)(b + j->o_x);
  v.t = (int*)(b + j->o_t);
  v.out = j->store ? (T*)(b + j->o_out) : nullptr;
  v.mom = j->store ? nullptr : (T*)(b + j->o_mom);
  v.mom_stride = (size_t)j->m * j->d;
  v.counts = (int*)(b + j->o_counts);
  v.steps = (long long*)(b + j->o_steps);
  v.err = (int*)(b + j->o_err);
  v.chains_done = (int*)(b + j->o_done);
  v.step_form = j->tun.step_form ? j->tun.step_form : 1;
}

template <typename T>
const TargetView<T>& target_view(const fsmc_target* t);
template <>
const TargetView<float>& target_view<float>(const fsmc_target* t) { return t->tv32; }
template <>
const TargetView<double>& target_view<double>(const fsmc_target* t) { return t->tv64; }

template <typename T>
EssView<T> ess_view(const fsmc_job* j) {
  EssView<T> v;
  fill_chains<T>(j, v);
  char* b = j->dev;
  v.tg = target_view<T>(j->tg);
  v.W = j->W;
  v.dstride = j->dstride;
  v.ell = (T*)(b + j->o_ell);
  v.logy = (T*)(b + j->o_logy);
  v.th = (T*)(b + j->o_th);
  v.thmin = v.th + j->m;
  v.thmax = v.th + 2 * j->m;
  v.k = (int*)(b + j->o_k);
  v.s = (int*)(b + j->o_s);
  v.gen_lo = (int*)(b + j->o_gen);
  v.gen_hi = v.gen_lo + j->m;
  v.nu = (T*)(b + j->o_nu);
  v.gen_cols = (unsigned long long*)(b + j->o_gencols);
  v.own_window = 1;
  v.col_base = (long long*)(b + j->o_colbase);
  v.colmap = (int2*)(b + j->o_colmap);
  return v;
}

template <typename T>
DrView<T> dr_view(const fsmc_job* j) {
  DrView<T> v;
  fill_chains<T>(j, v);
  char* b = j->dev;
  v.tg = target_view<T>(j->tg);
  v.n_stages = j->dr.n_stages;
  v.symmetric = j->dr.symmetric;
  for (int k = 0; k < 3; ++k)
    v.sig[k] = (T)(j->dr.symmetric ? j->dr.scale0 : j->dr.scale0 * std::pow(j->dr.factor, (double)k));
  v.lp = (T*)(b + j->o_ell);
  v.y = (T*)(b + j->o_y);
  v.lpy = (T*)(b + j->o_lpy);
  v.k = (int*)(b + j->o_k);
  v.lanes = j->tun.lanes_per_chain;
  return v;
}

template <typename T>
EssBlockView<T> ess_block_view(const fsmc_job* j) {
  EssBlockView<T> v;
  fill_chains<T>(j, v);
  char* b = j->dev;
  v.tg = target_view<T>(j->tg);
  v.ell = (T*)(b + j->o_ell);
  v.logy = (T*)(b + j->o_logy);
  v.th = (T*)(b + j->o_th);
  v.thmin = v.th + j->m;
  v.thmax = v.th + 2 * j->m;
  v.nu = (T*)(b + j->o_nu);
  v.k = (int*)(b + j->o_k);
  v.s = (int*)(b + j->o_s);
  v.work = (unsigned*)(b + j->o_work);
  v.spill = j->spill_stride ? (T*)(b + j->o_spill) : nullptr;
  v.spill_stride = j->spill_stride;
  v.max_ctas = j->spill_stride ? j->spill_ctas : INT64_MAX;
  v.rows_smem = j->rows_smem;
  v.wpc = j->tun.threads_per_block / 32;  // set by default_tuning when the caller left it open
  return v;
}

template <typename T>
SliceView<T> slice_view(const fsmc_job* j) {
  SliceView<T> v;
  fill_chains<T>(j, v);
  char* b = j->dev;
  v.tg = target_view<T>(j->tg);
  v.w = (T)j->slice.w;
  v.mlim = j->slice.m;
  v.lp = (T*)(b + j->o_ell);
  v.logy = (T*)(b + j->o_logy);
  v.L = (T*)(b + j->o_th);
  v.R = v.L + j->m;
  v.th = v.L + 2 * j->m;
  v.u = (T*)(b + j->o_y);
  v.k = (int*)(b + j->o_k);
  v.J = v.k + j->m;
  v.K = v.k + 2 * j->m;
  v.s = v.k + 3 * j->m;
  v.nev = v.k + 4 * j->m;
  v.aux = (int*)(b + j->o_aux);
  v.lanes = j->tun.lanes_per_chain;
  return v;
}

template <typename T>
static fsmc_status job_init_state(fsmc_job* j, cudaStream_t st) {
  char* b = j->dev;
  const size_t m = (size_t)j->m, d = (size_t)j->d;
  CK(launch_from_double<T>((const double*)j->x0_dev, (int64_t)(m * d), (T*)(b + j->o_x), st));
  CK(cudaMemsetAsync(b + j->o_t, 0, m * 4, st));
  CK(cudaMemsetAsync(b + j->o_counts, 0xff, m * (size_t)j->n * 4, st));
  CK(cudaMemsetAsync(b + j->o_steps, 0, m * 8, st));
  CK(cudaMemsetAsync(b + j->o_err, 0, 4, st));
  CK(cudaMemsetAsync(b + j->o_done, 0, 4, st));
  CK(cudaMemsetAsync(b + j->o_bar, 0, 64, st));
  CK(cudaMemsetAsync(b + j->o_gbar, 0, fsmc::kGridBarrierBytes, st));
  CK(cudaMemsetAsync(b + j->o_iters, 0, 8, st));
  if (!j->store) CK(cudaMemsetAsync(b + j->o_mom, 0, 4 * m * d * sizeof(T), st));
  if (ess_block(j)) {
    CK(cudaMemsetAsync(b + j->o_s, 0, m * 4, st));
    CK(cudaMemsetAsync(b + j->o_th, 0, 3 * m * sizeof(T), st));
    CK(cudaMemsetAsync(b + j->o_logy, 0, m * sizeof(T), st));
    CK(cudaMemsetAsync(b + j->o_nu, 0, m * d * sizeof(T), st));
    CK(cudaMemsetAsync(b + j->o_gencols, 0, 8, st));
    CK(launch_ess_block_init<T>(ess_block_view<T>(j), st));
  } else if (j->algo == FSMC_ESS) {
    CK(cudaMemsetAsync(b + j->o_k, 0, m * 4, st));
    CK(cudaMemsetAsync(b + j->o_s, 0, m * 4, st));
    CK(cudaMemsetAsync(b + j->o_th, 0, 3 * m * sizeof(T), st));
    CK(cudaMemsetAsync(b + j->o_logy, 0, m * sizeof(T), st));
    CK(cudaMemsetAsync(b + j->o_gencols, 0, 8, st));
    int* gen = (int*)(b + j->o_gen);
    CK(launch_fill_int(gen, j->m, 0, st));
    CK(launch_fill_int(gen + j->m, j->m, (int)std::min<int64_t>(j->W, j->n), st));
    CK(launch_ess_init<T>(ess_view<T>(j), st));
  } else if (j->algo == FSMC_DR) {
    CK(cudaMemsetAsync(b + j->o_k, 0, m * 4, st));
    CK(cudaMemsetAsync(b + j->o_y, 0, 3 * m * d * sizeof(T), st));
    CK(cudaMemsetAsync(b + j->o_lpy, 0, 10 * m * sizeof(T), st));
    CK(launch_dr_init<T>(dr_view<T>(j), st));
  } else if (j->algo == FSMC_SLICE) {
    CK(cudaMemsetAsync(b + j->o_k, 0, 5 * m * 4, st));
    CK(cudaMemsetAsync(b + j->o_th, 0, 3 * m * sizeof(T), st));
    CK(cudaMemsetAsync(b + j->o_aux, 0xff, m * (size_t)j->n * 4, st));
    CK(launch_slice_init<T>(slice_view<T>(j), st));
  } else {
    fsmc_status s = nuts_init_state(j, st);
    if (s != FSMC_OK) return s;
  }
  CK(cudaStreamSynchronize(st));
  j->sync_used = false;
  j->fsm_used = false;
  return FSMC_OK;
}

static fsmc_status job_init(fsmc_job* j, cudaStream_t st) {
  return j->prec == FSMC_FP64 ? job_init_state<double>(j, st) : job_init_state<float>(j, st);
}

extern "C" fsmc_status fsmc_job_create(fsmc_engine* e, fsmc_target* t, fsmc_algo algo,
                                       const void* algo_params, fsmc_precision prec,
                                       int64_t n_chains, int64_t n_samples, const double* x0_host,
                                       uint64_t seed, int store_samples, fsmc_job** out) {
  if (!e || !t || !out) return fsmc_fail(FSMC_EINVAL, "engine/target/out is NULL");
  if (n_chains < 1 || n_chains > (int64_t)1 << 31 || n_samples < 1 || n_samples > (int64_t)1 << 30)
    return fsmc_fail(FSMC_EINVAL, "n_chains / n_samples out of range");
  if (prec != FSMC_FP32 && prec != FSMC_FP64) return fsmc_fail(FSMC_EINVAL, "bad precision");
  const bool ess_kind = t->kind == FSMC_TGT_GAUSS_CONJ || t->kind == FSMC_TGT_GP_LOGIT ||
                        t->kind == FSMC_TGT_FLAT || t->kind == FSMC_TGT_GP_REG;
  if (algo == FSMC_ESS && !ess_kind) return fsmc_fail(FSMC_EINVAL, "ESS needs a target with a Gaussian prior factor");
  if ((algo == FSMC_DR || algo == FSMC_NUTS || algo == FSMC_SLICE) && ess_kind)
    return fsmc_fail(FSMC_EINVAL, "DR / NUTS / slice sampling need a full log-density target");
  if (algo != FSMC_ESS && algo != FSMC_DR && algo != FSMC_NUTS && algo != FSMC_SLICE)
    return fsmc_fail(FSMC_EINVAL, "bad algo");
  if (algo == FSMC_DR && t->d > 1024) return fsmc_fail(FSMC_EINVAL, "DR supports d <= 1024");
  if (t->kind == FSMC_TGT_GP_REG && prec == FSMC_FP64 && t->n_data > kGpRegMaxN64)
    return fsmc_fail(FSMC_EINVAL, "FP64 GP_REG jobs support n_data <= 512");
  if (algo == FSMC_SLICE && t->d > 1024) return fsmc_fail(FSMC_EINVAL, "slice sampling supports d <= 1024");
  auto* j = new (std::nothrow) fsmc_job();
  if (!j) return fsmc_fail(FSMC_ENOMEM, "host allocation failed");
  j->e = e;
  j->tg = t;
  j->algo = algo;
  j->prec = prec;
  j->m = n_chains;
  j->n = n_samples;
  j->d = t->d;
  j->seed = seed;
  j->store = store_samples ? 1 : 0;
  if (algo == FSMC_DR) {
    j->dr = algo_params ? *(const fsmc_dr_params*)algo_params : fsmc_dr_params{3, 1.0, 0.5, 0};
    const int max_stages = j->dr.symmetric ? 1000 : 3;
    if (j->dr.n_stages < 1 || j->dr.n_stages > max_stages || !(j->dr.scale0 > 0) ||
        !(j->dr.symmetric || j->dr.factor > 0) || (j->dr.symmetric != 0 && j->dr.symmetric != 1)) {
      delete j;
      return fsmc_fail(FSMC_EINVAL, "DR params: 1..3 stages (symmetric: 1..1000 tries), positive scales");
    }
  }
  if (algo == FSMC_SLICE) {
    j->slice = algo_params ? *(const fsmc_slice_params*)algo_params : fsmc_slice_params{1.0, 100};
    if (!(j->slice.w > 0) || !std::isfinite(j->slice.w) || j->slice.m < 1 || j->slice.m > 1000000) {
      delete j;
      return fsmc_fail(FSMC_EINVAL, "slice params: w > 0, 1 <= m <= 1000000");
    }
  }
  if (algo == FSMC_NUTS) {
    j->nuts = algo_params ? *(const fsmc_nuts_params*)algo_params : fsmc_nuts_params{0.05, 10, 1000.0};
    if (!(j->nuts.eps > 0) || j->nuts.max_depth < 1 || j->nuts.max_depth > 10 || !(j->nuts.max_dH > 0)) {
      delete j;
      return fsmc_fail(FSMC_EINVAL, "NUTS params: eps > 0, 1 <= max_depth <= 10, max_dH > 0");
    }
  }
  {  // the starting points go to the device now (one copy; fast from pinned memory)
    const size_t xb = (size_t)n_chains * t->d * sizeof(double);
    CK(cudaSetDevice(e->device));
    cudaError_t ce = arena_take(e, xb, &j->x0_dev, &j->x0_block);
    if (ce == cudaSuccess)
      ce = x0_host ? cudaMemcpy(j->x0_dev, x0_host, xb, cudaMemcpyHostToDevice) : cudaMemset(j->x0_dev, 0, xb);
    if (ce != cudaSuccess) {
      if (j->x0_dev) arena_give(e, j->x0_dev, j->x0_block);
      delete j;
      cudaGetLastError();
      return fsmc_fail(FSMC_ENOMEM, std::string("starting points: ") + cudaGetErrorString(ce));
    }
  }
  default_tuning(j);
  {
    std::lock_guard<std::mutex> g(e->mu);
    e->jobs.push_back(j);
  }
  *out = j;
  return FSMC_OK;
}

// Allocation and state initialisation happen on first use so that a queued serving job
// holds no device memory until it is admitted.
fsmc_status job_materialize(fsmc_job* j, cudaStream_t st) {
  if (j->dev) return FSMC_OK;
  CK(cudaSetDevice(j->e->device));
  fsmc_status s = job_layout_and_alloc(j);
  if (s != FSMC_OK) return s;
  return job_init(j, st);
}

extern "C" fsmc_status fsmc_job_set_tuning(fsmc_job* j, const fsmc_tuning* tu) {
  if (!j || !tu) return fsmc_fail(FSMC_EINVAL, "NULL argument");
  if (j->dev) return fsmc_fail(FSMC_ESTATE, "tuning must be set before the first run");
  fsmc_tuning t = *tu;
  if (ess_block(j) && ((t.lanes_per_chain && t.lanes_per_chain != 32) || t.generator || t.ring_slots ||
                       t.step_form == 2 ||
                       (t.threads_per_block && t.threads_per_block != 32 && t.threads_per_block != 64 &&
                        t.threads_per_block != 128)))
    return fsmc_fail(FSMC_EINVAL,
                     "GP_REG jobs run a CTA of 1, 2 or 4 warps per chain; only steps_per_launch and "
                     "threads_per_block (32, 64, 128) are tunable");
  if (t.lanes_per_chain && t.lanes_per_chain != 1 && t.lanes_per_chain != 8 && t.lanes_per_chain != 16 &&
      t.lanes_per_chain != 32)
    return fsmc_fail(FSMC_EINVAL, "lanes_per_chain must be 1, 8, 16 or 32");
  if ((j->algo == FSMC_DR || j->algo == FSMC_SLICE) && (t.lanes_per_chain == 8 || t.lanes_per_chain == 16))
    return fsmc_fail(FSMC_EINVAL, "DR and slice sampling run a chain per thread (d <= 32) or per warp");
  if ((j->algo == FSMC_DR || j->algo == FSMC_SLICE) && t.lanes_per_chain == 1 && j->d > 32)
    return fsmc_fail(FSMC_EINVAL, "chain-per-thread DR and slice sampling support d <= 32");
  if (j->algo == FSMC_DR && t.step_form == 2 && (t.lanes_per_chain == 32 || j->d > 32))
    return fsmc_fail(FSMC_EINVAL, "the 4-state DR ablation form runs a chain per thread only");
  if (t.lanes_per_chain == 16 && (j->algo != FSMC_ESS || j->d <= 32 || j->d > 512))
    return fsmc_fail(FSMC_EINVAL, "16 lanes per chain: ESS jobs with 32 < d <= 512");
  if (t.lanes_per_chain == 8 && (j->algo != FSMC_ESS || j->d <= 32 || j->d > 256))
    return fsmc_fail(FSMC_EINVAL, "8 lanes per chain: ESS jobs with 32 < d <= 256");
  if (j->algo == FSMC_NUTS && t.lanes_per_chain && t.lanes_per_chain != 32)
    return fsmc_fail(FSMC_EINVAL, "NUTS is chain-per-warp (32 lanes)");
  if (j->algo == FSMC_ESS && t.lanes_per_chain == 1 && j->d > 32)
    return fsmc_fail(FSMC_EINVAL, "chain-per-thread ESS supports d <= 32");
  if (t.threads_per_block && (t.threads_per_block % 32 || t.threads_per_block < 32 || t.threads_per_block > 256))
    return fsmc_fail(FSMC_EINVAL, "threads_per_block must be a multiple of 32 in [32, 256]");
  if (t.steps_per_launch < 0 || t.ring_slots < 0 || t.ring_slots > 4096)
    return fsmc_fail(FSMC_EINVAL, "negative steps / ring slots");
  // a launch's state budget plus a sample's shrink offsets stays far inside int
  if (t.steps_per_launch > (1 << 24))
    return fsmc_fail(FSMC_EINVAL, "steps_per_launch must be at most 2^24");
  if (t.generator < 0 || t.generator > 2) return fsmc_fail(FSMC_EINVAL, "generator must be 0, 1 or 2");
  if (t.pipelined < 0 || t.pipelined > 2) return fsmc_fail(FSMC_EINVAL, "pipelined must be 0, 1 or 2");
  if (t.step_form < 0 || t.step_form > 2) return fsmc_fail(FSMC_EINVAL, "step_form must be 0, 1 or 2");
  if (t.step_form == 2 && (j->algo == FSMC_NUTS || j->algo == FSMC_SLICE))
    return fsmc_fail(FSMC_EINVAL, "NUTS and slice sampling have step form 1 only");
  if (t.generator == 2 && (j->algo != FSMC_ESS || j->prec != FSMC_FP32 || j->d > 256))
    return fsmc_fail(FSMC_EINVAL, "the tensor-core generator needs an FP32 ESS job with d <= 256");
  if (t.barrier_spin_limit < 0 || t.barrier_test_missing < 0 || t.barrier_test_missing > 1)
    return fsmc_fail(FSMC_EINVAL, "barrier_spin_limit must be >= 0 and barrier_test_missing 0 or 1");
  if (t.sync_form < 0 || t.sync_form > 4) return fsmc_fail(FSMC_EINVAL, "sync_form must be 0, 1, 2, 3 or 4");
  if (t.sync_form == 4 &&
      !(j->algo == FSMC_ESS && !ess_block(j) && j->prec == FSMC_FP32 && j->tg->kind == FSMC_TGT_GP_LOGIT &&
        (j->d == 32 || j->d == 64 || j->d == 128 || j->d == 256) &&
        (t.lanes_per_chain == 0 || t.lanes_per_chain == 32) && t.step_form != 2))
    return fsmc_fail(FSMC_EINVAL,
                     "sync_form 4 (resident) needs a single-precision GP-logit ESS job, 32 lanes per chain, "
                     "d of 32, 64, 128 or 256");
  if (t.sync_form == 3 && t.barrier_test_missing)
    return fsmc_fail(FSMC_EINVAL, "the graph form of the synchronised program has no grid barrier");
  j->tun = t;
  default_tuning(j);
  return FSMC_OK;
}

extern "C" fsmc_status fsmc_job_get_tuning(const fsmc_job* j, fsmc_tuning* tu) {
  if (!j || !tu) return fsmc_fail(FSMC_EINVAL, "NULL argument");
  *tu = j->tun;
  return FSMC_OK;
}

extern "C" size_t fsmc_job_bytes(const fsmc_job* j) { return j ? j->bytes : 0; }

// ---- run loops -------------------------------------------------------------------------------------
// Refills the ESS direction rings with the job's generator (tensor cores or CUDA cores).
template <typename T>
static cudaError_t ess_generate(fsmc_job* j, const EssView<T>& v, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (j->tun.generator == 2) {
      fsmc_target* t = j->tg;
      if (!t->tc_img) {
        cudaError_t e = cudaMalloc((void**)&t->tc_img, ess_tc_image_bytes(t->d));
        if (e != cudaSuccess) { t->tc_img = nullptr; return e; }
        e = launch_ess_tc_build(t->tv32.L, t->d, t->tc_img, st);
        if (e != cudaSuccess) return e;
      }
      return launch_ess_nu_gen_tc(v, t->tc_img, j->e->sms, st);
    }
  }
  return launch_ess_nu_gen<T>(v, st);
}

// kernels one ess_generate call launches: prefix sum, column list and generator on the tensor
// cores, the generator alone on the CUDA cores
static int ess_generate_kernels(const fsmc_job* j) {
  return (j->prec == FSMC_FP32 && j->tun.generator == 2) ? 3 : 1;
}

// One FSM round: (ESS) refill the rings, then advance every chain by the step budget.
template <typename T>
static cudaError_t fsm_round(fsmc_job* j, cudaStream_t st) {
  const fsmc_tuning& tu = j->tun;
  cudaError_t e;
  if (ess_block(j)) {
    ProfScope p(j, 1, st);
    e = launch_ess_block_fsm<T>(ess_block_view<T>(j), tu.steps_per_launch, st);
    j->launches += 1;
  } else if (j->algo == FSMC_ESS) {
    const EssView<T> v = ess_view<T>(j);
    {
      ProfScope p(j, 0, st);
      if ((e = ess_generate<T>(j, v, st)) != cudaSuccess) return e;
    }
    ProfScope p(j, 1, st);
    e = launch_ess_fsm<T>(v, tu.lanes_per_chain, tu.steps_per_launch, tu.threads_per_block, st);
    j->launches += ess_generate_kernels(j) + 1;
  } else if (j->algo == FSMC_DR) {
    ProfScope p(j, 1, st);
    e = launch_dr_fsm<T>(dr_view<T>(j), tu.steps_per_launch, tu.threads_per_block, st);
    j->launches += 1;
  } else if (j->algo == FSMC_SLICE) {
    ProfScope p(j, 1, st);
    e = launch_slice_fsm<T>(slice_view<T>(j), tu.steps_per_launch, tu.threads_per_block, st);
    j->launches += 1;
  } else {
    ProfScope p(j, 1, st);
    e = nuts_fsm_round(j, st);
    j->launches += 1;
  }
  return e;
}

static fsmc_status read_done(fsmc_job* j, cudaStream_t st, int* done_chains, int* err) {
  int h[2] = {0, 0};
  CK(cudaMemcpyAsync(&h[0], j->dev + j->o_done, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&h[1], j->dev + j->o_err, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *done_chains = h[0];
  *err = h[1];
  return FSMC_OK;
}

// Captures `rounds` FSM rounds on `st` into an executable graph (views are fixed for the
// life of the job, so the graph stays valid across runs and resets).
template <typename T>
static fsmc_status capture_rounds(fsmc_job* j, int rounds, cudaStream_t st) {
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  const int64_t launches0 = j->launches;
  for (int b = 0; b < rounds && e == cudaSuccess; ++b) e = fsm_round<T>(j, st);
  j->launches = launches0;
  cudaError_t e2 = cudaStreamEndCapture(st, &g);
  if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return fsmc_cuda_fail(e, "FSM launch (capture)"); }
  if (e2 != cudaSuccess) return fsmc_cuda_fail(e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&j->graph_exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { j->graph_exec = nullptr; return fsmc_cuda_fail(e, "cudaGraphInstantiate"); }
  j->graph_rounds = rounds;
  return FSMC_OK;
}

// Whole ESS run with the direction refill of round r+1 on a second stream, overlapping the FSM
// kernel of round r.  Refill windows alternate between two buffers: buffer p holds the window
// the FSM kernel of a round-p round consumes (it reads only its upper bound), buffer p^1 the
// one being refilled.  The refill stream waits for the FSM kernel of round r-1 before writing
// buffer p^1, so it runs at most one round ahead.
// With the tensor-core generator the refill's small kernels (next window, prefix sum, column
// list) run on a third stream of the highest priority, after the generator of round r (the
// column list's previous reader) and the FSM kernel of round r-1: their blocks then take the
// first SM slots that FSM blocks of round r free, and only the generator kernel is left
// between round r's last FSM blocks and round r+1.
template <typename T>
static fsmc_status run_fsm_pipelined(fsmc_job* j, cudaStream_t st) {
  if (!j->side) {
    CK(cudaStreamCreateWithFlags(&j->side, cudaStreamNonBlocking));
    for (int p = 0; p < 2; ++p) {
      CK(cudaEventCreateWithFlags(&j->ev_gen[p], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&j->ev_fsm[p], cudaEventDisableTiming));
    }
  }
  const bool split = sizeof(T) == 4 && j->tun.generator == 2;
  if (split && !j->side_hi) {
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CK(cudaStreamCreateWithPriority(&j->side_hi, cudaStreamNonBlocking, greatest));
    CK(cudaEventCreateWithFlags(&j->ev_cols, cudaEventDisableTiming));
  }
  cudaStream_t sb = j->side;
  EssView<T> v[2];
  v[0] = ess_view<T>(j);  // buffer 0: the job's own window arrays
  v[1] = v[0];
  v[1].gen_lo = (int*)(j->dev + j->o_win);
  v[1].gen_hi = v[1].gen_lo + j->m;
  v[0].own_window = v[1].own_window = 0;
  const fsmc_tuning& tu = j->tun;
  // buffer 0 already holds the next window (set at init or by the last round of a previous run)
  CK(cudaEventRecord(j->ev_fsm[1], st));  // the caller's prior work on st
  CK(cudaStreamWaitEvent(sb, j->ev_fsm[1], 0));
  {
    ProfScope p(j, 0, sb);
    CK(ess_generate<T>(j, v[0], sb));
  }
  j->launches += ess_generate_kernels(j);
  CK(cudaEventRecord(j->ev_gen[0], sb));
  int p = 0;
  int64_t r = 0;
  while (true) {
    CK(cudaStreamWaitEvent(st, j->ev_gen[p], 0));
    {
      ProfScope ps(j, 1, st);
      CK(launch_ess_fsm<T>(v[p], tu.lanes_per_chain, tu.steps_per_launch, tu.threads_per_block, st));
    }
    CK(cudaEventRecord(j->ev_fsm[p], st));
    if (split) {
      if constexpr (sizeof(T) == 4) {
        cudaStream_t sh = j->side_hi;
        if (r >= 1) CK(cudaStreamWaitEvent(sh, j->ev_fsm[p ^ 1], 0));
        CK(cudaStreamWaitEvent(sh, j->ev_gen[p], 0));
        CK(launch_ess_window<T>(v[p ^ 1], v[p].gen_hi, sh));
        CK(launch_ess_tc_cols(v[p ^ 1], sh));
        CK(cudaEventRecord(j->ev_cols, sh));
        CK(cudaStreamWaitEvent(sb, j->ev_cols, 0));
        {
          ProfScope ps(j, 0, sb);
          CK(launch_ess_tc_gen(v[p ^ 1], j->tg->tc_img, j->e->sms, sb));
        }
      }
    } else {
      if (r >= 1) CK(cudaStreamWaitEvent(sb, j->ev_fsm[p ^ 1], 0));
      CK(launch_ess_window<T>(v[p ^ 1], v[p].gen_hi, sb));
      {
        ProfScope ps(j, 0, sb);
        CK(ess_generate<T>(j, v[p ^ 1], sb));
      }
    }
    CK(cudaEventRecord(j->ev_gen[p ^ 1], sb));
    j->launches += 2 + ess_generate_kernels(j);  // FSM step, window, refill
    ++r;
    p ^= 1;
    if (r % 8 == 0) {
      int done = 0, err = 0;
      fsmc_status s = read_done(j, st, &done, &err);
      if (s != FSMC_OK) return s;
      if (done >= j->m) break;
    }
  }
  // the last refill may still run on the side stream: join it, and leave the job's own
  // window arrays consistent for a later partial run
  CK(cudaStreamWaitEvent(st, j->ev_gen[p], 0));
  if (p == 1) {
    CK(cudaMemcpyAsync(v[0].gen_lo, v[1].gen_lo, j->m * sizeof(int), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(v[0].gen_hi, v[1].gen_hi, j->m * sizeof(int), cudaMemcpyDeviceToDevice, st));
  }
  return FSMC_OK;
}

template <typename T>
static fsmc_status run_fsm(fsmc_job* j, int64_t max_steps, cudaStream_t st) {
  if (j->algo == FSMC_ESS && !ess_block(j) && max_steps <= 0 && j->tun.pipelined == 1)
    return run_fsm_pipelined<T>(j, st);
  const int check_every = 8;
  int64_t rounds_limit = -1;
  if (max_steps > 0) rounds_limit = (max_steps + j->tun.steps_per_launch - 1) / j->tun.steps_per_launch;
  // whole runs on a real stream replay a captured burst; profiled or partial runs launch directly
  const bool graph = rounds_limit < 0 && !j->tun.profile_kernels && st != nullptr;
  if (graph && !j->graph_exec) {
    fsmc_status s = capture_rounds<T>(j, check_every, st);
    if (s != FSMC_OK) return s;
  }
  const int per_round = j->algo == FSMC_ESS && !ess_block(j) ? ess_generate_kernels(j) + 1 : 1;
  int64_t r = 0;
  while (true) {
    int done = 0, err = 0;
    fsmc_status s = read_done(j, st, &done, &err);
    if (s != FSMC_OK) return s;
    if (err & ERR_BARRIER_TIMEOUT) return fsmc_fail(FSMC_ETIMEOUT, "device barrier timed out");
    if (done >= j->m) break;
    if (rounds_limit >= 0 && r >= rounds_limit) break;
    int burst = check_every;
    if (rounds_limit >= 0) burst = (int)std::min<int64_t>(burst, rounds_limit - r);
    if (graph) {
      CK(cudaGraphLaunch(j->graph_exec, st));
      j->launches += (int64_t)per_round * j->graph_rounds;
      burst = j->graph_rounds;
    } else {
      for (int b = 0; b < burst; ++b) {
        cudaError_t e = fsm_round<T>(j, st);
        if (e != cudaSuccess) return fsmc_cuda_fail(e, "FSM launch");
      }
    }
    r += burst;
  }
  return FSMC_OK;
}

template <typename T>
static fsmc_status run_sync(fsmc_job* j, cudaStream_t st) {
  char* b = j->dev;
  GridBarrier bar = job_grid_barrier(j);
  unsigned* active = (unsigned*)(b + j->o_bar) + 4;
  unsigned long long* iters = (unsigned long long*)(b + j->o_iters);
  const int threads = j->tun.threads_per_block;
  if (ess_block(j)) {
    EssBlockView<T> v = ess_block_view<T>(j);
    const int chunk = 1000;
    for (int64_t t0 = 0; t0 < j->n; t0 += chunk) {
      const int t1 = (int)std::min<int64_t>(t0 + chunk, j->n);
      CK(clear_sync_counters(j, st));
      ProfScope p(j, 2, st);
      CK(launch_ess_block_sync<T>(v, (int)t0, t1, bar, active, iters, st));
      j->launches += 1;
    }
  } else if (j->algo == FSMC_ESS) {
    EssView<T> v = ess_view<T>(j);
    unsigned long long it0 = 0;
    if (j->tun.sync_form == 3) CK(cudaMemcpyAsync(&it0, iters, 8, cudaMemcpyDeviceToHost, st));
    for (int64_t t0 = 0; t0 < j->n; t0 += j->W) {
      const int t1 = (int)std::min<int64_t>(t0 + j->W, j->n);
      {
        ProfScope p(j, 3, st);
        CK(launch_fill_int(v.gen_lo, j->m, (int)t0, st));
        CK(launch_fill_int(v.gen_hi, j->m, t1, st));
      }
      {
        ProfScope p(j, 0, st);
        CK(ess_generate<T>(j, v, st));
      }
      int* lists = (int*)(b + j->o_slist);
      void* cg = b + j->o_slist + 2 * (size_t)j->m * 4;
      if (j->tun.sync_form == 3) {
        if (!j->sync_graph)
          CK(build_ess_sync_graph<T>(v, j->tun.lanes_per_chain, threads, cg, lists, iters, &j->sync_graph));
        ProfScope p(j, 2, st);
        CK(launch_ess_sync_graph(j->sync_graph, cg, (int)t0, t1, st));
        j->launches += 3 + ess_generate_kernels(j);  // two window fills, the refill, the loop-state reset
      } else {
        CK(clear_sync_counters(j, st));
        ProfScope p(j, 2, st);
        CK(launch_ess_sync<T>(v, j->tun.lanes_per_chain, (int)t0, t1, bar, active, iters, threads,
                              j->tun.sync_form, lists, st));
        j->launches += 3 + ess_generate_kernels(j);  // two window fills, the refill, the sync kernel
      }
    }
    if (j->tun.sync_form == 3) {  // the graph's launches: init and next per sample, one per iteration
      unsigned long long it1 = 0;
      CK(cudaMemcpyAsync(&it1, iters, 8, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      j->launches += 2 * j->n + (int64_t)(it1 - it0);
    }
  } else if (j->algo == FSMC_DR) {
    DrView<T> v = dr_view<T>(j);
    const int chunk = 1000;
    for (int64_t t0 = 0; t0 < j->n; t0 += chunk) {
      const int t1 = (int)std::min<int64_t>(t0 + chunk, j->n);
      CK(clear_sync_counters(j, st));
      ProfScope p(j, 2, st);
      CK(launch_dr_sync<T>(v, (int)t0, t1, bar, active, iters, threads, st));
      j->launches += 1;
    }
  } else if (j->algo == FSMC_SLICE) {
    SliceView<T> v = slice_view<T>(j);
    const int chunk = 1000;
    for (int64_t t0 = 0; t0 < j->n; t0 += chunk) {
      const int t1 = (int)std::min<int64_t>(t0 + chunk, j->n);
      CK(clear_sync_counters(j, st));
      ProfScope p(j, 2, st);
      CK(launch_slice_sync<T>(v, (int)t0, t1, bar, active, iters, threads, st));
      j->launches += 1;
    }
  } else {
    fsmc_status s = nuts_run_sync(j, st);
    if (s != FSMC_OK) return s;
  }
  int done = 0, err = 0;
  fsmc_status s = read_done(j, st, &done, &err);
  if (s != FSMC_OK) return s;
  if (err & ERR_BARRIER_TIMEOUT) return fsmc_fail(FSMC_ETIMEOUT, "device barrier timed out");
  return FSMC_OK;
}

fsmc_status job_run_impl(fsmc_job* j, fsmc_mode mode, int64_t max_fsm_steps, cudaStream_t st) {
  fsmc_status s = job_materialize(j, st);
  if (s != FSMC_OK) return s;
  CK(cudaSetDevice(j->e->device));
  if (mode == FSMC_MODE_SYNC && (j->fsm_used || j->sync_used))
    return fsmc_fail(FSMC_ESTATE, "SYNC mode needs a fresh or reset job");
  if (mode == FSMC_MODE_FSM && j->sync_used)
    return fsmc_fail(FSMC_ESTATE, "job was run in SYNC mode; reset it first");
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  j->launches = 0;
  prof_reset(j);
  unsigned long long cols0 = 0;
  if (j->algo == FSMC_ESS) CK(cudaMemcpy(&cols0, j->dev + j->o_gencols, 8, cudaMemcpyDeviceToHost));
  CK(cudaEventRecord(e0, st));
  if (mode == FSMC_MODE_FSM) {
    j->fsm_used = true;
    s = j->prec == FSMC_FP64 ? run_fsm<double>(j, max_fsm_steps, st) : run_fsm<float>(j, max_fsm_steps, st);
  } else if (mode == FSMC_MODE_SYNC) {
    j->sync_used = true;
    s = j->prec == FSMC_FP64 ? run_sync<double>(j, st) : run_sync<float>(j, st);
  } else {
    s = fsmc_fail(FSMC_EINVAL, "bad mode");
  }
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  j->device_ms = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  prof_collect(j);
  if (j->algo == FSMC_ESS) {
    unsigned long long cols1 = 0;
    cudaMemcpy(&cols1, j->dev + j->o_gencols, 8, cudaMemcpyDeviceToHost);
    j->columns_generated = (int64_t)(cols1 - cols0);
  }
  if (s != FSMC_OK) return s;
  int h_err = 0;
  CK(cudaMemcpy(&h_err, j->dev + j->o_err, 4, cudaMemcpyDeviceToHost));
  if (h_err & ERR_SHRINK_CAP) return fsmc_fail(FSMC_EDEVICE, "ESS shrink cap reached (error word 1)");
  return FSMC_OK;
}

extern "C" fsmc_status fsmc_job_run(fsmc_job* j, fsmc_mode mode, int64_t max_fsm_steps, void* stream) {
  if (!j) return fsmc_fail(FSMC_EINVAL, "job is NULL");
  if (j->submitted) return fsmc_fail(FSMC_ESTATE, "job is owned by the serving scheduler");
  return job_run_impl(j, mode, max_fsm_steps, (cudaStream_t)stream);
}

extern "C" fsmc_status fsmc_job_reset(fsmc_job* j) {
  if (!j) return fsmc_fail(FSMC_EINVAL, "job is NULL");
  if (j->submitted) return fsmc_fail(FSMC_ESTATE, "job is owned by the serving scheduler");
  if (!j->dev) return FSMC_OK;
  return job_init(j, 0);
}

extern "C" fsmc_status fsmc_job_progress(fsmc_job* j, int64_t* min_samples, int* done) {
  if (!j) return fsmc_fail(FSMC_EINVAL, "job is NULL");
  if (!j->dev) {
    if (min_samples) *min_samples = 0;
    if (done) *done = 0;
    return FSMC_OK;
  }
  std::vector<int> t((size_t)j->m);
  CK(cudaMemcpy(t.data(), j->dev + j->o_t, t.size() * 4, cudaMemcpyDeviceToHost));
  int mn = *std::min_element(t.begin(), t.end());
  if (min_samples) *min_samples = mn;
  if (done) *done = mn >= j->n;
  return FSMC_OK;
}

// ---- reads ------------------------------------------------------------------------------------------
template <typename T>
static fsmc_status read_samples_t(fsmc_job* j, int64_t c0, int64_t nc, int64_t s0, int64_t ns, double* dst) {
  const size_t d = (size_t)j->d;
  std::vector<T> row((size_t)ns * d);
  for (int64_t c = 0; c < nc; ++c) {
    const char* src = j->dev + j->o_out + (((size_t)(c0 + c) * j->n + s0) * d) * sizeof(T);
    CK(cudaMemcpy(row.data(), src, row.size() * sizeof(T), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < row.size(); ++i) dst[(size_t)c * ns * d + i] = (double)row[i];
  }
  return FSMC_OK;
}

static fsmc_status check_range(fsmc_job* j, int64_t c0, int64_t nc, int64_t s0, int64_t ns) {
  if (!j->dev) return fsmc_fail(FSMC_ESTATE, "job has not run");
  if (!j->store) return fsmc_fail(FSMC_ESTATE, "job keeps moments only");
  if (c0 < 0 || nc < 0 || c0 + nc > j->m || s0 < 0 || ns < 0 || s0 + ns > j->n)
    return fsmc_fail(FSMC_EINVAL, "range outside [0, m) x [0, n)");
  return FSMC_OK;
}

extern "C" fsmc_status fsmc_read_samples(fsmc_job* j, int64_t c0, int64_t nc, int64_t s0, int64_t ns,
                                         double* dst) {
  if (!j || (!dst && nc * ns > 0)) return fsmc_fail(FSMC_EINVAL, "NULL argument");
  fsmc_status s = check_range(j, c0, nc, s0, ns);
  if (s != FSMC_OK) return s;
  CK(cudaSetDevice(j->e->device));
  return j->prec == FSMC_FP64 ? read_samples_t<double>(j, c0, nc, s0, ns, dst)
                              : read_samples_t<float>(j, c0, nc, s0, ns, dst);
}

extern "C" fsmc_status fsmc_read_samples_dev(fsmc_job* j, int64_t c0, int64_t nc, int64_t s0, int64_t ns,
                                             void* dst, void* stream) {
  if (!j || (!dst && nc * ns > 0)) return fsmc_fail(FSMC_EINVAL, "NULL argument");
  fsmc_status s = check_range(j, c0, nc, s0, ns);
  if (s != FSMC_OK) return s;
  const size_t es = j->prec == FSMC_FP64 ? 8 : 4;
  const size_t d = (size_t)j->d;
  const char* src = j->dev + j->o_out + (((size_t)c0 * j->n + s0) * d) * es;
  CK(cudaMemcpy2DAsync(dst, (size_t)ns * d * es, src, (size_t)j->n * d * es, (size_t)ns * d * es,
                       (size_t)nc, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return FSMC_OK;
}

extern "C" fsmc_status fsmc_read_loop_counts(fsmc_job* j, int32_t* counts, int32_t* aux, int64_t* steps) {
  if (!j) return fsmc_fail(FSMC_EINVAL, "job is NULL");
  if (!j->dev) return fsmc_fail(FSMC_ESTATE, "job has not run");
  if (counts)
    CK(cudaMemcpy(counts, j->dev + j->o_counts, (size_t)j->m * j->n * 4, cudaMemcpyDeviceToHost));
  if (aux) {
    if (j->algo == FSMC_NUTS || j->algo == FSMC_SLICE)
      CK(cudaMemcpy(aux, j->dev + j->o_aux, (size_t)j->m * j->n * 4, cudaMemcpyDeviceToHost));
    else
      std::fill(aux, aux + (size_t)j->m * j->n, 0);
  }
  if (steps) CK(cudaMemcpy(steps, j->dev + j->o_steps, (size_t)j->m * 8, cudaMemcpyDeviceToHost));
  return FSMC_OK;
}

template <typename T>
static fsmc_status read_vec(const char* src, size_t n, double* dst) {
  std::vector<T> h(n);
  CK(cudaMemcpy(h.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < n; ++i) dst[i] = (double)h[i];
  return FSMC_OK;
}

extern "C" fsmc_status fsmc_read_state(fsmc_job* j, double* x) {
  if (!j || !x) return fsmc_fail(FSMC_EINVAL, "NULL argument");
  if (!j->dev) {
    CK(cudaMemcpy(x, j->x0_dev, (size_t)j->m * j->d * sizeof(double), cudaMemcpyDeviceToHost));
    return FSMC_OK;
  }
  const size_t n = (size_t)j->m * j->d;
  return j->prec == FSMC_FP64 ? read_vec<double>(j->dev + j->o_x, n, x) : read_vec<float>(j->dev + j->o_x, n, x);
}

extern "C" fsmc_status fsmc_read_moments(fsmc_job* j, double* sx, double* sx2, int64_t* n_kept) {
  if (!j) return fsmc_fail(FSMC_EINVAL, "job is NULL");
  if (!j->dev) return fsmc_fail(FSMC_ESTATE, "job has not run");
  const size_t md = (size_t)j->m * j->d;
  std::vector<int> t((size_t)j->m);
  CK(cudaMemcpy(t.data(), j->dev + j->o_t, t.size() * 4, cudaMemcpyDeviceToHost));
  if (n_kept) for (size_t c = 0; c < t.size(); ++c) n_kept[c] = t[c];
  char* m0 = j->dev + j->o_mom;
  if (j->store) {  // reduce the stored samples on the device into the [4][m][d] buffer
    cudaError_t ce = j->prec == FSMC_FP64
        ? launch_moments_from_samples<double>((const double*)(j->dev + j->o_out), (const int*)(j->dev + j->o_t),
                                              j->m, (int)j->n, j->d, (double*)m0, 0)
        : launch_moments_from_samples<float>((const float*)(j->dev + j->o_out), (const int*)(j->dev + j->o_t),
                                             j->m, (int)j->n, j->d, (float*)m0, 0);
    if (ce != cudaSuccess) return fsmc_cuda_fail(ce, "moments kernel");
  }
  // converted to double on the device, then copied straight into the caller's buffers (fast
  // when they are pinned)
  double* md2 = (double*)(j->dev + j->o_momd);
  CK(j->prec == FSMC_FP64 ? launch_moments_to_double<double>((const double*)m0, (int64_t)md, md2, 0)
                          : launch_moments_to_double<float>((const float*)m0, (int64_t)md, md2, 0));
  if (sx) CK(cudaMemcpy(sx, md2, md * 8, cudaMemcpyDeviceToHost));
  if (sx2) CK(cudaMemcpy(sx2, md2 + md, md * 8, cudaMemcpyDeviceToHost));
  return FSMC_OK;
}

extern "C" fsmc_status fsmc_read_stats(fsmc_job* j, fsmc_stats* o) {
  if (!j || !o) return fsmc_fail(FSMC_EINVAL, "NULL argument");
  *o = fsmc_stats{};
  o->R_hat = 1.0;
  if (!j->dev) return FSMC_OK;
  CK(cudaSetDevice(j->e->device));
  // reduced on the device (stats.cu); the host copies one record back
  unsigned* colmax = (unsigned*)(j->dev + j->o_stats);
  fsmc::DevStats* rec = (fsmc::DevStats*)(j->dev + j->o_stats + align_up((size_t)j->n * 4, 64));
  CK(fsmc::launch_job_stats((const int*)(j->dev + j->o_counts), (const int*)(j->dev + j->o_t),
                            (const long long*)(j->dev + j->o_steps), j->m, (int)j->n,
                            (const unsigned long long*)(j->dev + j->o_iters), (const int*)(j->dev + j->o_err),
                            colmax, rec, 0));
  fsmc::DevStats h{};
  CK(cudaMemcpy(&h, rec, sizeof h, cudaMemcpyDeviceToHost));
  const long long tmin = h.tmin;
  if (tmin > 0) {
    o->mean_N = (double)h.sum_all / ((double)tmin * (double)j->m);
    o->mean_max_N = (double)h.sum_max / (double)tmin;
    o->R_hat = h.sum_all > 0 ? o->mean_max_N / o->mean_N : 1.0;
  }
  o->samples_done = h.samples_done;
  o->fsm_steps = h.fsm_steps;
  o->sync_iterations = h.iters;
  o->launches = j->launches;
  o->device_ms = j->device_ms;
  o->error_word = h.err;
  for (int k = 0; k < 4; ++k) { o->kernel_ms[k] = j->kernel_ms[k]; o->kernel_launches[k] = j->kernel_launches[k]; }
  o->columns_generated = j->columns_generated;
  return FSMC_OK;
}

// ---- fused multi-job rounds (serving) -------------------------------------------------------------------
fsmc_status multibuf_ensure(MultiBuf& b, size_t bytes) {
  if (b.cap >= bytes) return FSMC_OK;
  multibuf_free(b);
  size_t cap = 4096;
  while (cap < bytes) cap *= 2;
  CK(cudaMalloc(&b.d_buf, cap));
  CK(cudaMallocHost(&b.h_stage, cap));
  b.cap = cap;
  return FSMC_OK;
}

void multibuf_free(MultiBuf& b) {
  if (b.d_buf) cudaFree(b.d_buf);
  if (b.h_stage) cudaFreeHost(b.h_stage);
  b = MultiBuf{};
}

int ess_job_group(const fsmc_job* j) { return j->tun.lanes_per_chain * 64 + ess_group_E(j->tun.lanes_per_chain, j->d); }

template <typename T>
static cudaError_t ess_generate(fsmc_job* j, const EssView<T>& v, cudaStream_t st);

template <typename T>
static cudaError_t ess_group_round_t(const std::vector<fsmc_job*>& jobs, MultiBuf& b, cudaStream_t st) {
  const int nj = (int)jobs.size();
  const size_t vb = sizeof(EssView<T>);
  const size_t views_bytes = (nj * vb + 15) / 16 * 16;
  char* hs = (char*)b.h_stage;
  int64_t* tile_off = (int64_t*)(hs + views_bytes);
  int64_t* chain_off = tile_off + (nj + 1);
  tile_off[0] = chain_off[0] = 0;
  for (int k = 0; k < nj; ++k) {
    fsmc_job* j = jobs[k];
    const EssView<T> v = ess_view<T>(j);
    std::memcpy(hs + k * vb, &v, vb);
    // jobs on the tensor-core generator refill their rings with it (identical directions to a
    // job run alone); the others share one fused CUDA-core generator launch
    const bool own = j->tun.generator == 2;
    if (own) {
      cudaError_t e = ess_generate<T>(j, v, st);
      if (e != cudaSuccess) return e;
    }
    tile_off[k + 1] = tile_off[k] + (own ? 0 : ((j->m + 63) / 64) * j->W * ((j->d + 255) / 256));
    chain_off[k + 1] = chain_off[k] + j->m;
  }
  const size_t bytes = views_bytes + 2 * (nj + 1) * sizeof(int64_t);
  cudaError_t e = cudaMemcpyAsync(b.d_buf, hs, bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  const EssView<T>* dv = (const EssView<T>*)b.d_buf;
  const int64_t* d_tile = (const int64_t*)((char*)b.d_buf + views_bytes);
  const int64_t* d_chain = d_tile + (nj + 1);
  e = launch_ess_nu_gen_multi<T>(dv, d_tile, nj, tile_off[nj], st);
  if (e != cudaSuccess) return e;
  const fsmc_tuning& tu = jobs[0]->tun;
  return launch_ess_fsm_multi<T>(ess_view<T>(jobs[0]), tu.lanes_per_chain, dv, d_chain, nj, chain_off[nj],
                                 tu.steps_per_launch, tu.threads_per_block, st);
}

cudaError_t ess_group_round(const std::vector<fsmc_job*>& jobs, MultiBuf& b, cudaStream_t st) {
  if (jobs.empty()) return cudaSuccess;
  return jobs[0]->prec == FSMC_FP64 ? ess_group_round_t<double>(jobs, b, st) : ess_group_round_t<float>(jobs, b, st);
}

// ---- checkpoint ---------------------------------------------------------------------------------------
struct SnapHeader {
  uint64_t magic, bytes, m, n, d, algo, prec, flags;
};
static const uint64_t kSnapMagic = 0x46534d43534e4150ull;  // "FSMCSNAP"

extern "C" fsmc_status fsmc_job_snapshot(fsmc_job* j, void* buf, size_t* bytes) {
  if (!j || !bytes) return fsmc_fail(FSMC_EINVAL, "NULL argument");
  if (!j->dev) return fsmc_fail(FSMC_ESTATE, "job has not run");
  const size_t need = sizeof(SnapHeader) + j->bytes;
  if (!buf) { *bytes = need; return FSMC_OK; }
  if (*bytes < need) return fsmc_fail(FSMC_EINVAL, "snapshot buffer too small");
  SnapHeader h{kSnapMagic, j->bytes, (uint64_t)j->m, (uint64_t)j->n, (uint64_t)j->d, (uint64_t)j->algo,
               (uint64_t)j->prec, (uint64_t)((j->fsm_used ? 1 : 0) | (j->sync_used ? 2 : 0))};
  std::memcpy(buf, &h, sizeof h);
  CK(cudaMemcpy((char*)buf + sizeof h, j->dev, j->bytes, cudaMemcpyDeviceToHost));
  *bytes = need;
  return FSMC_OK;
}

extern "C" fsmc_status fsmc_job_restore(fsmc_job* j, const void* buf, size_t bytes) {
  if (!j || !buf) return fsmc_fail(FSMC_EINVAL, "NULL argument");
  fsmc_status s = job_materialize(j, 0);
  if (s != FSMC_OK) return s;
  SnapHeader h;
  if (bytes < sizeof h) return fsmc_fail(FSMC_EINVAL, "snapshot too small");
  std::memcpy(&h, buf, sizeof h);
  if (h.magic != kSnapMagic || h.bytes != j->bytes || h.m != (uint64_t)j->m || h.n != (uint64_t)j->n ||
      h.d != (uint64_t)j->d || h.algo != (uint64_t)j->algo || h.prec != (uint64_t)j->prec ||
      bytes < sizeof h + h.bytes)
    return fsmc_fail(FSMC_EINVAL, "snapshot does not match this job");
  CK(cudaMemcpy(j->dev, (const char*)buf + sizeof h, j->bytes, cudaMemcpyHostToDevice));
  j->fsm_used = h.flags & 1;
  j->sync_used = h.flags & 2;
  return FSMC_OK;
}

extern "C" void fsmc_job_destroy(fsmc_job* j) {
  if (!j) return;
  serving_forget(j);
  fsmc_engine* e = j->e;
  for (cudaEvent_t ev : j->event_pool) cudaEventDestroy(ev);
  if (j->graph_exec) cudaGraphExecDestroy(j->graph_exec);
  if (j->sync_graph) cudaGraphExecDestroy(j->sync_graph);
  for (int p = 0; p < 2; ++p) {
    if (j->ev_gen[p]) cudaEventDestroy(j->ev_gen[p]);
    if (j->ev_fsm[p]) cudaEventDestroy(j->ev_fsm[p]);
  }
  if (j->side) cudaStreamDestroy(j->side);
  if (j->ev_cols) cudaEventDestroy(j->ev_cols);
  if (j->side_hi) cudaStreamDestroy(j->side_hi);
  if (j->dev) {
    cudaSetDevice(e->device);
    // a job run through fsmc_job_run has no work in flight; one the scheduler ran is freed
    // (cudaFree waits for the device)
    if (j->submitted) cudaFree(j->dev);
    else arena_give(e, j->dev, j->arena_bytes);
    engine_release(e, j->bytes);
  }
  if (j->x0_dev) {
    cudaSetDevice(e->device);
    if (j->submitted) cudaFree(j->x0_dev);
    else arena_give(e, j->x0_dev, j->x0_block);
  }
  {
    std::lock_guard<std::mutex> g(e->mu);
    e->jobs.erase(std::remove(e->jobs.begin(), e->jobs.end(), j), e->jobs.end());
  }
  delete j;
}
