// Host-side object layouts shared by the engine, the NUTS launcher and the serving scheduler.
#pragma once
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fsmc.h"
#include "fsmc_device.cuh"

struct fsmc_engine {
  int device = 0;
  int sms = 148;
  size_t budget = 0;
  size_t in_use = 0;
  mutable std::mutex mu;
  std::vector<fsmc_job*> jobs;        // materialised jobs (hold device memory)
  std::vector<std::pair<char*, size_t>> spare;  // device blocks of destroyed jobs, kept for reuse
  std::vector<fsmc_target*> targets;
  // serving scheduler
  std::thread sched;
  std::condition_variable cv;
  std::deque<fsmc_job*> queue;        // submitted, not yet admitted
  std::vector<fsmc_job*> active;      // admitted, running
  bool stop = false;
  bool sched_running = false;
  int64_t pending = 0;                // submitted and not finished
  cudaStream_t sched_stream = nullptr;
  std::string sched_error;
};

struct fsmc_target {
  fsmc_engine* e = nullptr;
  int kind = 0, d = 0, n_data = 0;
  std::vector<double> params;
  std::vector<void*> bufs;
  size_t bytes = 0;
  fsmc::TargetView<float> tv32{};
  fsmc::TargetView<double> tv64{};
  unsigned char* tc_img = nullptr;  // FP16 hi/lo image of L for the tensor-core generator
};

struct fsmc_job {
  fsmc_engine* e = nullptr;
  fsmc_target* tg = nullptr;
  fsmc_algo algo = FSMC_ESS;
  fsmc_precision prec = FSMC_FP32;
  int64_t m = 0, n = 0;
  int d = 0;
  uint64_t seed = 0;
  uint32_t chain0 = 0;
  int store = 1;
  fsmc_tuning tun{};
  fsmc_dr_params dr{3, 1.0, 0.5, 0};
  fsmc_nuts_params nuts{0.05, 10, 1000.0};
  fsmc_slice_params slice{1.0, 100};
  char* x0_dev = nullptr;  // [n_chains][d] starting points (double), copied in at creation
  size_t x0_block = 0;     // size of the device block behind x0_dev
  // device arena and offsets into it
  char* dev = nullptr;
  size_t bytes = 0;
  int W = 0, dstride = 0;
  size_t o_x = 0, o_t = 0, o_counts = 0, o_steps = 0, o_err = 0, o_done = 0, o_out = 0, o_mom = 0,
         o_bar = 0, o_iters = 0;
  size_t o_ell = 0, o_logy = 0, o_th = 0, o_k = 0, o_s = 0, o_gen = 0, o_nu = 0,  // ESS (o_ell/o_k: DR too)
         o_gencols = 0;
  size_t o_y = 0, o_lpy = 0;                                                      // DR
  size_t o_aux = 0, o_nuts = 0, o_nuts_end = 0;                                   // NUTS (o_aux: SLICE too)
  // run bookkeeping
  bool fsm_used = false, sync_used = false;
  int64_t launches = 0;
  double device_ms = 0;
  // per-kernel-class timing (tuning.profile_kernels)
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_events;
  std::vector<cudaEvent_t> event_pool;
  size_t event_next = 0;
  double kernel_ms[4] = {0, 0, 0, 0};
  int64_t kernel_launches[4] = {0, 0, 0, 0};
  int64_t columns_generated = 0;
  // captured burst of FSM rounds (replayed by run_fsm when kernel profiling is off)
  cudaGraphExec_t graph_exec = nullptr;
  int graph_rounds = 0;
  // pipelined ESS rounds: second stream and the events ordering the two
  cudaStream_t side = nullptr;
  cudaEvent_t ev_gen[2] = {nullptr, nullptr}, ev_fsm[2] = {nullptr, nullptr};
  cudaStream_t side_hi = nullptr;  // high-priority stream of the refills' column lists
  cudaEvent_t ev_cols = nullptr;
  size_t o_win = 0;  // second refill-window buffer [2][m]
  size_t o_colbase = 0, o_colmap = 0;  // compacted refill list: [m+1] prefix sums, [m*W] (chain, sample)
  size_t o_work = 0;  // block-likelihood ESS: chain counter of the current FSM launch
  size_t o_spill = 0, spill_stride = 0;  // block-likelihood ESS: per-CTA scratch for rows
  int64_t spill_ctas = 0;                // beyond shared memory
  int rows_smem = 0;                     // covariance rows kept in shared memory
  size_t o_momd = 0;  // [2][m][d] doubles: the moment sums for the host read
  size_t o_gbar = 0;   // grid barrier of synchronised launches (fsmc::kGridBarrierBytes)
  size_t o_stats = 0;  // device statistics: [n] column maxima, then the DevStats record
  size_t o_slist = 0;  // ESS synchronised list and graph forms: [2][m] chain lists, graph loop state
  cudaGraphExec_t sync_graph = nullptr;  // ESS synchronised graph form (built at the first SYNC run)
  size_t arena_bytes = 0;  // size of the device block behind dev (>= bytes when reused)
  // serving
  bool submitted = false;
  fsmc_mode serve_mode = FSMC_MODE_FSM;
  std::atomic<int> finished{0};
  std::atomic<int> cancel{0};
  fsmc_status serve_status = FSMC_OK;
  std::chrono::steady_clock::time_point t_submit, t_done;
};

// The job's grid barrier for synchronised launches, with the tuning's wait limit and test hook.
// Its counters (o_gbar) and the loop's active-chain counters (o_bar, at 16..27) are zeroed before
// every synchronised launch (clear_sync_counters).
inline fsmc::GridBarrier job_grid_barrier(const fsmc_job* j) {
  fsmc::GridBarrier bar{(unsigned*)(j->dev + j->o_gbar)};
  if (j->tun.barrier_spin_limit > 0) bar.spin_limit = (unsigned)j->tun.barrier_spin_limit;
  bar.missing = (unsigned)j->tun.barrier_test_missing;
  return bar;
}

inline cudaError_t clear_sync_counters(const fsmc_job* j, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(j->dev + j->o_bar, 0, 64, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(j->dev + j->o_gbar, 0, fsmc::kGridBarrierBytes, st);
  return e;
}

fsmc_status fsmc_fail(fsmc_status st, const std::string& msg);
fsmc_status fsmc_cuda_fail(cudaError_t e, const char* what);
bool engine_reserve(fsmc_engine* e, size_t bytes);
void engine_release(fsmc_engine* e, size_t bytes);
fsmc_status job_materialize(fsmc_job* j, cudaStream_t st);
fsmc_status job_run_impl(fsmc_job* j, fsmc_mode mode, int64_t max_fsm_steps, cudaStream_t st);
// Brackets one launch of kernel class `cls` with events when profiling is on.
struct ProfScope {
  fsmc_job* j;
  int cls;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(fsmc_job* job, int c, cudaStream_t s);
  ~ProfScope();
};

// Device table of job views for a fused multi-job launch, with its pinned host staging.
struct MultiBuf {
  void* d_buf = nullptr;
  void* h_stage = nullptr;
  size_t cap = 0;
};
fsmc_status multibuf_ensure(MultiBuf& b, size_t bytes);
void multibuf_free(MultiBuf& b);
// Group keys and fused rounds (one direction refill + one FSM launch for ESS groups).
int ess_job_group(const fsmc_job* j);   // (lanes, E) code of an ESS job
int nuts_group_E(int d);
cudaError_t ess_group_round(const std::vector<fsmc_job*>& jobs, MultiBuf& b, cudaStream_t st);
cudaError_t nuts_group_round(const std::vector<fsmc_job*>& jobs, MultiBuf& b, cudaStream_t st);

// NUTS (nuts.cu)
void nuts_layout(fsmc_job* j, size_t& off);
fsmc_status nuts_init_state(fsmc_job* j, cudaStream_t st);
cudaError_t nuts_fsm_round(fsmc_job* j, cudaStream_t st);
fsmc_status nuts_run_sync(fsmc_job* j, cudaStream_t st);

// serving (serving.cu)
void serving_shutdown(fsmc_engine* e);
void serving_forget(fsmc_job* j);
