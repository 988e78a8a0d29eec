// Serving scheduler: continuous batching of sampling jobs on one GPU.
//
// fsmc_submit queues a job; a scheduler thread admits queued jobs in arrival order as
// soon as their device footprint fits the engine's HBM budget (device memory is
// allocated at admission, not at submission), then runs rounds.  A job that does not fit
// yet does not hold back the smaller jobs behind it, unless it has waited longer than
// kAgingSeconds: then nothing behind it is admitted until it fits (no starvation).  In a
// round every admitted FSM job advances by one fused launch per group of jobs that share a kernel shape
// (sampler, precision, lanes per chain, coordinates per lane): all jobs of a group are one
// launch over their concatenated chains, and groups go to separate streams so that their
// work overlaps on the device.  After the round, finished jobs are retired (their latency
// recorded); their memory is returned when the caller destroys them, which lets the next
// queued jobs in.  Jobs submitted in SYNC mode are the baseline: they run one at a time to
// completion with the synchronised kernels.
#include <algorithm>
#include <chrono>
#include <map>

#include "engine_internal.h"

namespace {

constexpr int kMaxActive = 128;
constexpr int kStreams = 8;
constexpr double kAgingSeconds = 1.0;

using Clock = std::chrono::steady_clock;

// A cancelled job leaves the scheduler (caller holds e->mu).
void cancel_finish_locked(fsmc_engine* e, fsmc_job* j) {
  j->serve_status = FSMC_ECANCELED;
  j->t_done = Clock::now();
  j->finished.store(1);
  e->pending -= 1;
  e->cv.notify_all();
}

void finish_job(fsmc_engine* e, fsmc_job* j, fsmc_status st) {
  j->serve_status = st;
  j->t_done = Clock::now();
  j->finished.store(1);
  std::lock_guard<std::mutex> g(e->mu);
  e->pending -= 1;
  e->cv.notify_all();
}

void scheduler_main(fsmc_engine* e) {
  cudaSetDevice(e->device);
  cudaStream_t streams[kStreams];
  for (auto& s : streams) cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  MultiBuf bufs[kStreams];
  int* h_done = nullptr;
  cudaMallocHost(&h_done, sizeof(int) * kMaxActive);
  std::vector<fsmc_job*> active;
  while (true) {
    // ---- retire cancelled jobs, admit queued ones --------------------------------------------------
    std::vector<fsmc_job*> to_admit;
    {
      std::unique_lock<std::mutex> lk(e->mu);
      for (auto it = active.begin(); it != active.end();) {
        if ((*it)->cancel.load()) {
          cancel_finish_locked(e, *it);
          it = active.erase(it);
        } else {
          ++it;
        }
      }
      if (e->stop) break;
      if (active.empty() && e->queue.empty()) {
        e->cv.wait_for(lk, std::chrono::milliseconds(20));
        continue;
      }
      // arrival order; every queued job is tried (see the admission loop below)
      while (!e->queue.empty() && active.size() + to_admit.size() < (size_t)kMaxActive) {
        fsmc_job* j = e->queue.front();
        if (j->cancel.load()) {
          e->queue.pop_front();
          cancel_finish_locked(e, j);
          continue;
        }
        // the footprint is known only after layout: materialisation refuses with EADMIT
        // when memory is short, and the job returns to the head of the queue
        to_admit.push_back(j);
        e->queue.pop_front();
      }
    }
    std::vector<fsmc_job*> refused;
    bool hold = false;  // an aged job ahead did not fit: keep every later job queued
    const auto now = Clock::now();
    for (fsmc_job* j : to_admit) {
      if (hold) {
        refused.push_back(j);
        continue;
      }
      fsmc_status st = job_materialize(j, streams[0]);
      if (st == FSMC_EADMIT) {
        refused.push_back(j);
        if (std::chrono::duration<double>(now - j->t_submit).count() > kAgingSeconds && j->bytes <= e->budget)
          hold = true;
      } else if (st != FSMC_OK) {
        finish_job(e, j, st);
      } else {
        active.push_back(j);
      }
    }
    for (auto it = refused.begin(); it != refused.end();) {  // larger than the whole budget
      if ((*it)->bytes > e->budget) {
        finish_job(e, *it, fsmc_fail(FSMC_EADMIT, "job footprint exceeds the engine budget"));
        it = refused.erase(it);
      } else {
        ++it;
      }
    }
    if (!refused.empty()) {  // back to the head of the queue, in order; wait for memory
      std::lock_guard<std::mutex> g(e->mu);
      for (auto it = refused.rbegin(); it != refused.rend(); ++it) e->queue.push_front(*it);
    }
    if (active.empty()) {
      std::unique_lock<std::mutex> lk(e->mu);
      e->cv.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    // ---- synchronised baseline: one job at a time, to completion -------------------------------------
    if (active.front()->serve_mode == FSMC_MODE_SYNC) {
      fsmc_job* j = active.front();
      fsmc_status st = job_run_impl(j, FSMC_MODE_SYNC, 0, streams[0]);
      active.erase(active.begin());
      finish_job(e, j, st);
      continue;
    }
    // ---- one FSM round: a fused launch per kernel shape ----------------------------------------------
    std::map<long long, std::vector<fsmc_job*>> groups;
    for (fsmc_job* j : active) {
      if (j->serve_mode != FSMC_MODE_FSM) continue;
      long long key = ((long long)j->algo << 40) | ((long long)j->prec << 32);
      key |= j->algo == FSMC_ESS ? (long long)ess_job_group(j)
                                 : (long long)nuts_group_E(j->d) | ((long long)j->tg->kind << 8);
      if (j->algo == FSMC_DR) key |= 1LL << 20;
      groups[key].push_back(j);
    }
    int gi = 0;
    fsmc_status round_err = FSMC_OK;
    std::vector<std::pair<fsmc_job*, int>> watched;
    for (auto& kv : groups) {
      const int si = gi++ % kStreams;
      std::vector<fsmc_job*>& jobs = kv.second;
      cudaError_t ce = cudaSuccess;
      if (jobs[0]->algo == FSMC_DR) {
        for (fsmc_job* j : jobs) {  // DR jobs are cheap; they advance one launch each
          fsmc_status s = job_run_impl(j, FSMC_MODE_FSM, j->tun.steps_per_launch, streams[si]);
          if (s != FSMC_OK) { round_err = s; break; }
        }
      } else {
        const size_t need = jobs.size() * 1024 + 4096;
        if (multibuf_ensure(bufs[si], need) != FSMC_OK) { round_err = FSMC_ENOMEM; break; }
        ce = jobs[0]->algo == FSMC_ESS ? ess_group_round(jobs, bufs[si], streams[si])
                                       : nuts_group_round(jobs, bufs[si], streams[si]);
      }
      if (ce != cudaSuccess) {
        round_err = fsmc_cuda_fail(ce, "serving round");
        break;
      }
      for (fsmc_job* j : jobs) {
        const int slot = (int)watched.size();
        cudaMemcpyAsync(&h_done[slot], j->dev + j->o_done, sizeof(int), cudaMemcpyDeviceToHost, streams[si]);
        watched.push_back({j, slot});
      }
    }
    for (auto& s : streams) cudaStreamSynchronize(s);
    if (round_err != FSMC_OK) {
      for (fsmc_job* j : active) finish_job(e, j, round_err);
      active.clear();
      continue;
    }
    for (auto& w : watched) {
      fsmc_job* j = w.first;
      if (h_done[w.second] >= j->m) {
        active.erase(std::remove(active.begin(), active.end(), j), active.end());
        finish_job(e, j, FSMC_OK);
      }
    }
  }
  for (auto& b : bufs) multibuf_free(b);
  cudaFreeHost(h_done);
  for (auto& s : streams) cudaStreamDestroy(s);
}

}  // namespace

void serving_shutdown(fsmc_engine* e) {
  {
    std::lock_guard<std::mutex> g(e->mu);
    if (!e->sched_running) return;
    e->stop = true;
    e->cv.notify_all();
  }
  e->sched.join();
  std::lock_guard<std::mutex> g(e->mu);
  e->sched_running = false;
}

void serving_forget(fsmc_job* j) {
  if (!j->submitted) return;
  fsmc_engine* e = j->e;
  std::unique_lock<std::mutex> lk(e->mu);
  if (j->finished.load()) return;
  auto it = std::find(e->queue.begin(), e->queue.end(), j);
  if (it != e->queue.end()) {
    e->queue.erase(it);
    j->finished.store(1);
    e->pending -= 1;
    e->cv.notify_all();
    return;
  }
  if (!e->sched_running) return;
  j->cancel.store(1);
  e->cv.notify_all();
  e->cv.wait(lk, [&] { return j->finished.load() != 0; });
}

extern "C" fsmc_status fsmc_submit(fsmc_engine* e, fsmc_job* j, fsmc_mode mode) {
  if (!e || !j) return fsmc_fail(FSMC_EINVAL, "engine/job is NULL");
  if (j->e != e) return fsmc_fail(FSMC_EINVAL, "job belongs to another engine");
  if (mode != FSMC_MODE_FSM && mode != FSMC_MODE_SYNC) return fsmc_fail(FSMC_EINVAL, "bad mode");
  if (j->submitted || j->dev) return fsmc_fail(FSMC_ESTATE, "job was already submitted or run");
  if (j->tun.step_form == 2) return fsmc_fail(FSMC_EINVAL, "ablation step forms run through fsmc_job_run only");
  if (j->algo == FSMC_SLICE || j->tg->kind == FSMC_TGT_GP_REG)
    return fsmc_fail(FSMC_EINVAL, "slice-sampling and GP_REG jobs run through fsmc_job_run only");
  j->submitted = true;
  j->serve_mode = mode;
  j->t_submit = Clock::now();
  std::lock_guard<std::mutex> g(e->mu);
  e->queue.push_back(j);
  e->pending += 1;
  if (!e->sched_running) {
    e->stop = false;
    e->sched_running = true;
    e->sched = std::thread(scheduler_main, e);
  }
  e->cv.notify_all();
  return FSMC_OK;
}

extern "C" fsmc_status fsmc_poll(fsmc_job* j, int* done, double* latency_s) {
  if (!j) return fsmc_fail(FSMC_EINVAL, "job is NULL");
  if (!j->submitted) return fsmc_fail(FSMC_ESTATE, "job was not submitted");
  const int f = j->finished.load();
  if (done) *done = f;
  if (latency_s) *latency_s = f ? std::chrono::duration<double>(j->t_done - j->t_submit).count() : 0.0;
  if (f && j->serve_status != FSMC_OK) return fsmc_fail(j->serve_status, "job failed in the scheduler");
  return FSMC_OK;
}

extern "C" fsmc_status fsmc_cancel(fsmc_job* j) {
  if (!j) return fsmc_fail(FSMC_EINVAL, "job is NULL");
  if (!j->submitted) return fsmc_fail(FSMC_ESTATE, "job was not submitted");
  fsmc_engine* e = j->e;
  std::lock_guard<std::mutex> g(e->mu);
  if (j->finished.load()) return FSMC_OK;
  auto it = std::find(e->queue.begin(), e->queue.end(), j);
  if (it != e->queue.end()) {
    e->queue.erase(it);
    cancel_finish_locked(e, j);
    return FSMC_OK;
  }
  j->cancel.store(1);  // admitted (or being admitted): retired before the next round
  e->cv.notify_all();
  return FSMC_OK;
}

extern "C" fsmc_status fsmc_wait_all(fsmc_engine* e, double timeout_s) {
  if (!e) return fsmc_fail(FSMC_EINVAL, "engine is NULL");
  std::unique_lock<std::mutex> lk(e->mu);
  const bool ok = e->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return e->pending <= 0; });
  return ok ? FSMC_OK : fsmc_fail(FSMC_ETIMEOUT, "jobs still pending");
}
