// Autotuner for the FSM launch shape (fsmc_autotune in include/fsmc.h).
//
// A candidate shape is timed on a scratch job with the caller's chain count: a short warm-up
// run, then a timed run of a fixed number of rounds; the score is device time per FSM state
// executed (every state costs one expensive evaluation, so this is the quantity the shape
// can change -- the samples themselves do not depend on it).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "engine_internal.h"

namespace {

std::string tune_key(fsmc_engine* e, fsmc_target* t, fsmc_algo algo, fsmc_precision prec, int64_t m) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, e->device);
  std::string name(prop.name);
  for (auto& ch : name) if (ch == ' ') ch = '_';
  const int lg = (int)std::floor(std::log2((double)std::max<int64_t>(1, m)));
  std::ostringstream k;
  k << name << ":a" << (int)algo << ":t" << t->kind << ":d" << t->d << ":n" << t->n_data << ":p" << (int)prec
    << ":m" << lg;
  return k.str();
}

bool cache_lookup(const std::string& path, const std::string& key, fsmc_tuning* out) {
  std::ifstream f(path);
  if (!f) return false;
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    std::istringstream is(line);
    std::string k;
    fsmc_tuning t{};
    if (is >> k >> t.lanes_per_chain >> t.steps_per_launch >> t.ring_slots >> t.threads_per_block >> t.generator &&
        k == key) {
      *out = t;  // the last entry for a key wins
      found = true;
    }
  }
  return found;
}

void cache_store(const std::string& path, const std::string& key, const fsmc_tuning& t) {
  std::ofstream f(path, std::ios::app);
  if (f) f << key << " " << t.lanes_per_chain << " " << t.steps_per_launch << " " << t.ring_slots << " "
           << t.threads_per_block << " " << t.generator << "\n";
}

std::vector<fsmc_tuning> candidates(fsmc_target* t, fsmc_algo algo, fsmc_precision prec) {
  std::vector<fsmc_tuning> c;
  if (algo == FSMC_ESS && t->kind == FSMC_TGT_GP_REG) {
    for (int steps : {4, 8, 16}) c.push_back(fsmc_tuning{32, steps, 0, 32, 0, 0, 2});
  } else if (algo == FSMC_ESS) {
    std::vector<int> lanes = {32};
    if (t->d <= 32) lanes.push_back(1);
    if (t->d > 32 && t->d <= 512) lanes.push_back(16);
    if (t->d > 32 && t->d <= 256) lanes.push_back(8);
    std::vector<int> gens = {1};
    if (prec == FSMC_FP32 && t->d <= 256) gens.push_back(2);
    // (states per launch, ring slots): short rounds, and the long rounds that amortise the
    // refill and FSM launches' fixed costs on large jobs
    const int shapes[][2] = {{32, 32}, {32, 64}, {64, 32}, {64, 64}, {128, 32}, {128, 64}, {384, 128}};
    for (int G : lanes)
      for (const auto& sr : shapes)
        for (int gen : gens)
          for (int threads : (G == 1 ? std::vector<int>{128, 256} : std::vector<int>{256}))
            c.push_back(fsmc_tuning{G, sr[0], sr[1], threads, 0, gen, 0});
  } else if (algo == FSMC_DR || algo == FSMC_SLICE) {
    for (int steps : {64, 128, 256, 512, 1024})
      for (int threads : {64, 128, 256}) c.push_back(fsmc_tuning{1, steps, 0, threads, 0, 0, 0});
  } else {
    for (int steps : {32, 128, 256}) c.push_back(fsmc_tuning{32, steps, 0, 128, 0, 0, 0});
  }
  return c;
}

}  // namespace

extern "C" fsmc_status fsmc_autotune(fsmc_engine* e, fsmc_target* t, fsmc_algo algo, const void* algo_params,
                                     fsmc_precision prec, int64_t n_chains, const char* cache_path,
                                     fsmc_tuning* best) {
  if (!e || !t || !best) return fsmc_fail(FSMC_EINVAL, "engine/target/best is NULL");
  if (n_chains < 1) return fsmc_fail(FSMC_EINVAL, "n_chains must be >= 1");
  std::string path = cache_path ? cache_path : (getenv("FSMC_TUNE_CACHE") ? getenv("FSMC_TUNE_CACHE") : "");
  const std::string key = tune_key(e, t, algo, prec, n_chains);
  if (!path.empty() && cache_lookup(path, key, best)) return FSMC_OK;

  const std::vector<fsmc_tuning> cand = candidates(t, algo, prec);
  double best_score = 1e300;
  fsmc_tuning best_t{};
  std::string last_err;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return fsmc_cuda_fail(cudaGetLastError(), "stream");
  for (const fsmc_tuning& tu : cand) {
    const int rounds = 6;
    const int64_t n = std::max<int64_t>(64, (int64_t)(rounds + 2) * tu.steps_per_launch + 8);
    fsmc_job* j = nullptr;
    fsmc_status s = fsmc_job_create(e, t, algo, algo_params, prec, n_chains, n, nullptr, 12345, 0, &j);
    if (s != FSMC_OK) { last_err = fsmc_last_error(); continue; }
    s = fsmc_job_set_tuning(j, &tu);
    if (s == FSMC_OK) s = fsmc_job_run(j, FSMC_MODE_FSM, 2 * tu.steps_per_launch, st);  // warm-up
    fsmc_stats a{}, b{};
    if (s == FSMC_OK) s = fsmc_read_stats(j, &a);
    if (s == FSMC_OK) s = fsmc_job_run(j, FSMC_MODE_FSM, (int64_t)rounds * tu.steps_per_launch, st);
    if (s == FSMC_OK) s = fsmc_read_stats(j, &b);
    if (s == FSMC_OK && b.fsm_steps > a.fsm_steps) {
      const double score = b.device_ms / (double)(b.fsm_steps - a.fsm_steps);
      if (score < best_score) { best_score = score; best_t = tu; }
    } else if (s != FSMC_OK) {
      last_err = fsmc_last_error();
    }
    fsmc_job_destroy(j);
  }
  cudaStreamDestroy(st);
  if (best_score >= 1e300) return fsmc_fail(FSMC_EINVAL, "autotune: no candidate ran (" + last_err + ")");
  *best = best_t;
  if (!path.empty()) cache_store(path, key, best_t);
  return FSMC_OK;
}
