// Structure-of-arrays job views passed by value to the kernels, and the host-side
// launchers each sampler's .cu file exports to the engine.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fsmc {

template <typename T> struct TargetView;
struct GridBarrier;

// Fields common to every sampler: chain range, sample bookkeeping, outputs.
template <typename T>
struct ChainsView {
  int64_t m;             // chains in this view
  int n;                 // samples per chain
  uint32_t chain0;       // global chain id of chain 0 (RNG key)
  uint32_t seed_lo, seed_hi;
  T* x;                  // [m][d] current state
  int* t;                // [m] samples emitted
  T* out;                // [m][n][d] samples, or null (moments only)
  T* mom;                // [4][m][d] Kahan sums of x and x^2 (moments only)
  size_t mom_stride;     // m * d
  int* counts;           // [m][n] loop-body count N_ij
  long long* steps;      // [m] FSM states executed
  int* err;              // error word
  int* chains_done;      // chains that reached n
  int step_form = 1;     // 1: bundled + amortised / condensed step; 2: the paper's ablation forms
};

template <typename T>
struct EssView : ChainsView<T> {
  TargetView<T> tg;
  int W;                 // ring slots per chain
  int dstride;           // ring row stride (elements)
  T* ell;                // [m] log f(x)
  T* logy;               // [m] threshold
  T* th; T* thmin; T* thmax;  // [m] angle and bracket
  int* k;                // [m] FSM state
  int* s;                // [m] shrinks in the current sample
  int* gen_lo; int* gen_hi;   // [m] ring fill window [gen_lo, gen_hi) in samples
  T* nu;                 // [m][W][dstride] pre-generated ellipse directions
  unsigned long long* gen_cols;  // directions generated so far (statistics)
  int own_window;        // 1: the FSM kernel sets the next refill window itself
  // Compacted refill list (tensor-core generator): col_base[c] = sum over chains c' < c of
  // gen_hi - gen_lo, col_base[m] = total; colmap[j] = (chain, sample) of refill column j.
  // Null: the generator walks (chain block, ring offset) tiles instead.
  long long* col_base = nullptr;
  int2* colmap = nullptr;
};

template <typename T>
struct DrView : ChainsView<T> {
  TargetView<T> tg;
  int n_stages;
  int symmetric;         // 1: symmetric delayed rejection, re-centred tries (sig[0] each)
  T sig[3];              // stage scales
  T* lp;                 // [m] log pi(x)
  T* y;                  // [3][m][d] rejected proposals y1, y2 of the current sample; the
                         // current proposal (4-state ablation form)
  T* lpy;                // [10][m] log pi(y1), log pi(y2); the current proposal's log pi and ratio;
                         // the later stages' kept ratio terms (DrCache in dr.cu)
  int* k;                // [m] next stage to try
  int lanes = 1;         // 1: a chain per thread (d <= 32); 32: a chain per warp (d <= 1024)
};

// ESS on a target whose likelihood is one dense linear-algebra problem per evaluation (GP
// regression, Sec. 7.2): a chain per warp, the likelihood warp-wide.
template <typename T>
struct EssBlockView : ChainsView<T> {
  TargetView<T> tg;      // prior factor L [d][d]; GP_REG: X = D [n][n], vec = y [n], n_data = n
  T* ell;                // [m] log f(x)
  T* logy;               // [m] threshold
  T* th; T* thmin; T* thmax;  // [m] angle and bracket
  T* nu;                 // [m][d] the current sample's ellipse direction
  int* k;                // [m] FSM state
  int* s;                // [m] shrinks in the current sample
  unsigned* work;        // chain counter of the current FSM launch (zeroed before each launch)
  T* spill;              // per-CTA scratch for covariance rows beyond shared memory
  size_t spill_stride;   // its elements per CTA
  int64_t max_ctas;      // CTAs the scratch has room for (launches use at most this many)
  int rows_smem;         // covariance rows kept in shared memory (the rest in the scratch)
  int wpc = 0;           // warps per chain's CTA: 1, 2 or 4; 0 chooses by chain count
};

template <typename T>
struct SliceView : ChainsView<T> {
  TargetView<T> tg;
  T w;                   // step-out width
  int mlim;              // stepping-out limit m (J + K = m - 1 steps at most)
  T* lp;                 // [m] log pi(x)
  T* logy;               // [m] threshold of the current sample
  T* L; T* R; T* th;     // [m] interval ends and the current proposal, along the line
  T* u;                  // [m][d] the current sample's direction
  int* k;                // [m] state: 0 start of a sample, 1 left end, 2 right end, 3 proposal
  int* J; int* K;        // [m] stepping-out budgets left
  int* s;                // [m] proposals made in the current sample
  int* nev;              // [m] log-density evaluations in the current sample
  int* aux;              // [m][n] proposals per sample
  int lanes = 1;         // 1: a chain per thread (d <= 32); 32: a chain per warp (d <= 1024)
};

template <typename T>
cudaError_t launch_ess_nu_gen(const EssView<T>& v, cudaStream_t st);
template <typename T>
cudaError_t launch_ess_fsm(const EssView<T>& v, int G, int budget, int threads, cudaStream_t st);
// Synchronised ESS program (Alg. 6) for samples [t0, t1): form 1 the sweep kernel, form 2 the
// kernel with a compacted list of the chains still in the loop (lists: [2][m] ints); both
// cooperative, one grid barrier per loop iteration.
template <typename T>
cudaError_t launch_ess_sync(const EssView<T>& v, int G, int t0, int t1, GridBarrier bar,
                            unsigned* active_cnt, unsigned long long* iters, int threads, int form,
                            int* lists, cudaStream_t st);
// Form 3: the list iterations as kernels of a graph with conditional while nodes; cg_state is
// kEssCgStateBytes of device memory, built once per job and launched per chunk of samples.
constexpr size_t kEssCgStateBytes = 64;
template <typename T>
cudaError_t build_ess_sync_graph(const EssView<T>& v, int G, int threads, void* cg_state, int* lists,
                                 unsigned long long* iters, cudaGraphExec_t* out);
cudaError_t launch_ess_sync_graph(cudaGraphExec_t exec, void* cg_state, int t0, int t1, cudaStream_t st);
template <typename T>
cudaError_t launch_ess_init(const EssView<T>& v, cudaStream_t st);
// Fused launches over several ESS jobs: views[k] is job k's view in device memory and
// off[k] .. off[k+1] its range of work items (direction tiles, or chains).
template <typename T>
cudaError_t launch_ess_nu_gen_multi(const EssView<T>* views, const int64_t* off, int njobs,
                                    int64_t total_tiles, cudaStream_t st);
template <typename T>
cudaError_t launch_ess_fsm_multi(const EssView<T>& any, int G, const EssView<T>* views, const int64_t* off,
                                 int njobs, int64_t total, int budget, int threads, cudaStream_t st);
int ess_group_E(int G, int d);
// Tensor-core direction generator (d <= 256, FP32): L image in the MMA layout, built once
// per target, and the persistent generator kernel.
size_t ess_tc_image_bytes(int d);
cudaError_t launch_ess_tc_build(const float* L, int d, unsigned char* img, cudaStream_t st);
cudaError_t launch_ess_nu_gen_tc(const EssView<float>& v, const unsigned char* img, int sms, cudaStream_t st);
// its two halves: the compacted column list of the refill (prefix sum over the chains' refill
// counts, then the (chain, sample) list), and the generator kernel that walks it
cudaError_t launch_ess_tc_cols(const EssView<float>& v, cudaStream_t st);
cudaError_t launch_ess_tc_gen(const EssView<float>& v, const unsigned char* img, int sms, cudaStream_t st);

template <typename T>
cudaError_t launch_dr_fsm(const DrView<T>& v, int budget, int threads, cudaStream_t st);
template <typename T>
cudaError_t launch_dr_sync(const DrView<T>& v, int t0, int t1, GridBarrier bar, unsigned* active_cnt,
                           unsigned long long* iters, int threads, cudaStream_t st);
template <typename T>
cudaError_t launch_dr_init(const DrView<T>& v, cudaStream_t st);

// GP_REG likelihood: the packed lower triangle in shared memory, the rows that do not fit in a
// per-CTA scratch block; n <= kGpRegMaxN32 (FP32) / kGpRegMaxN64 (FP64).
constexpr int kGpRegMaxN32 = 512, kGpRegMaxN64 = 512;
template <typename T>
size_t gpreg_spill_elems(int n);
template <typename T>
int gpreg_smem_rows(int n);
// warps per chain of a GP-regression job of m chains on `sms` SMs when the caller leaves it open
int ess_block_auto_wpc(int64_t m, int sms);
template <typename T>
cudaError_t launch_ess_block_fsm(const EssBlockView<T>& v, int budget, cudaStream_t st);
template <typename T>
cudaError_t launch_ess_block_sync(const EssBlockView<T>& v, int t0, int t1, GridBarrier bar, unsigned* active_cnt,
                                  unsigned long long* iters, cudaStream_t st);
template <typename T>
cudaError_t launch_ess_block_init(const EssBlockView<T>& v, cudaStream_t st);

template <typename T>
cudaError_t launch_slice_fsm(const SliceView<T>& v, int budget, int threads, cudaStream_t st);
template <typename T>
cudaError_t launch_slice_sync(const SliceView<T>& v, int t0, int t1, GridBarrier bar, unsigned* active_cnt,
                              unsigned long long* iters, int threads, cudaStream_t st);
template <typename T>
cudaError_t launch_slice_init(const SliceView<T>& v, cudaStream_t st);

cudaError_t launch_fill_int(int* p, int64_t n, int value, cudaStream_t st);

// Device reduction of a job's run statistics (stats.cu): one record the host copies back.
struct DevStats {
  long long tmin;                // min_j t_j: samples every chain has completed
  long long samples_done;        // sum_j t_j
  long long fsm_steps;           // sum_j FSM states executed
  unsigned long long sum_all;    // sum over i < tmin, all j, of N_ij
  unsigned long long sum_max;    // sum over i < tmin of max_j N_ij
  long long iters;               // synchronised loop-body iterations
  long long err;                 // error word
  long long pad;
};
// colmax: [n] scratch; out: the record (device memory).
cudaError_t launch_job_stats(const int* counts, const int* t, const long long* steps, int64_t m, int n,
                             const unsigned long long* iters, const int* err, unsigned* colmax,
                             DevStats* out, cudaStream_t st);
// dst[i] = (T) src[i], i < n (device arrays).
template <typename T>
cudaError_t launch_from_double(const double* src, int64_t n, T* dst, cudaStream_t st);
// Next refill window for the pipelined ESS rounds: lo = hi_cur, hi = max(lo, min(t + W, n)),
// written to v's gen_lo / gen_hi.
template <typename T>
cudaError_t launch_ess_window(const EssView<T>& v, const int* hi_cur, cudaStream_t st);
// Per-chain Kahan sums of x and x^2 over the first t[c] stored samples: out [4][m][d]
// (sum, compensation, sum of squares, compensation).
template <typename T>
cudaError_t launch_moments_from_samples(const T* samples, const int* t, int64_t m, int n, int d, T* out,
                                        cudaStream_t st);
// Sums of x and x^2 from the [4][md] moment buffer as doubles into out [2][md].
template <typename T>
cudaError_t launch_moments_to_double(const T* mom, int64_t md, double* out, cudaStream_t st);

}  // namespace fsmc
