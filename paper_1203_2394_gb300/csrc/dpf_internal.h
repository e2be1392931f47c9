// Host-side internals of the library: error reporting, temporary scratch for
// the standalone resampler, the filter context and the kernel-variant table.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dpf.h"

namespace dpf {

dpf_status set_error(dpf_status st, const std::string& msg);
void clear_error();
dpf_status cuda_error(cudaError_t e, const char* what);

// cudaMalloc for the allocations a context, batch or proposal owns; fails with
// cudaErrorMemoryAllocation when dpf_fail_allocation_after has armed it for this call.
cudaError_t device_malloc(void** p, size_t bytes);

// Look-back state of one scan: per-tile flag words and values, and the
// monotone ticket counter that hands out tile indices in launch order.
struct ScanState {
  uint32_t* flags;           // n_tiles words: (epoch << 2) | state, state 1 = aggregate, 2 = prefix
  unsigned long long* agg;   // n_tiles
  unsigned long long* incl;  // n_tiles
  unsigned long long* ticket;
};

// Temporary device memory of one dpf_resample call (stream-ordered allocation).
struct Scratch {
  void* block = nullptr;
  unsigned long long* maxkey = nullptr;
  unsigned long long* C = nullptr;
  int* shift = nullptr;
  int* err = nullptr;
  ScanState scan{};
};
dpf_status scratch_alloc(Scratch& sc, long long tiles, cudaStream_t s);
void scratch_free(Scratch& sc, cudaStream_t s);
// Synchronise, read the device error word, free, and map it to a status.
dpf_status scratch_finish(Scratch& sc, cudaStream_t s, const char* what);
// The status a device error word maps to (0: DPF_OK).
dpf_status err_word_status(int w, const char* what);
// The outer stage with one CTA that never reaches the grid barrier: the waits run
// out and the status is DPF_E_TIMEOUT (dpf_check_bounded_wait).
dpf_status check_outer_barrier(cudaStream_t s);

// Launch the global systematic-resampling kernels on caller-provided scratch
// (laid out as by scratch_alloc and zeroed); no allocation, no synchronisation.
void launch_global_on(const void* w, int32_t dtype, long long n, const uint32_t* u, int32_t* out,
                      Scratch& sc, cudaStream_t s);

// Model constants prepared on the host in double precision, in the internal
// (x-first) coordinate order. Matrices are row-major.
struct HostModel {
  int d1, d2, dy;
  int growth, quad;
  double ga, gb, gc, gw, qc;
  std::vector<double> Axx, Axz, Azx, Azz, Hx, Hz;
  std::vector<double> Lqx, Lqz, LqxInv, LrInv, Ls, K;
  std::vector<double> WAxz, HzAzz, HzAzx, LrHz;
  std::vector<double> m0x, m0z, Lp0x, G0, Lp0c;
  double lognorm_y;
  bool xz;  // x transition depends on z (A_xz != 0)
};

// Device buffers and state of one filter (defined below).
using Ctx = ::dpf_ctx;

// One batched launch: the filters of one (variant, PPL, x-kind) class.
struct BatchLaunch {
  const void* mcs;          // device: the class's model constants, one block per filter
  const void* mc_shared;    // host: the constants when every filter of the class shares them, else null
  const void* descs;        // device: the class's per-filter launch arguments
  const long long* fstart;  // device: F + 1 cumulative group counts
  int F;
  long long chunk;          // groups per warp
  uint32_t region;          // bytes of shared memory per warp
  size_t smem;              // bytes per CTA
  int ppl;
  int mf;                   // 32 ppl when every filter of the class has M = 32 ppl, else 0
  bool xz;
  int grid;
};

// Per-variant launchers, one set per compiled (precision, d1, d2, dy).
// Tiles of the decoupled look-back scan of the global resampling.
constexpr int SCAN_NT = 256;   // threads per scan tile
constexpr int SCAN_IPT = 8;    // items per thread
constexpr int SCAN_TILE = SCAN_NT * SCAN_IPT;
// the outer stage of a step (dpf_outer.cuh): threads a CTA, items a thread in one
// chunk, items a chunk, the bound on its grid (rows of partial sums, count totals),
// and the sums a filter: W, W^2 and the d <= 64 weighted means
constexpr int OF_NT = 256;
constexpr int OF_IPT = 2;
constexpr int OF_CHUNK = OF_NT * OF_IPT;
constexpr int OF_MAX_CTAS = 1024;
constexpr int OF_MAX_NV = 2 + 64;

struct Variant {
  int prec, d1, d2, dy;
  dpf_status (*make_const)(const HostModel&, std::vector<unsigned char>&);
  dpf_status (*init)(Ctx&);
  dpf_status (*step)(Ctx&, int profile_slot);
  dpf_status (*outer)(Ctx&, double* mean_out, double* logz_out, cudaStream_t s);
  dpf_status (*pf_step)(Ctx&) = nullptr;  // the bootstrap particle filter's step (null: none)
  dpf_status (*std_step)(Ctx&) = nullptr;  // the DPF without look-ahead (null: none)
  // the outer stage in two launches, for many filters at once: the per-filter
  // arguments, the filter's CTA count, the sums (one variant), then the
  // resampling and statistics (any variant of the precision)
  void (*outer_args)(Ctx&, double* mean_out, double* logz_out, void* args);
  int (*outer_ctas)(long long N) = nullptr;
  dpf_status (*outer_batch)(const void* args, const int* cstart, int nctas, int F, cudaStream_t s);
  dpf_status (*scan_batch)(const void* args, const int* cstart, int nctas, int F, cudaStream_t s);
  size_t (*step_smem)(int M, int L, bool xz, int nt);
  int (*xpad)();
  void (*batch_args)(Ctx&, const void* y_prev, const void* y_cur, bool xz, void* out);
  size_t (*region_bytes)(int M, int L, bool xz);
  dpf_status (*batch_launch)(const BatchLaunch&, cudaStream_t, int* occ);
  // a batched member's step as its own launch of the single-filter kernel
  dpf_status (*single_launch)(Ctx&, const void* args, int ppl, bool xz, cudaStream_t s) = nullptr;
  bool batch_serial = false;  // its launches share state (a constant bank): one stream
  bool (*use_xz)(const Ctx&);
  int (*ppl_for)(int M);
  size_t args_size, const_size, oargs_size;
  int max_m = 1024;       // largest M the variant's kernels accept
  bool has_tc = false;    // has a tensor-core propagation (see dpf_set_tensor_cores)
  bool xz_supported = true;  // serves models whose x transition depends on z
};
const Variant* find_variant(int prec, int d1, int d2, int dy);
// the paper's models 1 and 2 (FP32); swapped: model 1 with the table's z as the outer block
const Variant* find_paper_variant(int kind, bool swapped);
dpf_status learned_inner_step(Ctx& x);
bool oa_wide_shape(const Ctx& x);  // the amortised proposal's wide pass serves this filter
dpf_status oa_wide_step(Ctx& x, dpf_proposal& p);
dpf_status oa_wide_record(Ctx& x, long long i0, long long n_outer, float* G, float* Z, float* w);
dpf_status learned_fallback_lists(Ctx& x);  // dpf_learned_step.cu
int dpf_proposal_dout(const dpf_proposal* p);  // head outputs of a proposal
int dpf_proposal_kind(const dpf_proposal* p);  // 0 mixture, 1 outer-amortised

}  // namespace dpf

struct dpf_ctx {
  // sizes
  int prec = 0, d = 0, d1 = 0, d2 = 0, dy = 0;
  long long N = 0;
  int M = 0, L = 0;
  uint64_t seed = 0;
  cudaStream_t stream = nullptr;
  std::vector<int> perm;
  dpf::HostModel hm;
  const dpf::Variant* var = nullptr;
  int model_id = 0;  // 0 a conditionally linear-Gaussian model; 2, 3 the paper's models, 4 model 1 swapped
  std::vector<unsigned char> mconst;  // device-constant model block (variant layout)
  // device state (element type = precision)
  void* z[2] = {nullptr, nullptr};
  void* lq[2] = {nullptr, nullptr};
  void* x[2] = {nullptr, nullptr};
  void* lwh[2] = {nullptr, nullptr};
  void* xbb[2] = {nullptr, nullptr};
  void* lw = nullptr;
  void* xm = nullptr;
  void* zm = nullptr;
  void* wout = nullptr;
  void* yb = nullptr;   // 2 x dy observations (slot t % 2 holds y_t)
  int32_t* anc = nullptr;
  int32_t* sel = nullptr;
  int32_t* dbg_b = nullptr;
  int32_t* dbg_j = nullptr;     // debug: the look-ahead's mixture components (N x L; Table 1 models)
  int32_t* anc_prev = nullptr;  // debug: the ancestors the last inner update used
  void* dbg_head = nullptr;     // debug: the learned proposal's head outputs of the last inner update
  void* oa_bidx = nullptr;      // amortised proposal: local resampling indices, group features, head outputs
  void* oa_feat = nullptr;
  void* oa_out = nullptr;
  void* oa_hidden = nullptr;    // ... and at the wide size, two N x hidden buffers of the network's layers
  void* oa_mu = nullptr;        // ... and the prior means of the inner particles, [d2][N M]
  // small device block: reduction partials, statistics, counters, error word
  void* small = nullptr;
  double* stats = nullptr;          // [logZ_total, logZ_step, ess, s1, mean[d]]
  // pinned, mapped host mirror of the statistics and the error word (4 + d + 1 doubles),
  // written by the outer stage of a dpf_step call with host outputs, so that the call
  // reads them after one synchronisation instead of two device-to-host copies
  double* hstats = nullptr;
  double* hstats_dev = nullptr;     // ... its device address
  bool host_out = false;            // the coming outer stage writes the mirror
  double* diag_inner = nullptr;     // [sum of the groups' inner ESS, their minimum (as bits)]
  void* lwmax_t = nullptr;          // the largest log-weight of the step, as T
  unsigned long long* lwmax_key = nullptr;
  unsigned long long* Csum = nullptr;
  unsigned int* done = nullptr;
  double* partials = nullptr;       // the outer stage's sums, one row a CTA
  unsigned long long* ctot = nullptr;  // ... and its quantised count totals
  int* err = nullptr;
  // step counter (number of completed steps)
  long long t = 0;
  bool debug = false;
  int ppt = 1;        // inner particles per thread of the step kernel
  int xp = 4;         // padded x row length (elements; 16-byte rows)
  int grid_step = 0;  // persistent grid of the step kernel (0 = not yet sized)
  const void* grid_kernel = nullptr;  // ... the warp-step kernel it was sized for
  void* d_mconst = nullptr;  // the model constants in device memory (variants that read them there)
  bool tensor_cores = true;  // tensor-core propagation where the variant has one
  dpf_proposal* proposal = nullptr;  // learned inner proposal (null: the prior)
  bool la_only = false;      // the next step kernel runs the look-ahead only
  bool pf = false;           // a bootstrap particle filter (dpf_create_pf), not the LA-DPF
  bool std_dpf = false;      // the DPF without look-ahead (dpf_create_std)
  bool std_gauss = false;    // ... drawing x_t from the mixture's moment-matched Gaussian
  // the learned proposal's per-group fallback to the plain inner update
  double fb_frac = 0.25;          // a group falls back when its inner ESS < fb_frac * M (0: never)
  int32_t* fb_flag = nullptr;     // [N] 1 where the last learned inner update fell back
  int32_t* fb_list = nullptr;     // [N] the groups that fall back
  int32_t* fb_count = nullptr;    // [1] their count
  const int32_t* glist_cur = nullptr;   // the next step kernel's group subset (null: all)
  const int32_t* gcount_cur = nullptr;
  const int32_t* gskip_cur = nullptr;   // ... groups it leaves untouched (null: none)
  // profiling of the main kernel
  bool profiling = false;
  std::vector<cudaEvent_t> pev;  // pairs bracketing the step kernel
  size_t pev_used = 0;
  size_t bytes = 0;
  std::vector<void*> allocs;
};
