// Batched form: many independent filters (different N, M, models and x/z
// splits) stepped together. Filters of one (precision, d1, d2, dy, PPL,
// x-kind) class share one persistent launch of the warp-per-group kernel; the
// outer reductions of all filters of one variant share one launch, and the
// outer resamplings of all filters one more, so a step is a fixed, small
// number of launches whatever the number of filters. A whole run of T steps
// can be captured as one CUDA graph. The launch shape of each class is chosen
// by a small autotuner that times the candidates on the live state.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "dpf_internal.h"

namespace dpf {

constexpr int BATCH_AUX_STREAMS = 3;  // streams beside the batch's own for a step's launches

struct BatchClass {
  const Variant* var = nullptr;
  bool xz = false;
  int ppl = 1;
  std::vector<int> members;      // filter indices
  std::vector<long long> fstart; // host copy
  long long* d_fstart = nullptr;
  void* d_mcs = nullptr;
  void* d_descs = nullptr;       // a ring of descriptor sets
  size_t desc_bytes = 0;         // one set
  int ring = 0;                  // sets in the ring
  BatchLaunch launch{};
  std::vector<unsigned char> shared_mc;  // the constants, when all members share them
  int occ = 0;                   // CTAs per SM at this launch shape
  double tuned_us = 0.0;
  // the other schedule the autotuner may pick: one launch a member of the single-filter
  // step kernel, its launch arguments and model constants launch parameters (read as
  // constant-bank operands), instead of one launch for the class with each filter's
  // arguments and constants staged in shared memory; the results are the same
  bool split = false;
  std::vector<unsigned char> host_descs;   // the descriptor set of the coming step, host copy
  const unsigned char* host_cur = nullptr; // the set the next launch reads (split)
};

// The filters of one variant, whose outer reductions share a launch.
struct OuterGroup {
  const Variant* var = nullptr;
  std::vector<int> members;      // filter indices
  int nblocks = 0;               // CTAs of the sums launch: the members' outer-stage CTAs
  int* d_bstart = nullptr;       // prefix of the members' CTA counts
  void* d_oargs = nullptr;       // a ring of argument sets, one FusedOuterArgs per member
  size_t set_bytes = 0;
  const void* cur = nullptr;     // the set the next launch reads
};

}  // namespace dpf

struct dpf_batch {
  int F = 0, d = 0, dy = 0, prec = 0;
  size_t s = 4;
  cudaStream_t stream = nullptr;
  std::vector<dpf_ctx*> ctx;
  std::vector<dpf::BatchClass> cls;
  std::vector<dpf::OuterGroup> og;
  int* d_tstart = nullptr;      // prefix of the filters' outer-stage CTA counts
  int ntiles = 0;               // their sum: CTAs of the resampling launch
  void* d_gargs = nullptr;      // a ring of sets of F outer-stage arguments, in filter order
  size_t gset_bytes = 0;
  const void* gcur = nullptr;
  int oring = 0;                // sets in the outer-argument rings
  void* yhist = nullptr;  // [2][F][dy]: slot t % 2 holds y_t
  long long t = 0;
  int nsm = 0;
  bool profiling = false;
  std::vector<cudaEvent_t> pev;
  size_t pev_used = 0;
  // streams beside `stream` over which a step's kernel launches are spread (the filters
  // are independent, so one launch can take the SMs another's tail leaves idle), and
  // the events that fork them from `stream` and join them back
  std::vector<cudaStream_t> aux;
  cudaEvent_t fork_ev = nullptr;
  std::vector<cudaEvent_t> join_ev;
  std::vector<void*> allocs;
};

namespace dpf {

static dpf_status balloc(dpf_batch& b, void** p, size_t bytes) {
  cudaError_t e = device_malloc(p, bytes < 16 ? 16 : bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(DPF_E_NOMEM, "batch: device allocation failed");
  }
  b.allocs.push_back(*p);
  return DPF_OK;
}

// Grid and chunking of one class at its current PPL (nothing to shape for a variant
// without a launch for a whole class, whose members always launch one by one).
static dpf_status shape_class(dpf_batch& b, BatchClass& c) {
  if (!c.var->batch_launch) {
    c.split = true;
    return DPF_OK;
  }
  size_t region = 0;
  for (int f : c.members) region = std::max(region, c.var->region_bytes(b.ctx[f]->M, b.ctx[f]->L, c.xz));
  c.launch.region = (uint32_t)region;
  // WARPS_PER_CTA warps per CTA, then one filter's launch arguments and, unless the
  // class shares one set, its model constants
  c.launch.smem = region * 4 + (c.var->args_size + 15) / 16 * 16 +
                  (c.shared_mc.empty() ? (c.var->const_size + 15) / 16 * 16 : 0);
  c.launch.ppl = c.ppl;
  bool full = true;  // every lane of every member holds ppl particles: the compile-time-M kernel
  for (int f : c.members) full &= b.ctx[f]->M == 32 * c.ppl;
  c.launch.mf = full ? 32 * c.ppl : 0;
  c.launch.xz = c.xz;
  c.launch.F = (int)c.members.size();
  c.launch.fstart = c.d_fstart;
  c.launch.mcs = c.d_mcs;
  c.launch.mc_shared = c.shared_mc.empty() ? nullptr : c.shared_mc.data();
  int occ = 0;
  dpf_status st = c.var->batch_launch(c.launch, nullptr, &occ);
  if (st) return st;
  c.occ = occ > 0 ? occ : 1;
  const long long total = c.fstart.back();
  const long long warps_max = (long long)c.occ * b.nsm * 4;
  const long long warps = std::max<long long>(1, std::min<long long>(warps_max, total));
  c.launch.chunk = (total + warps - 1) / warps;
  c.launch.grid = (int)((((total + c.launch.chunk - 1) / c.launch.chunk) + 3) / 4);
  return DPF_OK;
}

// The step kernel launches of one class (its descriptors at c.launch.descs, and at
// c.host_cur on the host), each on the stream `next` returns.
template <typename Next>
static dpf_status class_launch(dpf_batch& b, BatchClass& c, Next next) {
  if (!c.split) return c.var->batch_launch(c.launch, next(), nullptr);
  for (size_t q = 0; q < c.members.size(); ++q) {
    dpf_status st = c.var->single_launch(*b.ctx[c.members[q]], c.host_cur + q * c.var->args_size, c.ppl,
                                         c.xz, next());
    if (st) return st;
  }
  return DPF_OK;
}

// Fill descriptor set `slot` of every class for the coming step (y rows given).
static dpf_status upload_descs(dpf_batch& b, const void* y_prev_rows, const void* y_cur_rows,
                               int slot, cudaStream_t s) {
  for (BatchClass& c : b.cls) {
    std::vector<unsigned char>& host = c.host_descs;
    host.assign(c.desc_bytes, 0);
    const size_t as = c.var->args_size;
    for (size_t q = 0; q < c.members.size(); ++q) {
      const int f = c.members[q];
      c.var->batch_args(*b.ctx[f], (const char*)y_prev_rows + (size_t)f * b.dy * b.s,
                        (const char*)y_cur_rows + (size_t)f * b.dy * b.s, c.xz,
                        host.data() + q * as);
    }
    void* dst = (char*)c.d_descs + (size_t)slot * c.desc_bytes;
    cudaError_t e = cudaMemcpyAsync(dst, host.data(), c.desc_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "batch: descriptor upload");
    // pageable source: the copy is staged before cudaMemcpyAsync returns; the host copy
    // stays for the split schedule's launches, which take the arguments as parameters
    c.launch.descs = dst;
    c.host_cur = host.data();
  }
  return DPF_OK;
}

// Arguments of the outer stages that follow the coming step, one set per step
// from `slot` on (counters advanced as the launches will consume them).
static void fill_outer(dpf_batch& b, double* means_dev, double* logz_dev,
                       std::vector<std::vector<unsigned char>>& oh, std::vector<unsigned char>& gh,
                       size_t k) {
  for (size_t gi = 0; gi < b.og.size(); ++gi) {
    OuterGroup& g = b.og[gi];
    for (size_t q = 0; q < g.members.size(); ++q) {
      const int f = g.members[q];
      unsigned char* dst = oh[gi].data() + k * g.set_bytes + q * g.var->oargs_size;
      g.var->outer_args(*b.ctx[f], means_dev ? means_dev + (size_t)f * b.d : nullptr,
                        logz_dev ? logz_dev + f : nullptr, dst);
      memcpy(gh.data() + k * b.gset_bytes + (size_t)f * g.var->oargs_size, dst, g.var->oargs_size);
    }
  }
}

static dpf_status upload_outer(dpf_batch& b, std::vector<std::vector<unsigned char>>& oh,
                               std::vector<unsigned char>& gh, int slot, size_t nsets, cudaStream_t s) {
  for (size_t gi = 0; gi < b.og.size(); ++gi) {
    OuterGroup& g = b.og[gi];
    char* dst = (char*)g.d_oargs + (size_t)slot * g.set_bytes;
    cudaError_t e = cudaMemcpyAsync(dst, oh[gi].data(), g.set_bytes * nsets, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "batch: outer argument upload");
    g.cur = dst;
  }
  char* dst = (char*)b.d_gargs + (size_t)slot * b.gset_bytes;
  cudaError_t e = cudaMemcpyAsync(dst, gh.data(), b.gset_bytes * nsets, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_error(e, "batch: resampling argument upload");
  b.gcur = dst;
  return DPF_OK;
}

static void outer_host_sets(dpf_batch& b, size_t nsets, std::vector<std::vector<unsigned char>>& oh,
                            std::vector<unsigned char>& gh) {
  oh.resize(b.og.size());
  for (size_t gi = 0; gi < b.og.size(); ++gi) oh[gi].assign(b.og[gi].set_bytes * nsets, 0);
  gh.assign(b.gset_bytes * nsets, 0);
}

// One batched step whose descriptors are already in place.
static dpf_status step_launch(dpf_batch& b) {
  // the profiling events time live launches only: an event recorded while a stream is
  // being captured into a graph becomes a dependency, not a timestamp
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(b.stream, &cs);
  const bool prof = b.profiling && cs == cudaStreamCaptureStatusNone;
  if (prof) {
    if (b.pev_used + 2 > b.pev.size())
      for (int q = 0; q < 64; ++q) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return cuda_error(cudaGetLastError(), "event");
        b.pev.push_back(e);
      }
    cudaEventRecord(b.pev[b.pev_used], b.stream);
  }
  // the launches go round the batch's stream and its auxiliary streams, forked from and
  // joined back to the batch's stream
  const int S = 1 + (int)b.aux.size();
  if (S > 1) {
    cudaEventRecord(b.fork_ev, b.stream);
    for (cudaStream_t s : b.aux) cudaStreamWaitEvent(s, b.fork_ev, 0);
  }
  int k = 0;
  auto next = [&]() { const int q = k++ % S; return q == 0 ? b.stream : b.aux[q - 1]; };
  auto own = [&]() { return b.stream; };
  for (BatchClass& c : b.cls) {
    dpf_status st = c.var->batch_serial ? class_launch(b, c, own) : class_launch(b, c, next);
    if (st) return st;
  }
  for (size_t q = 0; q < b.aux.size(); ++q) {
    cudaEventRecord(b.join_ev[q], b.aux[q]);
    cudaStreamWaitEvent(b.stream, b.join_ev[q], 0);
  }
  if (prof) {
    cudaEventRecord(b.pev[b.pev_used + 1], b.stream);
    b.pev_used += 2;
  }
  for (OuterGroup& g : b.og) {
    dpf_status st = g.var->outer_batch(g.cur, g.d_bstart, g.nblocks, (int)g.members.size(), b.stream);
    if (st) return st;
  }
  dpf_status st = b.og[0].var->scan_batch(b.gcur, b.d_tstart, b.ntiles, b.F, b.stream);
  if (st) return st;
  for (int f = 0; f < b.F; ++f) b.ctx[f]->t += 1;
  b.t += 1;
  return cuda_error(cudaGetLastError(), "batch step");
}

}  // namespace dpf

using namespace dpf;

extern "C" {

dpf_status dpf_batch_create(const dpf_model_desc* const* models, const int32_t* d1,
                            const int64_t* N, const int32_t* M, int32_t L, const uint64_t* seeds,
                            int32_t F, void* stream, dpf_batch** out) {
  clear_error();
  if (!models || !d1 || !N || !M || !seeds || !out || F < 1)
    return set_error(DPF_E_INVALID, "dpf_batch_create: bad arguments");
  *out = nullptr;
  dpf_batch* b = new dpf_batch();
  b->F = F;
  b->stream = (cudaStream_t)stream;
  b->d = models[0]->d;
  b->dy = models[0]->dy;
  b->prec = models[0]->precision;
  b->s = b->prec == DPF_F64 ? 8 : 4;
  auto fail = [&](dpf_status st) {
    std::string msg = dpf_last_error();
    dpf_batch_destroy(b);
    return set_error(st, msg);
  };
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess)
    return fail(cuda_error(cudaGetLastError(), "dpf_batch_create: event"));
  for (int q = 0; q < BATCH_AUX_STREAMS; ++q) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
      return fail(cuda_error(cudaGetLastError(), "dpf_batch_create: stream"));
    b->aux.push_back(s);
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return fail(cuda_error(cudaGetLastError(), "dpf_batch_create: event"));
    b->join_ev.push_back(e);
  }
  for (int f = 0; f < F; ++f) {
    if (!models[f] || models[f]->d != b->d || models[f]->dy != b->dy || models[f]->precision != b->prec)
      return fail(set_error(DPF_E_INVALID, "dpf_batch_create: all filters need the same d, dy and precision"));
    dpf_ctx* x = nullptr;
    dpf_status st = dpf_create(models[f], d1[f], models[f]->d - d1[f], N[f], M[f], L, seeds[f], stream, &x);
    if (st) return fail(st);
    b->ctx.push_back(x);
    if (!x->var->batch_launch && !x->var->single_launch)
      return fail(set_error(DPF_E_UNSUPPORTED, "dpf_batch_create: this (d1, d2, dy) variant has no batched form"));
    const size_t sz = b->s;
    const int ppl = x->var->ppl_for(M[f]);
    if (!(M[f] <= 256 && M[f] % ppl == 0 && (M[f] * sz) % 16 == 0 && (L * sz) % 16 == 0 &&
          (L * d1[f] * sz) % 16 == 0))
      return fail(set_error(DPF_E_UNSUPPORTED,
                            "dpf_batch_create: each M must be <= 256 with 16-byte rows (and L rows too)"));
  }
  // classes: (variant, x-kind, PPL, M = 32 PPL): a filter steps with the same compiled
  // kernel as when it runs alone, so a member reproduces the single filter bit for bit
  std::map<std::tuple<const Variant*, bool, int, bool>, int> key2cls;
  for (int f = 0; f < F; ++f) {
    dpf_ctx* x = b->ctx[f];
    const bool xz = x->var->use_xz(*x);
    const int ppl = x->var->ppl_for(x->M);
    const auto k = std::make_tuple(x->var, xz, ppl, x->M == 32 * ppl);
    auto it = key2cls.find(k);
    if (it == key2cls.end()) {
      BatchClass c;
      c.var = x->var;
      c.xz = xz;
      c.ppl = std::get<2>(k);
      b->cls.push_back(c);
      it = key2cls.emplace(k, (int)b->cls.size() - 1).first;
    }
    b->cls[it->second].members.push_back(f);
  }
  for (BatchClass& c : b->cls) {
    c.fstart.assign(1, 0);
    for (int f : c.members) c.fstart.push_back(c.fstart.back() + b->ctx[f]->N);
    const size_t nf = c.members.size();
    if (balloc(*b, (void**)&c.d_fstart, sizeof(long long) * (nf + 1)) ||
        balloc(*b, &c.d_mcs, c.var->const_size * nf))
      return fail(DPF_E_NOMEM);
    c.desc_bytes = c.var->args_size * nf;
    c.ring = 2;
    if (balloc(*b, &c.d_descs, c.desc_bytes * c.ring)) return fail(DPF_E_NOMEM);
    std::vector<unsigned char> mcs(c.var->const_size * nf);
    for (size_t q = 0; q < nf; ++q)
      memcpy(mcs.data() + q * c.var->const_size, b->ctx[c.members[q]]->mconst.data(), c.var->const_size);
    bool same = true;
    for (size_t q = 1; q < nf; ++q)
      same &= memcmp(mcs.data(), mcs.data() + q * c.var->const_size, c.var->const_size) == 0;
    if (same) c.shared_mc.assign(mcs.begin(), mcs.begin() + c.var->const_size);
    cudaMemcpy(c.d_fstart, c.fstart.data(), sizeof(long long) * (nf + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(c.d_mcs, mcs.data(), mcs.size(), cudaMemcpyHostToDevice);
    dpf_status st = shape_class(*b, c);
    if (st) return fail(st);
  }
  if (balloc(*b, &b->yhist, 2 * (size_t)F * b->dy * b->s)) return fail(DPF_E_NOMEM);
  // outer groups: one per variant
  std::map<const Variant*, int> var2g;
  for (int f = 0; f < F; ++f) {
    auto it = var2g.find(b->ctx[f]->var);
    if (it == var2g.end()) {
      OuterGroup g;
      g.var = b->ctx[f]->var;
      b->og.push_back(g);
      it = var2g.emplace(b->ctx[f]->var, (int)b->og.size() - 1).first;
    }
    b->og[it->second].members.push_back(f);
  }
  b->oring = 2;
  for (OuterGroup& g : b->og) {
    std::vector<int> bs(1, 0);
    for (int f : g.members) bs.push_back(bs.back() + g.var->outer_ctas(b->ctx[f]->N));
    g.nblocks = bs.back();
    g.set_bytes = g.var->oargs_size * g.members.size();
    if (balloc(*b, (void**)&g.d_bstart, sizeof(int) * bs.size()) ||
        balloc(*b, &g.d_oargs, g.set_bytes * b->oring))
      return fail(DPF_E_NOMEM);
    cudaMemcpy(g.d_bstart, bs.data(), sizeof(int) * bs.size(), cudaMemcpyHostToDevice);
    g.cur = g.d_oargs;
  }
  std::vector<int> ts(1, 0);
  for (int f = 0; f < F; ++f) {
    const long long ctas = b->ctx[f]->var->outer_ctas(b->ctx[f]->N);
    if (ts.back() + ctas > (long long)INT32_MAX)
      return fail(set_error(DPF_E_UNSUPPORTED, "dpf_batch_create: too many outer particles in all"));
    ts.push_back(ts.back() + (int)ctas);
  }
  b->ntiles = ts.back();
  b->gset_bytes = b->og[0].var->oargs_size * (size_t)F;
  if (balloc(*b, (void**)&b->d_tstart, sizeof(int) * ts.size()) ||
      balloc(*b, &b->d_gargs, b->gset_bytes * b->oring))
    return fail(DPF_E_NOMEM);
  cudaMemcpy(b->d_tstart, ts.data(), sizeof(int) * ts.size(), cudaMemcpyHostToDevice);
  b->gcur = b->d_gargs;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return fail(cuda_error(e, "dpf_batch_create"));
  *out = b;
  return DPF_OK;
}

dpf_status dpf_batch_step(dpf_batch* b, const void* y_dev, double* means_dev, double* logz_dev) {
  clear_error();
  if (!b || !y_dev) return set_error(DPF_E_INVALID, "dpf_batch_step: null argument");
  const long long t = b->t + 1;
  const size_t rows = (size_t)b->F * b->dy * b->s;
  char* cur = (char*)b->yhist + (t % 2) * rows;
  char* prev = (char*)b->yhist + ((t + 1) % 2) * rows;
  cudaError_t e = cudaMemcpyAsync(cur, y_dev, rows, cudaMemcpyDeviceToDevice, b->stream);
  if (e != cudaSuccess) return cuda_error(e, "dpf_batch_step: y copy");
  dpf_status st = upload_descs(*b, prev, cur, (int)(t % 2), b->stream);
  if (st) return st;
  std::vector<std::vector<unsigned char>> oh;
  std::vector<unsigned char> gh;
  outer_host_sets(*b, 1, oh, gh);
  fill_outer(*b, means_dev, logz_dev, oh, gh, 0);
  st = upload_outer(*b, oh, gh, (int)(t % 2), 1, b->stream);
  if (st) return st;
  return step_launch(*b);
}

dpf_status dpf_batch_run(dpf_batch* b, const void* ys_dev, int64_t T, double* means_dev,
                         double* logz_dev, int32_t use_graph) {
  clear_error();
  if (!b || !ys_dev || T < 1) return set_error(DPF_E_INVALID, "dpf_batch_run: bad arguments");
  const size_t rows = (size_t)b->F * b->dy * b->s;
  // every step's descriptors are prepared on the device before the run, so the
  // captured graph holds only kernels (ring of T sets)
  for (BatchClass& c : b->cls) {
    if (c.ring < T) {
      void* p = nullptr;
      if (balloc(*b, &p, c.desc_bytes * (size_t)T)) return set_error(DPF_E_NOMEM, "dpf_batch_run");
      c.d_descs = p;
      c.ring = (int)T;
    }
  }
  if (b->oring < T) {
    for (OuterGroup& g : b->og)
      if (balloc(*b, &g.d_oargs, g.set_bytes * (size_t)T)) return set_error(DPF_E_NOMEM, "dpf_batch_run");
    if (balloc(*b, &b->d_gargs, b->gset_bytes * (size_t)T)) return set_error(DPF_E_NOMEM, "dpf_batch_run");
    b->oring = (int)T;
  }
  const long long t0 = b->t;
  std::vector<long long> ctx_t(b->F);
  for (int f = 0; f < b->F; ++f) ctx_t[f] = b->ctx[f]->t;
  // descriptors: build them step by step with the host-side counters advanced as the run will
  std::vector<std::vector<unsigned char>> sets(b->cls.size());
  for (size_t ci = 0; ci < b->cls.size(); ++ci) sets[ci].resize(b->cls[ci].desc_bytes * (size_t)T);
  std::vector<std::vector<unsigned char>> oh;
  std::vector<unsigned char> gh;
  outer_host_sets(*b, (size_t)T, oh, gh);
  for (long long k = 0; k < T; ++k) {
    const long long t = t0 + k + 1;
    const char* cur = (const char*)ys_dev + (size_t)k * rows;
    const char* prev = k > 0 ? (const char*)ys_dev + (size_t)(k - 1) * rows
                             : (const char*)b->yhist + ((t + 1) % 2) * rows;
    for (size_t ci = 0; ci < b->cls.size(); ++ci) {
      BatchClass& c = b->cls[ci];
      for (size_t q = 0; q < c.members.size(); ++q) {
        const int f = c.members[q];
        c.var->batch_args(*b->ctx[f], prev + (size_t)f * b->dy * b->s, cur + (size_t)f * b->dy * b->s,
                          c.xz, sets[ci].data() + (size_t)k * c.desc_bytes + q * c.var->args_size);
      }
    }
    fill_outer(*b, means_dev ? means_dev + (size_t)k * b->F * b->d : nullptr,
               logz_dev ? logz_dev + (size_t)k * b->F : nullptr, oh, gh, (size_t)k);
    for (int f = 0; f < b->F; ++f) b->ctx[f]->t += 1;
  }
  for (int f = 0; f < b->F; ++f) b->ctx[f]->t = ctx_t[f];
  {
    dpf_status so = upload_outer(*b, oh, gh, 0, (size_t)T, b->stream);
    if (so) return so;
  }
  for (size_t ci = 0; ci < b->cls.size(); ++ci) {
    cudaError_t e = cudaMemcpyAsync(b->cls[ci].d_descs, sets[ci].data(), sets[ci].size(),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return cuda_error(e, "dpf_batch_run: descriptors");
  }
  // capture on a private stream (the legacy default stream cannot be captured),
  // ordered after the batch stream's pending work and before its later work
  cudaGraph_t graph = nullptr;
  cudaStream_t user = b->stream, cap = nullptr;
  if (use_graph) {
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamSynchronize(user);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      if (cap) cudaStreamDestroy(cap);
      return cuda_error(e, "dpf_batch_run: begin capture");
    }
    b->stream = cap;
  }
  dpf_status st = DPF_OK;
  for (long long k = 0; k < T && !st; ++k) {
    for (size_t ci = 0; ci < b->cls.size(); ++ci) {
      BatchClass& c = b->cls[ci];
      c.launch.descs = (char*)c.d_descs + (size_t)k * c.desc_bytes;
      c.host_cur = sets[ci].data() + (size_t)k * c.desc_bytes;
    }
    for (OuterGroup& g : b->og) g.cur = (const char*)g.d_oargs + (size_t)k * g.set_bytes;
    b->gcur = (const char*)b->d_gargs + (size_t)k * b->gset_bytes;
    st = step_launch(*b);
  }
  // the last observation becomes y_{t-1} of a later dpf_batch_step
  if (!st) {
    cudaError_t e = cudaMemcpyAsync((char*)b->yhist + ((t0 + T) % 2) * rows,
                                    (const char*)ys_dev + (size_t)(T - 1) * rows, rows,
                                    cudaMemcpyDeviceToDevice, b->stream);
    if (e != cudaSuccess) st = cuda_error(e, "dpf_batch_run: y history");
  }
  if (use_graph) {
    cudaError_t e = cudaStreamEndCapture(cap, &graph);
    b->stream = user;
    if (st || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaStreamDestroy(cap);
      return st ? st : cuda_error(e, "dpf_batch_run: end capture");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, cap);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cap);
    if (exec) cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return cuda_error(e, "dpf_batch_run: graph");
  }
  for (BatchClass& c : b->cls) {  // back to the two-set ring of dpf_batch_step
    c.launch.descs = c.d_descs;
    c.host_cur = nullptr;  // the next dpf_batch_step rebuilds its host copy
  }
  return st ? st : dpf_batch_sync(b);
}

dpf_status dpf_batch_sync(dpf_batch* b) {
  clear_error();
  if (!b) return set_error(DPF_E_INVALID, "dpf_batch_sync: null batch");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_error(e, "dpf_batch_sync");
  for (int f = 0; f < b->F; ++f) {
    dpf_status st = dpf_sync(b->ctx[f]);
    if (st) return st;
  }
  return DPF_OK;
}

dpf_status dpf_batch_autotune(dpf_batch* b, int32_t reps, char* report, size_t report_bytes) {
  clear_error();
  if (!b || reps < 1) return set_error(DPF_E_INVALID, "dpf_batch_autotune: bad arguments");
  if (b->t < 1)
    return set_error(DPF_E_INVALID,
                     "dpf_batch_autotune: step the batch once first (the first step has no inner update)");
  // candidates per class: the smallest inner-particles-per-lane that fits M, and twice
  // that (more instruction-level parallelism per lane, fewer lanes busy), each as one
  // launch for the class or (a class of several filters) one launch a filter; each is
  // timed on the live state with the next step's arguments, which only rewrites the
  // outputs the next real step rewrites anyway
  const long long t = b->t + 1;
  const size_t rows = (size_t)b->F * b->dy * b->s;
  char* cur = (char*)b->yhist + (t % 2) * rows;  // the candidate runs read whatever y is there
  char* prev = (char*)b->yhist + ((t + 1) % 2) * rows;
  dpf_status st = upload_descs(*b, prev, cur, (int)(t % 2), b->stream);
  if (st) return st;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::string rep = "{\"classes\": [";
  for (size_t ci = 0; ci < b->cls.size(); ++ci) {
    BatchClass& c = b->cls[ci];
    int maxM = 0;
    for (int f : c.members) maxM = std::max(maxM, b->ctx[f]->M);
    std::vector<int> cand = {c.var->ppl_for(maxM)};
    if (cand[0] * 2 <= 8 && c.var->batch_launch) {
      bool ok = true;
      for (int f : c.members) ok &= (b->ctx[f]->M % (cand[0] * 2) == 0);
      if (ok) cand.push_back(cand[0] * 2);
    }
    int best = c.ppl;
    bool best_split = false;
    double best_us = 1e300;
    std::string tried;
    for (int ppl : cand) {
      const int split0 = c.var->batch_launch ? 0 : 1;  // no shared launch to try for the class
      for (int split = split0; split < (c.var->batch_launch && c.members.size() > 1 ? 2 : 1) + split0 && !st; ++split) {
        c.ppl = ppl;
        c.split = split != 0;
        st = shape_class(*b, c);
        if (st) break;
        auto one = [&]() { return b->stream; };
        class_launch(*b, c, one);  // warm-up
        cudaEventRecord(e0, b->stream);
        for (int r = 0; r < reps; ++r) class_launch(*b, c, one);
        cudaEventRecord(e1, b->stream);
        cudaError_t ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) {
          st = cuda_error(ce, "dpf_batch_autotune");
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double us = ms * 1e3 / reps;
        tried += (tried.empty() ? "" : ", ") + std::string("{\"ppl\": ") + std::to_string(ppl) +
                 ", \"split\": " + (c.split ? "true" : "false") + ", \"us\": " + std::to_string(us) + "}";
        if (us < best_us) {
          best_us = us;
          best = ppl;
          best_split = c.split;
        }
      }
    }
    if (st) break;
    c.ppl = best;
    c.split = best_split;
    c.tuned_us = best_us;
    st = shape_class(*b, c);
    if (st) break;
    rep += (ci ? ", " : "") + std::string("{\"d1\": ") + std::to_string(c.var->d1) +
           ", \"d2\": " + std::to_string(c.var->d2) + ", \"xz\": " + (c.xz ? "true" : "false") +
           ", \"filters\": " + std::to_string(c.members.size()) + ", \"groups\": " +
           std::to_string(c.fstart.back()) + ", \"chosen_ppl\": " + std::to_string(c.ppl) +
           ", \"split\": " + (c.split ? "true" : "false") +
           ", \"grid\": " + std::to_string(c.launch.grid) + ", \"chunk\": " +
           std::to_string(c.launch.chunk) + ", \"tried\": [" + tried + "]}";
  }
  rep += "]}";
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  for (BatchClass& c : b->cls) c.launch.descs = c.d_descs;
  if (report && report_bytes) {
    const size_t n = std::min(report_bytes - 1, rep.size());
    memcpy(report, rep.data(), n);
    report[n] = 0;
  }
  return DPF_OK;
}

dpf_status dpf_batch_set_split(dpf_batch* b, int32_t split) {
  clear_error();
  if (!b) return set_error(DPF_E_INVALID, "dpf_batch_set_split: null batch");
  cudaError_t e = cudaStreamSynchronize(b->stream);  // no launch in flight reads the shapes
  if (e != cudaSuccess) return cuda_error(e, "dpf_batch_set_split");
  for (BatchClass& c : b->cls) c.split = !c.var->batch_launch || (split != 0 && c.members.size() > 1);
  return DPF_OK;
}

dpf_status dpf_batch_filter(dpf_batch* b, int32_t f, dpf_ctx** out) {
  clear_error();
  if (!b || !out || f < 0 || f >= b->F) return set_error(DPF_E_INVALID, "dpf_batch_filter: bad index");
  *out = b->ctx[f];
  return DPF_OK;
}

dpf_status dpf_batch_profile(dpf_batch* b, int32_t enable) {
  clear_error();
  if (!b) return set_error(DPF_E_INVALID, "dpf_batch_profile: null batch");
  b->profiling = enable != 0;
  return DPF_OK;
}

dpf_status dpf_batch_profile_read(dpf_batch* b, double* ms, int64_t* launches) {
  clear_error();
  if (!b) return set_error(DPF_E_INVALID, "dpf_batch_profile_read: null batch");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_error(e, "dpf_batch_profile_read");
  double tot = 0.0;
  for (size_t q = 0; q + 1 < b->pev_used; q += 2) {
    float f = 0.f;
    if (cudaEventElapsedTime(&f, b->pev[q], b->pev[q + 1]) == cudaSuccess)
      tot += f;
    else
      cudaGetLastError();  // a pair that holds no time leaves no error behind
  }
  if (ms) *ms = tot;
  if (launches) *launches = (int64_t)(b->pev_used / 2);
  b->pev_used = 0;
  return DPF_OK;
}

void dpf_batch_destroy(dpf_batch* b) {
  if (!b) return;
  if (b->stream || !b->ctx.empty()) cudaStreamSynchronize(b->stream);
  for (cudaStream_t s : b->aux) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (cudaEvent_t e : b->join_ev) cudaEventDestroy(e);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  for (cudaEvent_t e : b->pev) cudaEventDestroy(e);
  for (dpf_ctx* x : b->ctx) dpf_destroy(x);
  for (void* p : b->allocs) cudaFree(p);
  delete b;
}

}  // extern "C"
