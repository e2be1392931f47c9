// Host side of the C ABI: model preparation (double precision), the filter
// context, step sequencing and the small utility entry points.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "dpf_common.cuh"
#include "dpf_internal.h"

namespace dpf {

static thread_local std::string g_err;

dpf_status set_error(dpf_status st, const std::string& msg) {
  g_err = msg;
  return st;
}
void clear_error() { g_err.clear(); }
dpf_status cuda_error(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return DPF_OK;
  cudaGetLastError();  // clear the runtime's last-error state so later calls start clean
  if (e == cudaErrorMemoryAllocation)
    return set_error(DPF_E_NOMEM, std::string(what) + ": " + cudaGetErrorString(e));
  return set_error(DPF_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

dpf_status err_word_status(int w, const char* what) {
  if (w & 2) return set_error(DPF_E_TIMEOUT, std::string(what) + ": a device wait timed out");
  if (w & 1) return set_error(DPF_E_NUMERIC, std::string(what) + ": no positive or a NaN weight");
  if (w) return set_error(DPF_E_CUDA, std::string(what) + ": device bounds check failed");
  return DPF_OK;
}

dpf_status scratch_alloc(Scratch& sc, long long tiles, cudaStream_t s) {
  const size_t head = 64;
  const size_t bytes = head + (size_t)tiles * (4 + 8 + 8) + 16;
  cudaError_t e = cudaMallocAsync(&sc.block, bytes, s);
  if (e != cudaSuccess) {
    sc.block = nullptr;
    return cuda_error(e, "scratch allocation");
  }
  e = cudaMemsetAsync(sc.block, 0, bytes, s);
  if (e != cudaSuccess) return cuda_error(e, "scratch memset");
  unsigned char* b = (unsigned char*)sc.block;
  sc.maxkey = (unsigned long long*)(b + 0);
  sc.C = (unsigned long long*)(b + 8);
  sc.scan.ticket = (unsigned long long*)(b + 16);
  sc.shift = (int*)(b + 24);
  sc.err = (int*)(b + 28);
  sc.scan.agg = (unsigned long long*)(b + head);
  sc.scan.incl = sc.scan.agg + tiles;
  sc.scan.flags = (uint32_t*)(sc.scan.incl + tiles);
  return DPF_OK;
}

void scratch_free(Scratch& sc, cudaStream_t s) {
  if (sc.block) cudaFreeAsync(sc.block, s);
  sc.block = nullptr;
}

dpf_status scratch_finish(Scratch& sc, cudaStream_t s, const char* what) {
  int w = 0;
  cudaError_t e = cudaMemcpyAsync(&w, sc.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  scratch_free(sc, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, what);
  return err_word_status(w, what);
}

// ---------------------------------------------------------------------------
// Small dense linear algebra in double (row-major), for the model constants.
// ---------------------------------------------------------------------------
static bool chol(const std::vector<double>& S, int n, std::vector<double>& Lo) {
  Lo.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = S[i * n + j];
      for (int k = 0; k < j; ++k) s -= Lo[i * n + k] * Lo[j * n + k];
      if (i == j) {
        if (!(s > 0.0)) return false;
        Lo[i * n + i] = std::sqrt(s);
      } else {
        Lo[i * n + j] = s / Lo[j * n + j];
      }
    }
  return true;
}
// Inverse of a lower-triangular matrix (column by column forward substitution).
static std::vector<double> tri_inv(const std::vector<double>& Lo, int n) {
  std::vector<double> X((size_t)n * n, 0.0);
  for (int c = 0; c < n; ++c)
    for (int i = c; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) s -= Lo[i * n + k] * X[k * n + c];
      X[i * n + c] = s / Lo[i * n + i];
    }
  return X;
}
static std::vector<double> matmul(const std::vector<double>& A, const std::vector<double>& B, int n,
                                  int k, int m) {
  std::vector<double> C((size_t)n * m, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int q = 0; q < k; ++q) s += A[i * k + q] * B[q * m + j];
      C[i * m + j] = s;
    }
  return C;
}
static std::vector<double> transpose(const std::vector<double>& A, int n, int m) {
  std::vector<double> T((size_t)n * m);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) T[j * n + i] = A[i * m + j];
  return T;
}
// S^{-1} for SPD S via its Cholesky factor: S^{-1} = Lo^{-T} Lo^{-1}.
static bool spd_inv(const std::vector<double>& S, int n, std::vector<double>& out) {
  std::vector<double> Lo;
  if (!chol(S, n, Lo)) return false;
  std::vector<double> Li = tri_inv(Lo, n);
  out = matmul(transpose(Li, n, n), Li, n, n, n);
  return true;
}
static std::vector<double> block(const std::vector<double>& A, int lda, int r0, int nr, int c0,
                                 int nc) {
  std::vector<double> B((size_t)nr * nc);
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nc; ++j) B[i * nc + j] = A[(r0 + i) * lda + c0 + j];
  return B;
}

static dpf_status prepare_model(const dpf_model_desc* m, int d1, int d2, std::vector<int>& perm,
                                HostModel& h) {
  const int d = m->d, dy = m->dy;
  if (m->kind != DPF_MODEL_CLG) return set_error(DPF_E_INVALID, "model kind must be DPF_MODEL_CLG");
  if (d < 2 || d1 < 1 || d2 < 1 || d1 + d2 != d || dy < 1 || d > 128 || dy > 64)
    return set_error(DPF_E_INVALID, "model dimensions out of range (d1 + d2 == d, all >= 1)");
  if (!m->A || !m->Q || !m->H || !m->R || !m->m0 || !m->P0)
    return set_error(DPF_E_INVALID, "model matrices must be non-null");
  if (m->quad_obs && dy != d1) return set_error(DPF_E_INVALID, "quad_obs needs dy == d1");
  perm.resize(d);
  std::vector<int> seen(d, 0);
  for (int c = 0; c < d; ++c) {
    perm[c] = m->perm ? m->perm[c] : c;
    if (perm[c] < 0 || perm[c] >= d || seen[perm[c]]++)
      return set_error(DPF_E_INVALID, "perm is not a permutation of 0..d-1");
  }
  std::vector<double> A(d * d), Q(d * d), H(dy * d), P0(d * d), m0(d), R(m->R, m->R + dy * dy);
  for (int r = 0; r < d; ++r) {
    m0[r] = m->m0[perm[r]];
    for (int c = 0; c < d; ++c) {
      A[r * d + c] = m->A[perm[r] * d + perm[c]];
      Q[r * d + c] = m->Q[perm[r] * d + perm[c]];
      P0[r * d + c] = m->P0[perm[r] * d + perm[c]];
    }
  }
  for (int q = 0; q < dy; ++q)
    for (int c = 0; c < d; ++c) H[q * d + c] = m->H[q * d + perm[c]];
  for (int r = 0; r < d1; ++r)
    for (int c = d1; c < d; ++c)
      if (Q[r * d + c] != 0.0 || Q[c * d + r] != 0.0)
        return set_error(DPF_E_INVALID, "Q must have no x/z cross-covariance");
  h.d1 = d1;
  h.d2 = d2;
  h.dy = dy;
  h.growth = m->growth_x ? 1 : 0;
  h.quad = m->quad_obs ? 1 : 0;
  h.ga = m->growth[0];
  h.gb = m->growth[1];
  h.gc = m->growth[2];
  h.gw = m->growth[3];
  h.qc = m->qc;
  h.Axx = block(A, d, 0, d1, 0, d1);
  h.Axz = block(A, d, 0, d1, d1, d2);
  h.Azx = block(A, d, d1, d2, 0, d1);
  h.Azz = block(A, d, d1, d2, d1, d2);
  h.Hx = block(H, d, 0, dy, 0, d1);
  h.Hz = block(H, d, 0, dy, d1, d2);
  std::vector<double> Qx = block(Q, d, 0, d1, 0, d1), Qz = block(Q, d, d1, d2, d1, d2), Lr;
  if (!chol(Qx, d1, h.Lqx) || !chol(Qz, d2, h.Lqz) || !chol(R, dy, Lr))
    return set_error(DPF_E_INVALID, "Q and R must be symmetric positive definite");
  h.LqxInv = tri_inv(h.Lqx, d1);
  h.LrInv = tri_inv(Lr, dy);
  h.lognorm_y = -0.5 * dy * std::log(2.0 * M_PI);
  for (int q = 0; q < dy; ++q) h.lognorm_y -= std::log(Lr[q * dy + q]);
  h.WAxz = matmul(h.LqxInv, h.Axz, d1, d1, d2);
  std::vector<double> QHt = matmul(Qz, transpose(h.Hz, dy, d2), d2, d2, dy);
  std::vector<double> S = matmul(h.Hz, QHt, dy, d2, dy), Sinv;
  if (!chol(S, dy, h.Ls) || !spd_inv(S, dy, Sinv))
    return set_error(DPF_E_INVALID, "H_z Q_z H_z^T must be positive definite");
  h.K = matmul(QHt, Sinv, d2, dy, dy);
  h.HzAzz = matmul(h.Hz, h.Azz, dy, d2, d2);
  h.HzAzx = matmul(h.Hz, h.Azx, dy, d2, d1);
  h.LrHz = matmul(h.LrInv, h.Hz, dy, dy, d2);
  h.m0x.assign(m0.begin(), m0.begin() + d1);
  h.m0z.assign(m0.begin() + d1, m0.end());
  std::vector<double> Pxx = block(P0, d, 0, d1, 0, d1), Pzx = block(P0, d, d1, d2, 0, d1),
                      Pxz = block(P0, d, 0, d1, d1, d2), Pzz = block(P0, d, d1, d2, d1, d2), Pxxi;
  if (!chol(Pxx, d1, h.Lp0x) || !spd_inv(Pxx, d1, Pxxi))
    return set_error(DPF_E_INVALID, "P0 must be symmetric positive definite");
  h.G0 = matmul(Pzx, Pxxi, d2, d1, d1);
  std::vector<double> GP = matmul(h.G0, Pxz, d2, d1, d2);
  for (size_t q = 0; q < Pzz.size(); ++q) Pzz[q] -= GP[q];
  if (!chol(Pzz, d2, h.Lp0c)) return set_error(DPF_E_INVALID, "P0 must be positive definite");
  h.xz = false;
  for (double v : h.Axz) h.xz |= (v != 0.0);
  return DPF_OK;
}

// Armed by dpf_fail_allocation_after: the count of device allocations still to
// succeed before one fails (0: nothing armed).
static std::atomic<long long> g_alloc_countdown{0};

cudaError_t device_malloc(void** p, size_t bytes) {
  long long c = g_alloc_countdown.load();
  while (c > 0 && !g_alloc_countdown.compare_exchange_weak(c, c - 1)) {
  }
  if (c == 1) {  // this call is the armed one
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

template <class P>
static dpf_status dalloc(Ctx& x, P*& p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = device_malloc(&q, bytes < 16 ? 16 : bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(DPF_E_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  x.allocs.push_back(q);
  x.bytes += bytes;
  p = (P*)q;
  return DPF_OK;
}

static void free_all(Ctx* x) {
  for (void* p : x->allocs) cudaFree(p);
  x->allocs.clear();
  if (x->hstats) cudaFreeHost(x->hstats);
  x->hstats = x->hstats_dev = nullptr;
  for (cudaEvent_t e : x->pev) cudaEventDestroy(e);
  x->pev.clear();
}

static dpf_status read_err(Ctx& x, const char* what) {
  int w = 0;
  cudaError_t e = cudaMemcpyAsync(&w, x.err, sizeof(int), cudaMemcpyDeviceToHost, x.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x.stream);
  if (e != cudaSuccess) return cuda_error(e, what);
  if (w) {
    cudaMemsetAsync(x.err, 0, sizeof(int), x.stream);
    return err_word_status(w, what);
  }
  return DPF_OK;
}

}  // namespace dpf

using namespace dpf;

extern "C" {

const char* dpf_last_error(void) { return g_err.c_str(); }

dpf_status dpf_create(const dpf_model_desc* model, int32_t d1, int32_t d2, int64_t N, int32_t M,
                      int32_t L, uint64_t seed, void* stream, dpf_ctx** out) {
  clear_error();
  if (!model || !out) return set_error(DPF_E_INVALID, "dpf_create: null argument");
  *out = nullptr;
  if (N < 1 || N >= (1ll << 31) || M < 1 || M > 1024 || L < 1 || L > 64)
    return set_error(DPF_E_INVALID, "dpf_create: need 1 <= N < 2^31, 1 <= M <= 1024, 1 <= L <= 64");
  if (model->precision != DPF_F32 && model->precision != DPF_F64)
    return set_error(DPF_E_INVALID, "dpf_create: precision must be DPF_F32 or DPF_F64");
  Ctx* x = new Ctx();
  x->prec = model->precision;
  x->d = model->d;
  x->d1 = d1;
  x->d2 = d2;
  x->dy = model->dy;
  x->N = N;
  x->M = M;
  x->L = L;
  x->seed = seed;
  x->stream = (cudaStream_t)stream;
  const bool paper = model->kind == DPF_MODEL_PAPER1 || model->kind == DPF_MODEL_PAPER2;
  dpf_status st = DPF_OK;
  bool swapped = false;
  if (paper) {  // the paper's models: fixed dimensions, FP32
    const int want_d = model->kind == DPF_MODEL_PAPER1 ? 2 : 4;
    if (model->d != want_d || model->dy != 1 || d1 != want_d / 2 || d2 != want_d / 2 || model->precision != DPF_F32) {
      delete x;
      return set_error(DPF_E_INVALID, "dpf_create: the paper's model 1 needs d = 2, model 2 d = 4, with dy = 1, "
                                      "d1 = d2 = d / 2 and FP32");
    }
    // the coordinate order: the table's, or for model 1 also (z, x) (perm = {1, 0})
    x->perm.resize(want_d);
    for (int c = 0; c < want_d; ++c) x->perm[c] = model->perm ? model->perm[c] : c;
    bool ident = true;
    for (int c = 0; c < want_d; ++c) ident = ident && x->perm[c] == c;
    swapped = !ident;
    if (swapped && !(model->kind == DPF_MODEL_PAPER1 && x->perm[0] == 1 && x->perm[1] == 0)) {
      delete x;
      return set_error(DPF_E_INVALID, "dpf_create: the paper's models take the table's coordinate order, "
                                      "or {1, 0} for model 1");
    }
    x->hm.d1 = d1;
    x->hm.d2 = d2;
    x->hm.dy = 1;
    x->hm.xz = true;
  } else {
    st = prepare_model(model, d1, d2, x->perm, x->hm);
  }
  if (st) {
    delete x;
    return st;
  }
  x->var = paper ? find_paper_variant(model->kind, swapped) : find_variant(x->prec, d1, d2, x->dy);
  x->model_id = paper ? model->kind + (swapped ? 2 : 0) : 0;
  if (!x->var) {
    delete x;
    return set_error(DPF_E_UNSUPPORTED,
                     "dpf_create: no compiled kernel for (precision, d1, d2, dy) = (" +
                         std::to_string(model->precision) + ", " + std::to_string(d1) + ", " +
                         std::to_string(d2) + ", " + std::to_string(model->dy) + ")");
  }
  if (x->hm.xz && !x->var->xz_supported) {
    delete x;
    return set_error(DPF_E_UNSUPPORTED,
                     "dpf_create: this (d1, d2, dy) variant serves only models whose x transition is free of z");
  }
  if (M > x->var->max_m) {
    const int mm = x->var->max_m;
    delete x;
    return set_error(DPF_E_UNSUPPORTED, "dpf_create: this (d1, d2, dy) variant accepts M <= " +
                                            std::to_string(mm));
  }
  x->ppt = M >= 64 ? 2 : 1;
  if (const char* e = getenv("DPF_PPT")) x->ppt = atoi(e) == 2 ? 2 : 1;
  const size_t sm = x->var->step_smem(M, L, x->hm.xz, ((M + x->ppt - 1) / x->ppt + 31) / 32 * 32);
  if (sm > 226 * 1024) {  // 227 KB of dynamic shared memory a block, less the static part
    delete x;
    return set_error(DPF_E_UNSUPPORTED, "dpf_create: M * L too large for the step's shared memory");
  }
  x->var->make_const(x->hm, x->mconst);
  x->xp = x->var->xpad();
  const size_t s = x->prec == DPF_F64 ? 8 : 4;
  const size_t NM = (size_t)N * M;
  const int d = x->d;
  const long long out_ctas = std::min<long long>((N + OF_CHUNK - 1) / OF_CHUNK, OF_MAX_CTAS);
  const size_t ssz = sizeof(double) * (4 + 2 * d);
  bool ok = true;
  for (int q = 0; q < 2 && ok; ++q) {
    ok &= !dalloc(*x, x->z[q], s * NM * d2);
    ok &= !dalloc(*x, x->lq[q], s * NM);
    ok &= !dalloc(*x, x->x[q], s * N * x->xp);
    ok &= !dalloc(*x, x->lwh[q], s * N * L);
    ok &= !dalloc(*x, x->xbb[q], s * N * L * d1);
  }
  ok = ok && !dalloc(*x, x->lw, s * N) && !dalloc(*x, x->xm, s * N * d1) &&
       !dalloc(*x, x->zm, s * N * d2) && !dalloc(*x, x->wout, s * N) &&
       !dalloc(*x, x->yb, s * 2 * x->dy) && !dalloc(*x, x->anc, 4 * N) && !dalloc(*x, x->sel, 4 * N) &&
       !dalloc(*x, x->stats, ssz) && !dalloc(*x, x->lwmax_t, 8) && !dalloc(*x, x->lwmax_key, 8) &&
       !dalloc(*x, x->Csum, 8) && !dalloc(*x, x->done, 8) && !dalloc(*x, x->err, 8) &&
       !dalloc(*x, x->partials, sizeof(double) * out_ctas * (4 + d)) &&
       !dalloc(*x, x->ctot, sizeof(unsigned long long) * out_ctas);
  if (!ok) {
    std::string msg = g_err;
    free_all(x);
    delete x;
    return set_error(DPF_E_NOMEM, "dpf_create: " + msg);
  }
  // the host mirror of the statistics (pinned and mapped; without it dpf_step copies them)
  if (cudaHostAlloc((void**)&x->hstats, sizeof(double) * (5 + d), cudaHostAllocMapped) == cudaSuccess) {
    if (cudaHostGetDevicePointer((void**)&x->hstats_dev, x->hstats, 0) != cudaSuccess) {
      cudaFreeHost(x->hstats);
      x->hstats = x->hstats_dev = nullptr;
    }
  } else {
    x->hstats = nullptr;
  }
  cudaGetLastError();  // a failed pinned allocation only disables the mirror
  cudaStream_t sr = x->stream;
  cudaMemsetAsync(x->stats, 0, ssz, sr);
  cudaMemcpyAsync((int*)(x->stats + 4 + d), x->perm.data(), sizeof(int) * d, cudaMemcpyHostToDevice, sr);
  cudaMemsetAsync(x->lwmax_key, 0, 8, sr);
  cudaMemsetAsync(x->Csum, 0, 8, sr);
  cudaMemsetAsync(x->done, 0, 8, sr);
  cudaMemsetAsync(x->err, 0, 8, sr);
  cudaMemsetAsync(x->anc, 0, 4 * N, sr);
  cudaMemsetAsync(x->sel, 0, 4 * N, sr);
  st = x->var->init(*x);
  if (!st) st = read_err(*x, "dpf_create");
  if (st) {
    std::string msg = g_err;
    free_all(x);
    delete x;
    return set_error(st, msg);
  }
  *out = x;
  return DPF_OK;
}

dpf_status dpf_create_pf(const dpf_model_desc* model, int32_t d1, int32_t d2, int64_t N, uint64_t seed,
                         void* stream, dpf_ctx** out) {
  clear_error();
  dpf_status st = dpf_create(model, d1, d2, N, 1, 1, seed, stream, out);
  if (st) return st;
  if (!(*out)->var->pf_step) {
    dpf_destroy(*out);
    *out = nullptr;
    return set_error(DPF_E_UNSUPPORTED, "dpf_create_pf: this (d1, d2, dy) variant has no particle-filter step");
  }
  (*out)->pf = true;
  return DPF_OK;
}

dpf_status dpf_create_std(const dpf_model_desc* model, int32_t d1, int32_t d2, int64_t N, int32_t M,
                          uint64_t seed, void* stream, dpf_ctx** out) {
  clear_error();
  dpf_status st = dpf_create(model, d1, d2, N, M, 1, seed, stream, out);
  if (st) return st;
  if (!(*out)->var->std_step) {
    dpf_destroy(*out);
    *out = nullptr;
    return set_error(DPF_E_UNSUPPORTED, "dpf_create_std: this (d1, d2, dy) variant has no DPF step");
  }
  (*out)->std_dpf = true;
  return DPF_OK;
}

dpf_status dpf_set_gaussian_approx(dpf_ctx* x, int32_t on) {
  clear_error();
  if (!x || !x->std_dpf)
    return set_error(DPF_E_INVALID, "dpf_set_gaussian_approx: needs a context from dpf_create_std");
  x->std_gauss = on != 0;
  return DPF_OK;
}

static dpf_status step_enqueue(dpf_ctx* x, double* mean_out, double* logz_out) {
  const long long t = x->t + 1;
  if (x->profiling) {
    if (x->pev_used + 2 > x->pev.size()) {
      for (int q = 0; q < 64; ++q) {
        cudaEvent_t ev;
        if (cudaEventCreate(&ev) != cudaSuccess) return cuda_error(cudaGetLastError(), "event");
        x->pev.push_back(ev);
      }
    }
    cudaEventRecord(x->pev[x->pev_used], x->stream);
  }
  dpf_status st = DPF_OK;
  if (x->pf || x->std_dpf) {  // bootstrap PF or DPF: their step, then the shared outer stages
    st = x->pf ? x->var->pf_step(*x) : x->var->std_step(*x);
    if (!st) st = x->var->outer(*x, mean_out, logz_out, x->stream);
    if (st) return st;
    x->t = t;
    return DPF_OK;
  }
  if (x->debug && x->anc_prev && t >= 2)  // the ancestors this call's inner update reads
    cudaMemcpyAsync(x->anc_prev, x->anc, sizeof(int32_t) * x->N, cudaMemcpyDeviceToDevice, x->stream);
  if (x->proposal && t >= 2) {
    // learned proposal: its inner update; groups whose inner ESS fell below
    // fb_frac * M redo it with the plain rule (and their look-ahead); the look-ahead
    // of the other groups then runs alone from the materialised state
    st = learned_inner_step(*x);
    const bool fallback = x->fb_frac > 0.0;
    if (!st) st = learned_fallback_lists(*x);
    if (!st && fallback) {
      x->glist_cur = x->fb_list;
      x->gcount_cur = x->fb_count;
      st = x->var->step(*x, 0);
      x->glist_cur = x->gcount_cur = nullptr;
      x->gskip_cur = x->fb_flag;
    }
    if (!st) {
      x->la_only = true;
      st = x->var->step(*x, 0);
      x->la_only = false;
    }
    x->glist_cur = x->gcount_cur = x->gskip_cur = nullptr;
  } else {
    st = x->var->step(*x, 0);
  }
  if (st) return st;
  if (x->profiling) {
    cudaEventRecord(x->pev[x->pev_used + 1], x->stream);
    x->pev_used += 2;
  }
  st = x->var->outer(*x, mean_out, logz_out, x->stream);
  if (st) return st;
  x->t = t;
  return DPF_OK;
}

dpf_status dpf_step_async(dpf_ctx* x, const void* y_dev, double* mean_out, double* logz_out) {
  clear_error();
  if (!x || !y_dev) return set_error(DPF_E_INVALID, "dpf_step_async: null argument");
  const size_t s = x->prec == DPF_F64 ? 8 : 4;
  const long long t = x->t + 1;
  cudaError_t e = cudaMemcpyAsync((char*)x->yb + (t % 2) * x->dy * s, y_dev, x->dy * s,
                                  cudaMemcpyDeviceToDevice, x->stream);
  if (e != cudaSuccess) return cuda_error(e, "dpf_step_async: y copy");
  return step_enqueue(x, mean_out, logz_out);
}

dpf_status dpf_step(dpf_ctx* x, const void* y_t, int32_t y_on_device, double* out_mean,
                    double* out_logZ) {
  clear_error();
  if (!x || !y_t) return set_error(DPF_E_INVALID, "dpf_step: null argument");
  const size_t s = x->prec == DPF_F64 ? 8 : 4;
  const long long t = x->t + 1;
  void* slot = (char*)x->yb + (t % 2) * x->dy * s;
  cudaError_t e = cudaMemcpyAsync(slot, y_t, x->dy * s,
                                  y_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  x->stream);
  if (e != cudaSuccess) return cuda_error(e, "dpf_step: y copy");
  const bool outs = out_mean || out_logZ;
  x->host_out = outs && x->hstats;
  dpf_status st = step_enqueue(x, nullptr, nullptr);
  const bool mirrored = x->host_out;
  x->host_out = false;
  if (st) return st;
  if (!outs) return DPF_OK;
  if (mirrored) {  // the outer stage wrote the statistics and the error word to the mirror
    e = cudaStreamSynchronize(x->stream);
    if (e != cudaSuccess) return cuda_error(e, "dpf_step");
    const volatile double* hs = x->hstats;
    if (hs[4 + x->d] != 0.0) return read_err(*x, "dpf_step");  // reads and clears the word
    if (out_mean)
      for (int c = 0; c < x->d; ++c) out_mean[c] = hs[4 + c];
    if (out_logZ) *out_logZ = hs[0];
    return DPF_OK;
  }
  std::vector<double> h(4 + x->d);
  e = cudaMemcpyAsync(h.data(), x->stats, sizeof(double) * (4 + x->d), cudaMemcpyDeviceToHost,
                      x->stream);
  if (e != cudaSuccess) return cuda_error(e, "dpf_step: output copy");
  st = read_err(*x, "dpf_step");
  if (st) return st;
  if (out_mean) memcpy(out_mean, h.data() + 4, sizeof(double) * x->d);
  if (out_logZ) *out_logZ = h[0];
  return DPF_OK;
}

dpf_status dpf_sync(dpf_ctx* x) {
  clear_error();
  if (!x) return set_error(DPF_E_INVALID, "dpf_sync: null context");
  return read_err(*x, "dpf_sync");
}

dpf_status dpf_diag(dpf_ctx* x, double* ess, int64_t* step, double* logz_step) {
  clear_error();
  if (!x) return set_error(DPF_E_INVALID, "dpf_diag: null context");
  double h[4];
  cudaError_t e = cudaMemcpyAsync(h, x->stats, sizeof(h), cudaMemcpyDeviceToHost, x->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  if (e != cudaSuccess) return cuda_error(e, "dpf_diag");
  if (ess) *ess = h[2];
  if (step) *step = x->t;
  if (logz_step) *logz_step = h[1];
  return DPF_OK;
}

}  // extern "C"

// Inner effective sample size of each group of the materialised state,
// (sum_j W_j)^2 / sum_j W_j^2 with W = exp(lq), one warp a group; the sum over the
// groups and their minimum (positive doubles order as their bit patterns) accumulate
// in acc[0] and acc[1].
template <typename T>
__global__ void inner_ess_kernel(const T* __restrict__ lq, long long N, int M, double* acc) {
  __shared__ double s_sum[8];
  __shared__ unsigned long long s_min[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long i = (long long)blockIdx.x * (blockDim.x >> 5) + w;
  double ess = 0.0;
  unsigned long long key = ~0ull;
  if (i < N) {
    double s1 = 0.0, s2 = 0.0;
    for (int k = lane; k < M; k += 32) {
      const double v = exp((double)lq[i * M + k]);
      s1 += v;
      s2 += v * v;
    }
    s1 = dpf::warp_sum(s1);
    s2 = dpf::warp_sum(s2);
    ess = s2 > 0.0 ? s1 * s1 / s2 : 0.0;
    key = (unsigned long long)__double_as_longlong(ess);
  }
  if (lane == 0) {
    s_sum[w] = ess;
    s_min[w] = key;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    unsigned long long m = ~0ull;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      t += s_sum[q];
      m = s_min[q] < m ? s_min[q] : m;
    }
    atomicAdd(&acc[0], t);
    atomicMin(reinterpret_cast<unsigned long long*>(&acc[1]), m);
  }
}

extern "C" {

dpf_status dpf_diag_inner(dpf_ctx* x, double* ess_min, double* ess_mean) {
  clear_error();
  if (!x || !ess_min || !ess_mean) return set_error(DPF_E_INVALID, "dpf_diag_inner: null argument");
  if (!x->diag_inner) {
    dpf_status st = dalloc(*x, x->diag_inner, sizeof(double) * 2);
    if (st) return st;
  }
  const long long t = x->t;
  const int mat = t >= 2 ? (int)((t - 1) % 2) : 0;
  const double init[2] = {0.0, __builtin_bit_cast(double, ~0ull)};
  cudaError_t e = cudaMemcpyAsync(x->diag_inner, init, sizeof(init), cudaMemcpyHostToDevice, x->stream);
  if (e != cudaSuccess) return cuda_error(e, "dpf_diag_inner");
  const unsigned blocks = (unsigned)((x->N + 7) / 8);
  if (x->prec == DPF_F64)
    inner_ess_kernel<double><<<blocks, 256, 0, x->stream>>>((const double*)x->lq[mat], x->N, x->M, x->diag_inner);
  else
    inner_ess_kernel<float><<<blocks, 256, 0, x->stream>>>((const float*)x->lq[mat], x->N, x->M, x->diag_inner);
  double h[2];
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, x->diag_inner, sizeof(h), cudaMemcpyDeviceToHost, x->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  if (e != cudaSuccess) return cuda_error(e, "dpf_diag_inner");
  *ess_mean = h[0] / (double)x->N;
  *ess_min = h[1];
  return DPF_OK;
}

// ---- checkpoints: everything the next step reads ----
namespace {
struct StateHeader {
  uint64_t magic;
  int32_t version, prec, d1, d2, dy, M, L, xp;
  int64_t N, t;
  uint64_t seed;
  int32_t kind;   // 0 the LA-DPF, 1 the bootstrap particle filter, 2 the DPF without look-ahead
  int32_t model;  // 0 a conditionally linear-Gaussian model; the paper's: 2 model 1, 3 model 2,
                  // 4 model 1 decomposed the other way (states written before it hold 0)
};
int32_t ctx_kind(const dpf_ctx& x) { return x.pf ? 1 : (x.std_dpf ? 2 : 0); }
constexpr uint64_t kStateMagic = 0x4450465354415445ull;  // "DPFSTATE"
struct StateLayout {
  size_t off[10];
  size_t len[10];
  size_t total;
};
StateLayout state_layout(const dpf_ctx& x) {
  const size_t s = x.prec == DPF_F64 ? 8 : 4;
  const size_t N = (size_t)x.N, M = (size_t)x.M, L = (size_t)x.L;
  const size_t len[10] = {sizeof(StateHeader), s * N * x.xp, s * N * M * x.d2, s * N * M, s * N * L,
                          s * N * L * x.d1, 4 * N, s * 2 * x.dy, sizeof(double) * (4 + x.d), 4 * N};
  StateLayout l{};
  size_t o = 0;
  for (int q = 0; q < 10; ++q) {
    l.off[q] = o;
    l.len[q] = len[q];
    o += (len[q] + 255) / 256 * 256;
  }
  l.total = o;
  return l;
}
// the device arrays of the sections (header excluded), in layout order
void state_arrays(dpf_ctx& x, void* a[10]) {
  const long long t = x.t;
  const int cur = (int)(t % 2);
  // the state the next step reads: the LA-DPF's materialised slot, the others' newest one
  const int mat = (x.pf || x.std_dpf) ? cur : (t >= 2 ? (int)((t - 1) % 2) : 0);
  a[0] = nullptr;
  a[1] = x.x[mat];
  a[2] = x.z[mat];
  a[3] = x.lq[mat];
  a[4] = x.lwh[cur];
  a[5] = x.xbb[cur];
  a[6] = x.anc;
  a[7] = x.yb;
  a[8] = x.stats;
  a[9] = x.sel;
}
}  // namespace

dpf_status dpf_state_bytes(dpf_ctx* x, size_t* bytes) {
  clear_error();
  if (!x || !bytes) return set_error(DPF_E_INVALID, "dpf_state_bytes: null argument");
  *bytes = state_layout(*x).total;
  return DPF_OK;
}

dpf_status dpf_get_state(dpf_ctx* x, void* dst, size_t bytes) {
  clear_error();
  if (!x || !dst) return set_error(DPF_E_INVALID, "dpf_get_state: null argument");
  const StateLayout l = state_layout(*x);
  if (bytes < l.total) return set_error(DPF_E_INVALID, "dpf_get_state: buffer smaller than dpf_state_bytes");
  StateHeader h{kStateMagic, 2, x->prec, x->d1, x->d2, x->dy, x->M, x->L, x->xp, x->N, x->t, x->seed,
                ctx_kind(*x), x->model_id};
  void* a[10];
  state_arrays(*x, a);
  cudaError_t e = cudaMemcpyAsync(dst, &h, sizeof(h), cudaMemcpyHostToDevice, x->stream);
  for (int q = 1; q < 10 && e == cudaSuccess; ++q)
    e = cudaMemcpyAsync((char*)dst + l.off[q], a[q], l.len[q], cudaMemcpyDeviceToDevice, x->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);  // h lives on this stack frame
  return cuda_error(e, "dpf_get_state");
}

dpf_status dpf_set_state(dpf_ctx* x, const void* src, size_t bytes) {
  clear_error();
  if (!x || !src) return set_error(DPF_E_INVALID, "dpf_set_state: null argument");
  const StateLayout l = state_layout(*x);
  if (bytes < l.total) return set_error(DPF_E_INVALID, "dpf_set_state: buffer smaller than dpf_state_bytes");
  StateHeader h{};
  cudaError_t e = cudaMemcpyAsync(&h, src, sizeof(h), cudaMemcpyDeviceToHost, x->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  if (e != cudaSuccess) return cuda_error(e, "dpf_set_state");
  if (h.magic != kStateMagic || h.version != 2 || h.prec != x->prec || h.d1 != x->d1 || h.d2 != x->d2 ||
      h.dy != x->dy || h.M != x->M || h.L != x->L || h.xp != x->xp || h.N != x->N || h.t < 0 ||
      h.kind != ctx_kind(*x) || h.model != x->model_id)
    return set_error(DPF_E_INVALID, "dpf_set_state: not a state of a filter of this kind, model, precision and "
                                    "these sizes");
  x->t = h.t;
  void* a[10];
  state_arrays(*x, a);
  for (int q = 1; q < 10 && e == cudaSuccess; ++q)
    e = cudaMemcpyAsync(a[q], (const char*)src + l.off[q], l.len[q], cudaMemcpyDeviceToDevice, x->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  return cuda_error(e, "dpf_set_state");
}

dpf_status dpf_read(dpf_ctx* x, const char* which, void* dst, size_t bytes) {
  clear_error();
  if (!x || !which || !dst) return set_error(DPF_E_INVALID, "dpf_read: null argument");
  const size_t s = x->prec == DPF_F64 ? 8 : 4;
  const long long N = x->N, M = x->M, L = x->L;
  const long long t = x->t;
  const int cur = (int)(t % 2);                   // look-ahead products of step t
  // newest materialised state (the particle filter's particles of step t)
  const int mat = (x->pf || x->std_dpf) ? cur : (t >= 2 ? (int)((t - 1) % 2) : 0);
  const void* src = nullptr;
  size_t need = 0;
  std::string w(which);
  if (w == "lw") { src = x->lw; need = s * N; }
  else if (w == "lwhat") { src = x->lwh[cur]; need = s * N * L; }
  else if (w == "xbb") { src = x->xbb[cur]; need = s * N * L * x->d1; }
  else if (w == "anc") { src = x->anc; need = 4 * N; }
  else if (w == "sel") { src = x->sel; need = 4 * N; }
  else if (w == "wout") { src = x->wout; need = s * N; }
  else if (w == "xm") { src = x->xm; need = s * N * x->d1; }
  else if (w == "zm") { src = x->zm; need = s * N * x->d2; }
  else if (w == "x") {  // rows are padded to xp elements on the device; returned packed
    if (bytes != s * N * x->d1)
      return set_error(DPF_E_INVALID, "dpf_read: 'x' needs " + std::to_string(s * N * x->d1) + " bytes");
    cudaError_t e = cudaMemcpy2DAsync(dst, s * x->d1, x->x[mat], s * x->xp, s * x->d1, N,
                                      cudaMemcpyDeviceToHost, x->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
    return cuda_error(e, "dpf_read");
  }
  else if (w == "z") { src = x->z[mat]; need = s * N * M * x->d2; }
  else if (w == "lq") { src = x->lq[mat]; need = s * N * M; }
  else if (w == "bidx") {
    if (!x->dbg_b) return set_error(DPF_E_INVALID, "dpf_read: bidx needs dpf_set_debug(ctx, 1)");
    src = x->dbg_b; need = 4 * N * M;
  } else if (w == "jla") {
    if (!x->dbg_j) return set_error(DPF_E_INVALID, "dpf_read: jla needs dpf_set_debug(ctx, 1)");
    src = x->dbg_j; need = 4 * N * L;
  } else if (w == "afeat" || w == "ahead") {
    if (!x->proposal || !x->oa_feat || dpf_proposal_kind(x->proposal) != 1)
      return set_error(DPF_E_INVALID, "dpf_read: afeat/ahead need an outer-amortised proposal");
    const int d = w == "afeat" ? 2 * x->d1 + x->dy + 2 * x->d2 : 2 * x->d2;
    src = w == "afeat" ? x->oa_feat : x->oa_out; need = 4 * N * (size_t)d;
  } else if (w == "fallback") {
    if (!x->fb_flag) return set_error(DPF_E_INVALID, "dpf_read: fallback needs a learned proposal");
    src = x->fb_flag; need = 4 * N;
  } else if (w == "head") {
    if (!x->dbg_head || !x->proposal)
      return set_error(DPF_E_INVALID, "dpf_read: head needs a learned proposal and dpf_set_debug(ctx, 1)");
    src = x->dbg_head; need = 4 * N * M * (size_t)dpf_proposal_dout(x->proposal);
  } else return set_error(DPF_E_INVALID, "dpf_read: unknown array '" + w + "'");
  if (bytes != need)
    return set_error(DPF_E_INVALID, "dpf_read: '" + w + "' needs " + std::to_string(need) + " bytes");
  cudaError_t e = cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToHost, x->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  return cuda_error(e, "dpf_read");
}

dpf_status dpf_set_tensor_cores(dpf_ctx* x, int32_t enable) {
  clear_error();
  if (!x) return set_error(DPF_E_INVALID, "dpf_set_tensor_cores: null context");
  if (x->tensor_cores != (enable != 0)) x->grid_step = 0;  // the other kernel sizes its own grid
  x->tensor_cores = enable != 0;
  return DPF_OK;
}

dpf_status dpf_set_debug(dpf_ctx* x, int32_t enable) {
  clear_error();
  if (!x) return set_error(DPF_E_INVALID, "dpf_set_debug: null context");
  if (enable && !x->dbg_b) {
    dpf_status st = dalloc(*x, x->dbg_b, (size_t)4 * x->N * x->M);
    if (!st) st = dalloc(*x, x->anc_prev, (size_t)4 * x->N);
    if (!st) st = dalloc(*x, x->dbg_j, (size_t)4 * x->N * x->L);
    if (!st && x->prec == DPF_F32) st = dalloc(*x, x->dbg_head, (size_t)4 * x->N * x->M * 32);
    if (st) return st;
  }
  x->debug = enable != 0;
  return DPF_OK;
}

dpf_status dpf_profile(dpf_ctx* x, int32_t enable) {
  clear_error();
  if (!x) return set_error(DPF_E_INVALID, "dpf_profile: null context");
  x->profiling = enable != 0;
  return DPF_OK;
}

dpf_status dpf_profile_read(dpf_ctx* x, double* ms, int64_t* launches) {
  clear_error();
  if (!x) return set_error(DPF_E_INVALID, "dpf_profile_read: null context");
  cudaError_t e = cudaStreamSynchronize(x->stream);
  if (e != cudaSuccess) return cuda_error(e, "dpf_profile_read");
  double tot = 0.0;
  for (size_t q = 0; q + 1 < x->pev_used; q += 2) {
    float f = 0.f;
    e = cudaEventElapsedTime(&f, x->pev[q], x->pev[q + 1]);
    if (e != cudaSuccess) return cuda_error(e, "dpf_profile_read: elapsed time");
    tot += f;
  }
  if (ms) *ms = tot;
  if (launches) *launches = (int64_t)(x->pev_used / 2);
  x->pev_used = 0;
  return DPF_OK;
}

dpf_status dpf_memory(dpf_ctx* x, size_t* bytes) {
  clear_error();
  if (!x || !bytes) return set_error(DPF_E_INVALID, "dpf_memory: null argument");
  *bytes = x->bytes;
  return DPF_OK;
}

void dpf_destroy(dpf_ctx* x) {
  if (!x) return;
  cudaStreamSynchronize(x->stream);
  free_all(x);
  delete x;
}

}  // extern "C"

extern "C" dpf_status dpf_fail_allocation_after(int64_t n) {
  dpf::clear_error();
  if (n < 0) return dpf::set_error(DPF_E_INVALID, "dpf_fail_allocation_after: n must be >= 0");
  dpf::g_alloc_countdown.store(n);
  return DPF_OK;
}
