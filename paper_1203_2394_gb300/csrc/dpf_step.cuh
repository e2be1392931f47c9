// The LA-DPF step kernels.
//
// One call t runs two kernels on the context's stream:
//  1. step_kernel (one CTA per outer particle i): the deferred inner step of
//     step t-1 for destination i (the selection of x_{t-1} among the
//     ancestor's look-ahead draws, local systematic resampling of the
//     ancestor's inner set, propagation and the y_{t-1} update of the inner
//     weights; Fig. 4 step 4, DPF step 6, eq. qbar), then the look-ahead of step
//     t on the fresh inner set held in shared memory (Fig. 4 steps 1-2, eqs.
//     approx1, qnobar, weightsMC). The inner set is read once and written once.
//  2. fused_outer_kernel (dpf_outer.cuh, one cooperative launch): evidence, ESS,
//     the filtered mean and the quantised total C of the outer weights (eq.
//     weightsopt), then the global systematic resampling of the outer set (Fig. 4
//     step 3) after one grid-wide barrier.
//
// Device layout (structure of arrays, element type T):
//   z[c][n][j] (d2 x N x M), lq[n][j], x[c][n] (d1 x N)   two slots each
//   lwh[n][m], xbb[n][m][c]                               two slots each
//   lw[n], xm[c][n], zm[c][n], wout[n], anc[n], sel[n]
// Slot parity: after call t the materialised state of step t-1 sits in slot
// (t-1) % 2 and the look-ahead products of step t in slot t % 2.
#pragma once

#include "dpf_common.cuh"
#include "dpf_tc.cuh"
#include "dpf_internal.h"
#include "dpf_resample.cuh"

namespace dpf {

// Model constants, by value as a kernel parameter (read through the constant
// cache with uniform indices). Internal x-first coordinates, row-major.
template <typename T, int D1, int D2, int DY>
struct MC {
  T Axx[D1][D1], Azx[D2][D1], Azz[D2][D2];
  T Lqx[D1][D1], LqxInv[D1][D1], Lqz[D2][D2];
  T WAxz[D1][D2];  // Lqx^{-1} A_xz
  T Hx[DY][D1], Hz[DY][D2], LrInv[DY][DY], LrHz[DY][D2];  // LrHz = R^{-1/2} H_z
  T HzAzz[DY][D2], HzAzx[DY][D1], Ls[DY][DY];
  T K[D2][DY];     // Q_z H_z^T (H_z Q_z H_z^T)^{-1}
  T m0x[D1], m0z[D2], Lp0x[D1][D1], G0[D2][D1], Lp0c[D2][D2];
  T ga, gb, qc, lognorm_y;
  int growth, quad, diag_qz;
};

template <typename T>
struct StepArgs {
  const T* z_old;
  const T* lq_old;
  const T* x_old;
  T* z_new;
  T* lq_new;
  T* x_new;
  const T* lwh_old;
  const T* xbb_old;
  T* lwh_new;
  T* xbb_new;
  const int32_t* anc;
  int32_t* sel;
  T* lw;
  T* xm;
  T* zm;
  const T* y_prev;
  const T* y_cur;
  unsigned long long* lwmax_key;
  unsigned long long* Csum;  // reset here for this step's outer reduction
  int32_t* dbg_b;
  int* err;
  long long N;
  int M, L;
  uint32_t t;
  Key key;
  T gcos_prev;  // growth cosine term of the transition into step t-1
  T gcos_cur;   // ... into step t
  int first;    // t == 1: the state is the initial one, no inner step to run
  // launch geometry, computed on the host (see step_geometry)
  int tpm, rows, stride;
  int xp;        // padded length of an x row (16-byte rows)
  T scaleM, scaleL;  // 2^(31 - ceil(log2 M)) and 2^(31 - ceil(log2 L)): the local-rule scalings
  T logM, logL;      // log M, log L
  uint32_t stage_bytes, stage_tx;
  uint32_t off_stage, off_sz, off_slq, off_sx, off_slwh, off_sxbb;
  uint32_t off_cum, off_kd, off_E, off_xw, off_cw, off_xbs, off_row, off_red, off_part;
  uint32_t off_zlo, off_ahi, off_alo;  // tensor-core operand tiles (block kernel, TC only)
  uint32_t off_zmat, off_sb;           // wide z (d2 > 32): [A_zz K] rows and the combined sums
  uint32_t off_zrow;  // warp step: the rows [A_zx A_zz K] for the z-mean, one copy a warp
  uint32_t off_proj;  // wide z, tensor cores: [L_r^-1 H_z | H_z A_zz] columns, A_zx rows, diag L_qz
  int la_only;  // the inner update already ran (learned proposal): look-ahead from the materialised state
  // optional subset of the groups: positions 0 .. *gcount - 1 of glist (device), in
  // place of every group 0 .. N - 1 (the learned proposal's per-group fallback)
  const int32_t* glist;
  const int32_t* gcount;
  const int32_t* gskip;  // optional [N]: groups with a nonzero entry are left untouched
};

// Group index at position g of the launch's group sequence.
template <typename T>
__device__ __forceinline__ long long group_at(const StepArgs<T>& a, long long g) {
  return a.glist ? (long long)a.glist[g] : g;
}
// Number of positions in the launch's group sequence.
template <typename T>
__device__ __forceinline__ long long group_count(const StepArgs<T>& a) {
  if (!a.glist) return a.N;
  const long long c = (long long)*a.gcount;
  return c < a.N ? c : a.N;
}

// Order-preserving unsigned keys of floating-point values (for atomicMax).
__device__ __forceinline__ unsigned long long order_key(float v) {
  const uint32_t b = __float_as_uint(v);
  return (unsigned long long)((b & 0x80000000u) ? ~b : (b | 0x80000000u));
}
__device__ __forceinline__ unsigned long long order_key(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ void order_decode(unsigned long long k, float& v) {
  const uint32_t b = (uint32_t)k;
  v = __uint_as_float((b & 0x80000000u) ? (b & 0x7fffffffu) : ~b);
}
__device__ __forceinline__ void order_decode(unsigned long long k, double& v) {
  v = __longlong_as_double(
      (long long)((k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k));
}

__device__ __forceinline__ float log_t(float v) { return logf(v); }
__device__ __forceinline__ double log_t(double v) { return log(v); }

// Threads per look-ahead row: a power of two <= 32 with rows * TPM <= NT.
inline int rows_tpm(int nt, int L) {
  int tpm = 1;
  while (tpm * 2 <= 32 && tpm * 2 * L <= nt) tpm *= 2;
  return tpm;
}

// Floats per packed look-ahead record of one inner particle:
// [a_k, g'_k (DY), f'_k (D1, when x depends on z)], padded to 16 bytes.
template <typename T, int D1, int DY, bool XZ>
constexpr int rec_len() {
  return ((1 + DY + (XZ ? D1 : 0)) * (int)sizeof(T) + 15) / 16 * 16 / (int)sizeof(T);
}

// Shared-memory carve-up and row mapping of step_kernel, on the host: two
// input stages (the source rows of a group), then the work buffers.
template <typename T, int D1, int D2, int DY, bool XZ>
inline size_t step_geometry(int M, int L, int nt, StepArgs<T>* a, bool first = false,
                            int nstages = 2, bool tc = false) {
  const int tpm = rows_tpm(nt, L);
  int stride = M;
  while (stride % 32 != tpm % 32) ++stride;
  const int xp = (int)((D1 * sizeof(T) + 15) / 16 * 16 / sizeof(T));
  auto r16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
  // stage layout
  size_t so = 0;
  const uint32_t sz = (uint32_t)so; so += r16(sizeof(T) * D2 * M);
  const uint32_t slq = (uint32_t)so; so += r16(sizeof(T) * M);
  const uint32_t sx = (uint32_t)so; so += r16(sizeof(T) * xp);
  const uint32_t slwh = (uint32_t)so; so += r16(sizeof(T) * L);
  const uint32_t sxbb = (uint32_t)so; so += r16(sizeof(T) * L * D1);
  const size_t stage = so;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += r16(bytes);
    return (uint32_t)at;
  };
  const uint32_t st0 = take(nstages * stage), cum = take(sizeof(uint32_t) * M),
                 kd = take(sizeof(T) * rec_len<T, D1, DY, XZ>() * M),
                 E = take(sizeof(T) * (size_t)L * stride), xw = take(sizeof(T) * L * D1),
                 cw = take(sizeof(T) * L * DY), xbs = take(sizeof(T) * L * D1),
                 row = take(sizeof(T) * L * 5), red = take(sizeof(T) * 32 + sizeof(uint32_t) * 64),
                 part = take(sizeof(T) * 32 * (D2 + DY));
  // tensor-core propagation: the ancestors' z as TF32 low parts (the high parts
  // reuse the stage's z rows), and A_zz split in two, padded to 16-row multiples
  const int np = (D2 + 15) / 16 * 16;
  const uint32_t zlo = tc ? take(sizeof(float) * (size_t)M * D2) : 0u,
                 ahi = tc ? take(sizeof(float) * (size_t)np * D2) : 0u,
                 alo = tc ? take(sizeof(float) * (size_t)np * D2) : 0u;
  // wide z: the rows [A_zz(r, .) K(r, .)] for the z-mean combine, one warp a row
  const uint32_t zmat = D2 > 32 ? take(sizeof(T) * (size_t)D2 * (D2 + DY)) : 0u,
                 sbo = D2 > 32 ? take(sizeof(T) * (size_t)(D2 + DY)) : 0u,
                 proj = (D2 > 32 && tc) ? take(sizeof(T) * (size_t)D2 * (2 * DY + D1 + 1)) : 0u;
  if (a) {
    a->tpm = tpm;
    a->rows = nt / tpm;
    a->stride = stride;
    a->xp = xp;
    a->stage_bytes = (uint32_t)stage;
    a->stage_tx = (uint32_t)(sizeof(T) * (D2 * M + M + xp + (first ? 0 : L + L * D1)));
    a->off_stage = st0; a->off_sz = sz; a->off_slq = slq; a->off_sx = sx; a->off_slwh = slwh;
    a->off_sxbb = sxbb;
    a->off_cum = cum; a->off_kd = kd; a->off_E = E; a->off_xw = xw;
    a->off_cw = cw; a->off_xbs = xbs; a->off_row = row; a->off_red = red; a->off_part = part;
    a->off_zlo = zlo; a->off_ahi = ahi; a->off_alo = alo;
    a->off_zmat = zmat; a->off_sb = sbo; a->off_proj = proj;
  }
  return o;
}

// Runtime-width block reductions (blockDim.x is a multiple of 32).
template <typename T>
__device__ __forceinline__ T bmax(T v, T* red) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  T r = red[0];
  for (int q = 1; q < nw; ++q) r = fmax(r, red[q]);
  return r;
}
template <typename T>
__device__ __forceinline__ T bsum(T v, T* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  T r = red[0];
  for (int q = 1; q < nw; ++q) r += red[q];
  return r;
}
__device__ __forceinline__ uint32_t bscan_u32(uint32_t v, uint32_t* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t n = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += n;
  }
  __syncthreads();
  if (lane == 31) red[w] = v;
  __syncthreads();
  uint32_t add = 0;
  for (int q = 0; q < w; ++q) add += red[q];
  return v + add;
}

// mean of x_{s+1} without the A_xz z part: g(x, s) + A_xx x
template <typename T, int D1, int D2, int DY>
__device__ __forceinline__ void mu_x(const MC<T, D1, D2, DY>& mc, const T (&x)[D1], T gcos,
                                     T (&out)[D1]) {
#pragma unroll
  for (int r = 0; r < D1; ++r) {
    T v = T(0);
    if (mc.growth) v = mc.ga * x[r] + mc.gb * x[r] / (T(1) + x[r] * x[r]) + gcos;
#pragma unroll
    for (int c = 0; c < D1; ++c) v += mc.Axx[r][c] * x[c];
    out[r] = v;
  }
}
// x part of the observation mean: qc x.^2 + H_x x
template <typename T, int D1, int D2, int DY>
__device__ __forceinline__ void h_x(const MC<T, D1, D2, DY>& mc, const T (&x)[D1], T (&out)[DY]) {
#pragma unroll
  for (int r = 0; r < DY; ++r) {
    T v = T(0);
    if (mc.quad) v = mc.qc * x[r < D1 ? r : 0] * x[r < D1 ? r : 0];
#pragma unroll
    for (int c = 0; c < D1; ++c) v += mc.Hx[r][c] * x[c];
    out[r] = v;
  }
}

// Initialisation (Fig. 4, "Initialize"): x_0 ~ N(m0x, P0xx), z_0 | x_0 from the
// conditional Gaussian, lq = -log M. One CTA per outer particle.
template <typename T, int D1, int D2, int DY>
__device__ __forceinline__ void init_body(const MC<T, D1, D2, DY>& mc, T* z, T* lq, T* x, long long N,
                                          int M, int xp, Key key) {
  const long long i = blockIdx.x;
  const int j = threadIdx.x;
  if (j >= M) return;
  T e1[D1], xi[D1];
  normals<D1>(key, 0u, (uint32_t)i, P_INIT_X, 0u, e1);
#pragma unroll
  for (int r = 0; r < D1; ++r) {
    T v = mc.m0x[r];
#pragma unroll
    for (int c = 0; c < D1; ++c) if (c <= r) v += mc.Lp0x[r][c] * e1[c];
    xi[r] = v;
  }
  T e2[D2];
  normals<D2>(key, 0u, (uint32_t)i, P_INIT_Z, (uint32_t)j, e2);
#pragma unroll
  for (int r = 0; r < D2; ++r) {
    T v = mc.m0z[r];
#pragma unroll
    for (int c = 0; c < D1; ++c) v += mc.G0[r][c] * (xi[c] - mc.m0x[c]);
#pragma unroll
    for (int c = 0; c < D2; ++c) if (c <= r) v += mc.Lp0c[r][c] * e2[c];
    z[((long long)r * N + i) * M + j] = v;
  }
  lq[i * M + j] = -log_t((T)M);
  if (j == 0) {
#pragma unroll
    for (int r = 0; r < xp; ++r) x[i * xp + r] = r < D1 ? xi[r < D1 ? r : 0] : T(0);
  }
}

template <typename T, int D1, int D2, int DY>
__global__ void init_kernel(const __grid_constant__ MC<T, D1, D2, DY> mc, T* z, T* lq, T* x,
                            long long N, int M, int xp, Key key) {
  init_body<T, D1, D2, DY>(mc, z, lq, x, N, M, xp, key);
}

// The same with the model constants in global memory.
template <typename T, int D1, int D2, int DY>
__global__ void init_kernel_g(const MC<T, D1, D2, DY>* __restrict__ mcp, T* z, T* lq, T* x,
                              long long N, int M, int xp, Key key) {
  init_body<T, D1, D2, DY>(*mcp, z, lq, x, N, M, xp, key);
}

__device__ __forceinline__ float exp2_t(float x) { return ex2_approx(x); }
__device__ __forceinline__ double exp2_t(double x) { return exp2(x); }
__device__ __forceinline__ float log2_t(float x) { return log2f(x); }
__device__ __forceinline__ double log2_t(double x) { return log2(x); }

constexpr int MBAR_SPIN_LIMIT = 1 << 16;  // bounded wait on a stage's barrier
constexpr double LOG2E_D = 1.4426950408889634;
constexpr double LN2_D = 0.6931471805599453;
constexpr double SQ_D = 0.84932180028801907;  // sqrt(log2(e) / 2): -x^2/2 in log2 units is -(SQ x)^2

// Inclusive scan over the particle index j = tid + p * NT of one uint32 per
// particle (PPT planes); `red` holds 32 * PPT words.
template <int PPT>
__device__ __forceinline__ void bscan_planes(const uint32_t (&c)[PPT], uint32_t (&incl)[PPT],
                                             uint32_t* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t v[PPT];
#pragma unroll
  for (int p = 0; p < PPT; ++p) v[p] = c[p];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const uint32_t n = __shfl_up_sync(FULL, v[p], o);
      if (lane >= o) v[p] += n;
    }
  }
  __syncthreads();
  if (lane == 31) {
#pragma unroll
    for (int p = 0; p < PPT; ++p) red[p * 32 + w] = v[p];
  }
  __syncthreads();
  uint32_t run = 0;
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    uint32_t before = 0, tot = 0;
    for (int q = 0; q < nw; ++q) {
      const uint32_t r = red[p * 32 + q];
      before += q < w ? r : 0u;
      tot += r;
    }
    incl[p] = v[p] + before + run;
    run += tot;
  }
}

// ---- mbarrier and bulk-copy (TMA, non-tensor) wrappers ----
// Stage the source rows of one group (its ancestor's, or its own on the first
// step): the inner set z (d2 rows of M), its log-weights, its x row and the
// ancestor's look-ahead products. BULK: one thread issues bulk copies that
// complete on the stage's mbarrier (WARP: issued by the calling warp, one lane a
// copy; otherwise by thread 0); otherwise all threads copy directly.
template <typename T, int D1, int D2, bool BULK, bool WARP = false>
__device__ __forceinline__ void stage_group(const StepArgs<T>& a, unsigned char* st, uint64_t* bar,
                                            long long src) {
  const int M = a.M, L = a.L;
  T* sz = (T*)(st + a.off_sz);
  T* slq = (T*)(st + a.off_slq);
  T* sx = (T*)(st + a.off_sx);
  T* slwh = (T*)(st + a.off_slwh);
  T* sxbb = (T*)(st + a.off_sxbb);
  const long long NM = a.N * (long long)M;
  if (BULK && WARP) {  // one warp: lane 0 arms the barrier, then one lane a copy
    const int lane = threadIdx.x & 31;
    if (lane == 0) mbar_arrive_tx(bar, a.stage_tx);
    for (int e = lane; e < D2 + 4; e += 32) {
      if (e < D2) {
        bulk_load(sz + e * M, a.z_old + e * NM + src * M, (uint32_t)(M * sizeof(T)), bar);
      } else if (e == D2) {
        bulk_load(slq, a.lq_old + src * M, (uint32_t)(M * sizeof(T)), bar);
      } else if (e == D2 + 1) {
        bulk_load(sx, a.x_old + src * a.xp, (uint32_t)(a.xp * sizeof(T)), bar);
      } else if (!a.first) {
        if (e == D2 + 2)
          bulk_load(slwh, a.lwh_old + src * L, (uint32_t)(L * sizeof(T)), bar);
        else
          bulk_load(sxbb, a.xbb_old + src * L * D1, (uint32_t)(L * D1 * sizeof(T)), bar);
      }
    }
  } else if (BULK) {
    if (threadIdx.x == 0) {
      mbar_arrive_tx(bar, a.stage_tx);
#pragma unroll
      for (int c = 0; c < D2; ++c)
        bulk_load(sz + c * M, a.z_old + c * NM + src * M, (uint32_t)(M * sizeof(T)), bar);
      bulk_load(slq, a.lq_old + src * M, (uint32_t)(M * sizeof(T)), bar);
      bulk_load(sx, a.x_old + src * a.xp, (uint32_t)(a.xp * sizeof(T)), bar);
      if (!a.first) {
        bulk_load(slwh, a.lwh_old + src * L, (uint32_t)(L * sizeof(T)), bar);
        bulk_load(sxbb, a.xbb_old + src * L * D1, (uint32_t)(L * D1 * sizeof(T)), bar);
      }
    }
  } else {
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
#pragma unroll
      for (int c = 0; c < D2; ++c) sz[c * M + j] = a.z_old[c * NM + src * M + j];
      slq[j] = a.lq_old[src * M + j];
    }
    for (int c = threadIdx.x; c < D1; c += blockDim.x) sx[c] = a.x_old[src * a.xp + c];
    if (!a.first) {
      for (int m = threadIdx.x; m < L; m += blockDim.x) slwh[m] = a.lwh_old[src * L + m];
      for (int q = threadIdx.x; q < L * D1; q += blockDim.x) sxbb[q] = a.xbb_old[src * L * D1 + q];
    }
  }
}

constexpr int TC_SPIN = 1 << 22;  // bounded wait for the tensor-core MMAs of one group

// The block step. TC: the propagation A_zz z runs on the tensor cores (3xTF32,
// FP32 only, one thread per inner particle, M a multiple of 128, one stage).
template <typename T, int D1, int D2, int DY, bool XZ, int PPT, bool BULK, bool TC>
__device__ __forceinline__ void step_body(const MC<T, D1, D2, DY>& mc, const StepArgs<T>& a) {
  static_assert(!TC || (sizeof(T) == 4 && PPT == 1 && !BULK && D2 % 8 == 0), "tensor-core step");
  static_assert(!TC || D2 <= 32 || DY % 4 == 0, "vector loads of the wide projections");
  // one stage filled by bulk copies issued as soon as the stage is free (tensor-core
  // step: right after the MMAs that read it), so the next group's rows arrive during
  // the rest of this group
  constexpr bool PF = TC;
  constexpr int NP = (D2 + 15) / 16 * 16;  // MMA N: A_zz rows padded to 16
  constexpr int KC16 = D2 * 4 / 16;        // 16-byte chunks per operand row
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int REC = rec_len<T, D1, DY, XZ>();
  const int NT = blockDim.x;
  const int M = a.M, L = a.L;
  const long long N = a.N;
  const long long NM = N * (long long)M;
  unsigned char* const stage0 = smem_raw + a.off_stage;  // two stages of a.stage_bytes
  uint32_t* cum = (uint32_t*)(smem_raw + a.off_cum);
  T* kd = (T*)(smem_raw + a.off_kd);
  T* E = (T*)(smem_raw + a.off_E);
  T* xw = (T*)(smem_raw + a.off_xw);
  T* cw = (T*)(smem_raw + a.off_cw);
  T* xbs = (T*)(smem_raw + a.off_xbs);
  T* rowS = (T*)(smem_raw + a.off_row);
  T* rowA = rowS + L;
  T* shS = rowA + L;
  T* shA = shS + L;
  T* coef = shA + L;
  T* red = (T*)(smem_raw + a.off_red);
  uint32_t* redU = (uint32_t*)(red + 32);
  T* part = (T*)(smem_raw + a.off_part);
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ __align__(8) uint64_t tcbar;
  __shared__ uint32_t s_taddr;
  __shared__ int s_m, s_fallback;
  __shared__ uint32_t s_uin;

  const int tid = threadIdx.x, lane = tid & 31;
  const T NEG = neg_inf<T>();
  const T LOG2E = (T)LOG2E_D, SQ = (T)SQ_D;
  const RoundKeys rk = round_keys(a.key);  // (the tensor-core path's noise)
  if (blockIdx.x == 0 && tid == 0) *a.Csum = 0ull;
  if ((BULK || PF) && tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_fence_init();
  }
  if constexpr (D2 > 32) {
    T* zmat = (T*)(smem_raw + a.off_zmat);
    for (int e = tid; e < D2 * (D2 + DY); e += NT) {
      const int r = e / (D2 + DY), c = e % (D2 + DY);
      zmat[e] = c < D2 ? mc.Azz[r][c] : mc.K[r][c - D2];
    }
  }
  if constexpr (TC && D2 > 32) {
    // per coordinate r: (L_r^-1 H_z)[., r] then (H_z A_zz)[., r]; then the rows of A_zx
    // and the diagonal of L_qz
    T* pj = (T*)(smem_raw + a.off_proj);
    for (int e = tid; e < D2 * 2 * DY; e += NT) {
      const int r = e / (2 * DY), q = e % (2 * DY);
      pj[e] = q < DY ? mc.LrHz[q][r] : mc.HzAzz[q - DY][r];
    }
    for (int e = tid; e < D2 * D1; e += NT) pj[D2 * 2 * DY + e] = mc.Azx[e / D1][e % D1];
    for (int r = tid; r < D2; r += NT) pj[D2 * (2 * DY + D1) + r] = mc.Lqz[r][r];
  }
  uint32_t taddr = 0, tc_phase = 0;
  constexpr uint32_t TC_COLS = TC ? (NP * 2 <= 32 ? 32 : NP * 2 <= 64 ? 64 : NP * 2 <= 128 ? 128 : 256) : 32;
  if constexpr (TC) {
    // B operand: A_zz (row n = output coordinate n) split hi/lo, K-major; rows >= D2 zero
    unsigned char* ahi = smem_raw + a.off_ahi;
    unsigned char* alo = smem_raw + a.off_alo;
    for (int e = tid; e < NP * D2; e += NT) {
      const int n = e / D2, k = e % D2;
      float hi = 0.f, lo = 0.f;
      if (n < D2) tc::split_tf32((float)mc.Azz[n][k], hi, lo);
      *(float*)(ahi + tc::kmajor_offset(n, 4 * k, KC16)) = hi;
      *(float*)(alo + tc::kmajor_offset(n, 4 * k, KC16)) = lo;
    }
    tc::fence_proxy_async();
    if (tid < 32) {
      tc::tmem_alloc(&s_taddr, TC_COLS);
      tc::tmem_relinquish();
    }
    if (tid == 0) {
      mbar_init(&tcbar, 1);
      mbar_fence_init();
    }
    tc::fence_before();
  }
  __syncthreads();
  if constexpr (TC) {
    tc::fence_after();
    taddr = s_taddr;
  }

  // prologue (bulk path): stage the first group; thread 0 keeps the next group's
  // source index in flight
  long long g = blockIdx.x;
  long long src_next = -1;
  const long long G = group_count(a);
  // the source group of position q (the next one a stage is filled for)
  auto source_of = [&](long long q) {
    const long long iq = group_at(a, q);
    return a.first ? iq : (long long)a.anc[iq];
  };
  if (PF && g < G && tid < 32) stage_group<T, D1, D2, true, true>(a, stage0, &bars[0], source_of(g));
  if (BULK && g < G) {
    const long long i0 = group_at(a, g);
    const long long src0 = a.first ? i0 : (long long)a.anc[i0];
    stage_group<T, D1, D2, BULK>(a, stage0, &bars[0], src0);
    if (tid == 0 && g + gridDim.x < G) {
      const long long i1 = group_at(a, g + gridDim.x);
      src_next = a.first ? i1 : (long long)a.anc[i1];
    }
  }
  for (int k = 0; g < G; g += gridDim.x, ++k) {
    const long long i = group_at(a, g);
    const int sidx = k & 1;
    unsigned char* st = stage0 + (BULK ? sidx * a.stage_bytes : 0);
    if (BULK) {
      // prefetch the next group into the other stage (released at the end of the last group)
      if (tid == 0 && g + gridDim.x < G) {
        stage_group<T, D1, D2, BULK>(a, stage0 + (sidx ^ 1) * a.stage_bytes, &bars[sidx ^ 1], src_next);
        const long long g2 = g + 2 * (long long)gridDim.x;
        if (g2 < G) {
          const long long i2 = group_at(a, g2);
          src_next = a.first ? i2 : (long long)a.anc[i2];
        }
      }
      int spins = 0;
      while (!mbar_test(&bars[sidx], (uint32_t)((k >> 1) & 1))) {
        if (++spins > MBAR_SPIN_LIMIT) {
          if (tid == 0) atomicOr(a.err, ERR_TIMEOUT);
          break;
        }
      }
    } else if (PF) {
      int spins = 0;
      while (!mbar_test(&bars[0], (uint32_t)(k & 1))) {
        if (++spins > MBAR_SPIN_LIMIT) {
          if (tid == 0) atomicOr(a.err, ERR_TIMEOUT);
          break;
        }
      }
    } else if (!(a.gskip && a.gskip[i])) {
      const long long src = a.first ? i : (long long)a.anc[i];
      stage_group<T, D1, D2, BULK>(a, st, nullptr, src);
      __syncthreads();
    }
    bool pf_issued = false;  // the next group's stage copy is under way
    if (a.gskip && a.gskip[i]) {  // every thread has left the stage wait before it is re-armed
      __syncthreads();
      if (PF && tid < 32 && g + gridDim.x < G)
        stage_group<T, D1, D2, true, true>(a, stage0, &bars[0], source_of(g + gridDim.x));
      continue;
    }
    T* sz = (T*)(st + a.off_sz);
    T* zsrc = sz;          // wide z: where the look-ahead's z sits for the z-mean
    bool zstored = false;  // z_t already written (the rolled tensor-core epilogue)
    T gz[DY];              // ... and its H_z A_zz z_t
#pragma unroll
    for (int q = 0; q < DY; ++q) gz[q] = T(0);
    T* slq = (T*)(st + a.off_slq);
    T* sx = (T*)(st + a.off_sx);
    T* slwh = (T*)(st + a.off_slwh);
    T* sxbb = (T*)(st + a.off_sxbb);

    T x[D1];         // x_{t-1}^(i): the group's outer particle
    T zr[PPT][D2];   // this thread's inner particles z_{t-1}^(i,j), j = tid + p NT
    T lqr[PPT];      // and their normalised log-weights
    T sigma, SA0;    // the largest inner log-weight, and sum_k exp(lq_k - sigma)
#pragma unroll
    for (int p = 0; p < PPT; ++p) lqr[p] = NEG;

    if (a.first) {
#pragma unroll
      for (int c = 0; c < D1; ++c) x[c] = sx[c];
#pragma unroll
      for (int p = 0; p < PPT; ++p) {
        const int j = tid + p * NT;
#pragma unroll
        for (int c = 0; c < D2; ++c) zr[p][c] = T(0);  // past M: zeros, never undefined
        if (j < M) {
#pragma unroll
          for (int c = 0; c < D2; ++c) zr[p][c] = sz[c * M + j];
          lqr[p] = slq[j];
        }
      }
      if (a.la_only) {  // the state's own weights: largest lq and sum exp(lq - largest)
        T mx = NEG;
#pragma unroll
        for (int p = 0; p < PPT; ++p) mx = fmax(mx, lqr[p]);
        sigma = bmax(mx, red);
        T se = T(0);
#pragma unroll
        for (int p = 0; p < PPT; ++p)
          if (tid + p * NT < M) se += exp2_t((lqr[p] - sigma) * LOG2E);
        SA0 = bsum(se, red);
      } else {
        sigma = -log_t((T)M);
        SA0 = (T)M;
      }
    } else {
      // ---- selection of x_{t-1}^(i) among the ancestor's look-ahead draws ----
      if (tid < 32) {
        const T l0 = lane < L ? slwh[lane] : NEG;
        const T l1 = lane + 32 < L ? slwh[lane + 32] : NEG;
        const T mx = warp_max(fmax(l0, l1));
        const T s2 = a.scaleL;
        const uint32_t c0 = lane < L ? (uint32_t)floor(exp2_t((l0 - mx) * LOG2E) * s2) : 0u;
        const uint32_t c1 = lane + 32 < L ? (uint32_t)floor(exp2_t((l1 - mx) * LOG2E) * s2) : 0u;
        uint32_t s0 = c0, s1 = c1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t n0 = __shfl_up_sync(FULL, s0, o), n1 = __shfl_up_sync(FULL, s1, o);
          if (lane >= o) {
            s0 += n0;
            s1 += n1;
          }
        }
        const uint32_t tot0 = __shfl_sync(FULL, s0, 31), tot1 = __shfl_sync(FULL, s1, 31);
        const uint64_t C = (uint64_t)tot0 + tot1;
        // lanes 0 and 1 draw the two per-group words (selection and local resampling)
        const uint32_t wsel = philox(ctr(a.t - 1, (uint32_t)i, lane == 0 ? P_SEL : P_INNER, 0u, 0u), a.key).x;
        const uint32_t usel = __shfl_sync(FULL, wsel, 0);
        const uint64_t rhs = (uint64_t)usel * C;
        const unsigned b0 = __ballot_sync(FULL, ((uint64_t)s0 << 32) > rhs);
        const unsigned b1 = __ballot_sync(FULL, ((uint64_t)(s1 + tot0) << 32) > rhs);
        if (lane == 0) {
          int m = b0 ? __ffs(b0) - 1 : (b1 ? 32 + __ffs(b1) - 1 : L - 1);
          if (C == 0 || m >= L) {  // no positive weight (NaN or -inf look-ahead weights)
            atomicOr(a.err, ERR_NUMERIC);
            m = L - 1;
          }
          s_m = m;
          a.sel[i] = m;
        }
        if (lane == 1) s_uin = wsel;
      }
      __syncthreads();
      const int msel = s_m;
      T xa[D1];
#pragma unroll
      for (int c = 0; c < D1; ++c) {
        x[c] = sxbb[msel * D1 + c];
        xa[c] = sx[c];
      }
      // ---- local resampling of the ancestor's inner set (eq. qnobar weights) ----
      T wres[D1];  // whitened x_{t-1} - (g + A_xx x_a): the z-free part of the residual
      if (XZ) {
        T mxa[D1];
        mu_x(mc, xa, a.gcos_prev, mxa);
#pragma unroll
        for (int r = 0; r < D1; ++r) {
          T v = T(0);
#pragma unroll
          for (int c = 0; c < D1; ++c) if (c <= r) v += mc.LqxInv[r][c] * (x[c] - mxa[c]);
          wres[r] = v;
        }
      }
      T alpha[PPT];
      T amax = NEG;
#pragma unroll
      for (int p = 0; p < PPT; ++p) {
        const int j = tid + p * NT;
        alpha[p] = NEG;
        if (j < M) {
          T al = slq[j];
          if (XZ) {
            T q = T(0);
#pragma unroll
            for (int r = 0; r < D1; ++r) {
              T v = wres[r];
#pragma unroll
              for (int c = 0; c < D2; ++c) v -= mc.WAxz[r][c] * sz[c * M + j];
              q += v * v;
            }
            al -= T(0.5) * q;
          }
          alpha[p] = al;
          amax = fmax(amax, al);
        }
      }
      amax = bmax(amax, red);
      uint32_t cw_[PPT], incl[PPT];
#pragma unroll
      for (int p = 0; p < PPT; ++p)
        cw_[p] = tid + p * NT < M ? (uint32_t)floor(exp2_t((alpha[p] - amax) * LOG2E) * a.scaleM) : 0u;
      bscan_planes<PPT>(cw_, incl, redU);
#pragma unroll
      for (int p = 0; p < PPT; ++p)
        if (tid + p * NT < M) cum[tid + p * NT] = incl[p];
      __syncthreads();
      // ---- propagation and the y_{t-1} update (eq. qbar) ----
      const uint32_t C = cum[M - 1];
      const uint32_t uin = s_uin;
      T azx[D2];
#pragma unroll
      for (int r = 0; r < D2; ++r) {
        T v = T(0);
#pragma unroll
        for (int c = 0; c < D1; ++c) v += mc.Azx[r][c] * xa[c];
        azx[r] = v;
      }
      T yh[DY];  // whitened y_{t-1} - q x.^2 - H_x x
      {
        T hx[DY], res[DY];
        h_x(mc, x, hx);
#pragma unroll
        for (int q = 0; q < DY; ++q) res[q] = a.y_prev[q] - hx[q];
#pragma unroll
        for (int q = 0; q < DY; ++q) {
          T v = T(0);
#pragma unroll
          for (int c = 0; c < DY; ++c) if (c <= q) v += mc.LrInv[q][c] * res[c];
          yh[q] = v;
        }
      }
      T ell[PPT];
      T lmax = NEG;
      if constexpr (!TC) {
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
          const int j = tid + p * NT;
          ell[p] = NEG;
          if (j < M) {
            const int b = sys_local_pick(cum, M, C, M, j, uin);
            if (a.dbg_b) a.dbg_b[i * M + j] = b;
            T eps[D2];
            normals<D2>(a.key, a.t - 1, (uint32_t)i, P_PROP, (uint32_t)j, eps);
            if constexpr (D2 > 32) {
              // wide z: column by column from the staged rows (same order per row)
#pragma unroll
              for (int r = 0; r < D2; ++r) zr[p][r] = azx[r];
#pragma unroll 1
              for (int c = 0; c < D2; ++c) {
                const T zc = sz[c * M + b];
#pragma unroll
                for (int r = 0; r < D2; ++r) zr[p][r] += mc.Azz[r][c] * zc;
              }
#pragma unroll
              for (int r = 0; r < D2; ++r) {
                if (mc.diag_qz) {
                  zr[p][r] += mc.Lqz[r][r] * eps[r];
                } else {
#pragma unroll
                  for (int c = 0; c < D2; ++c) if (c <= r) zr[p][r] += mc.Lqz[r][c] * eps[c];
                }
              }
            } else {
              T zb2[D2];
#pragma unroll
              for (int c = 0; c < D2; ++c) zb2[c] = sz[c * M + b];
#pragma unroll
              for (int r = 0; r < D2; ++r) {
                T v = azx[r];
#pragma unroll
                for (int c = 0; c < D2; ++c) v += mc.Azz[r][c] * zb2[c];
                if (mc.diag_qz) {
                  v += mc.Lqz[r][r] * eps[r];
                } else {
#pragma unroll
                  for (int c = 0; c < D2; ++c) if (c <= r) v += mc.Lqz[r][c] * eps[c];
                }
                zr[p][r] = v;
              }
            }
            T qf = T(0);
#pragma unroll
            for (int q = 0; q < DY; ++q) {
              T v = yh[q];
#pragma unroll
              for (int c = 0; c < D2; ++c) v -= mc.LrHz[q][c] * zr[p][c];
              qf += v * v;
            }
            ell[p] = T(-0.5) * qf;
            lmax = fmax(lmax, ell[p]);
          }
        }
      } else {
        // ---- z_new = A_zz z_b on the tensor cores, then + A_zx x_a + L_qz eps ----
        const int j = tid;  // one inner particle a thread, NT == M
        const int b = sys_local_pick(cum, M, C, M, j, uin);
        if (a.dbg_b) a.dbg_b[i * M + j] = b;
        float zb2[D2];
#pragma unroll
        for (int c = 0; c < D2; ++c) zb2[c] = (float)sz[c * M + b];
        // A_zx x_a, the same for the whole group, and the diagonal of L_qz (part is free
        // until the z-mean)
        T* s_azx = part;
        const T* s_lqd = (const T*)(smem_raw + a.off_proj) + D2 * (2 * DY + D1);
        if (tid < D2) {
          const T* azr = (const T*)(smem_raw + a.off_proj) + D2 * 2 * DY + tid * D1;
          T v = T(0);
#pragma unroll
          for (int c = 0; c < D1; ++c) v += azr[c] * xa[c];
          s_azx[tid] = v;
        }
        __syncthreads();  // every gather is done: the staged z rows become the A operand
        unsigned char* zhi = (unsigned char*)sz;
        unsigned char* zlo = smem_raw + a.off_zlo;
        const uint32_t tb = (uint32_t)(j >> 7) * 128u * (uint32_t)(D2 * 4);
        const int rr = j & 127;
        // four coordinates (one 16-byte chunk of the row) per store
#pragma unroll
        for (int c = 0; c < D2; c += 4) {
          float4 hi, lo;
          tc::split_tf32(zb2[c + 0], hi.x, lo.x);
          tc::split_tf32(zb2[c + 1], hi.y, lo.y);
          tc::split_tf32(zb2[c + 2], hi.z, lo.z);
          tc::split_tf32(zb2[c + 3], hi.w, lo.w);
          *(float4*)(zhi + tb + tc::kmajor_offset(rr, 4 * c, KC16)) = hi;
          *(float4*)(zlo + tb + tc::kmajor_offset(rr, 4 * c, KC16)) = lo;
        }
        tc::fence_proxy_async();
        tc::fence_before();
        __syncthreads();
        if (tid == 0) {
          tc::fence_after();
          const uint32_t idesc = tc::instr_desc(tc::FMT_TF32, 128, NP);
          const uint32_t s_zhi = smem_addr(zhi), s_zlo = smem_addr(zlo);
          const uint32_t s_ahi = smem_addr(smem_raw + a.off_ahi), s_alo = smem_addr(smem_raw + a.off_alo);
          for (int tt = 0; tt < M / 128; ++tt) {
            const uint32_t d = taddr + (uint32_t)(tt * NP), ob = (uint32_t)tt * 128u * (uint32_t)(D2 * 4);
#pragma unroll
            for (int ks = 0; ks < D2 / 8; ++ks) {
              const uint32_t o = (uint32_t)ks * 256u;
              tc::mma_tf32(d, tc::smem_desc(s_zlo + ob + o, KC16), tc::smem_desc(s_ahi + o, KC16), idesc, ks > 0);
              tc::mma_tf32(d, tc::smem_desc(s_zhi + ob + o, KC16), tc::smem_desc(s_alo + o, KC16), idesc, 1);
              tc::mma_tf32(d, tc::smem_desc(s_zhi + ob + o, KC16), tc::smem_desc(s_ahi + o, KC16), idesc, 1);
            }
          }
          tc::commit(&tcbar);
        }
        const uint32_t ta = taddr + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16) + (uint32_t)((j >> 7) * NP);
        if constexpr (D2 > 32) zsrc = (T*)(smem_raw + a.off_zlo);  // the low parts are consumed
        T qf = T(0);
        if (mc.diag_qz) {
          // diagonal Q_z: four coordinates at a time (a TMEM load, one Philox block of noise);
          // z_t goes to the state and to shared memory, and the whitened y residual and the
          // look-ahead's H_z A_zz z_t accumulate on the way (a rolled loop: small code)
          const bool ok = tc::bar_wait(&tcbar, tc_phase, TC_SPIN);
          tc_phase ^= 1u;
          if (!ok && tid == 0) atomicOr(a.err, ERR_TIMEOUT);
          tc::fence_after();
          // the MMAs have read the stage: the next group's rows may come in
          if (PF && tid < 32 && g + gridDim.x < G)
            stage_group<T, D1, D2, true, true>(a, stage0, &bars[0], source_of(g + gridDim.x));
          pf_issued = PF;
          const T* pj = (const T*)(smem_raw + a.off_proj);
          T* zn = a.z_new + i * M + j;
          T rl[DY];
#pragma unroll
          for (int q = 0; q < DY; ++q) rl[q] = yh[q];
#pragma unroll 2
          for (int cb = 0; cb < D2 / 8; ++cb) {  // eight coordinates: one TMEM load, two noise blocks
            float a8[8];
            tc::ld8(ta + (uint32_t)(8 * cb), a8);
            T e[8];
            {
              T e0[4], e1[4];
              normal_block_rk(rk, a.t - 1, (uint32_t)i, P_PROP, (uint32_t)j, 2 * cb, 4, e0);
              normal_block_rk(rk, a.t - 1, (uint32_t)i, P_PROP, (uint32_t)j, 2 * cb + 1, 4, e1);
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                e[u] = e0[u];
                e[4 + u] = e1[u];
              }
            }
            const float4* az4 = reinterpret_cast<const float4*>(s_azx + 8 * cb);
            const float4* lq4 = reinterpret_cast<const float4*>(s_lqd + 8 * cb);
            const float4 za = az4[0], zb = az4[1], la = lq4[0], lb = lq4[1];
            const T azv[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
            const T lqv[8] = {la.x, la.y, la.z, la.w, lb.x, lb.y, lb.z, lb.w};
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int r = 8 * cb + u;
              const T v = ((ok ? (T)a8[u] : T(0)) + azv[u]) + lqv[u] * e[u];
              zsrc[r * M + j] = v;
              zn[(long long)r * NM] = v;
              const float4* pr = reinterpret_cast<const float4*>(pj + r * 2 * DY);
#pragma unroll
              for (int h = 0; h < DY / 4; ++h) {
                const float4 l4 = pr[h];
                rl[4 * h + 0] -= l4.x * v;
                rl[4 * h + 1] -= l4.y * v;
                rl[4 * h + 2] -= l4.z * v;
                rl[4 * h + 3] -= l4.w * v;
              }
#pragma unroll
              for (int h = 0; h < DY / 4; ++h) {
                const float4 g4 = pr[DY / 4 + h];
                gz[4 * h + 0] += g4.x * v;
                gz[4 * h + 1] += g4.y * v;
                gz[4 * h + 2] += g4.z * v;
                gz[4 * h + 3] += g4.w * v;
              }
            }
          }
          tc::fence_before();
#pragma unroll
          for (int q = 0; q < DY; ++q) qf += rl[q] * rl[q];
          zstored = true;
        } else {
        // a general L_qz: every coordinate's noise at once, drawn while the MMAs run
        T eps[D2];
        normals_rk<D2>(rk, a.t - 1, (uint32_t)i, P_PROP, (uint32_t)j, eps);
        const bool ok = tc::bar_wait(&tcbar, tc_phase, TC_SPIN);
        tc_phase ^= 1u;
        if (!ok && tid == 0) atomicOr(a.err, ERR_TIMEOUT);
        tc::fence_after();
        if (PF && tid < 32 && g + gridDim.x < G)
          stage_group<T, D1, D2, true, true>(a, stage0, &bars[0], source_of(g + gridDim.x));
        pf_issued = PF;
        {
          float azz[(D2 + 15) / 16 * 16];
          if constexpr (NP == 64) {  // the whole padded row in one load
            tc::ld64(ta, *reinterpret_cast<float(*)[64]>(azz));
          } else {
#pragma unroll
            for (int c0 = 0; c0 < D2; c0 += 16) tc::ld16(ta + (uint32_t)c0, *reinterpret_cast<float(*)[16]>(azz + c0));
          }
          tc::fence_before();
          // z_new = A_zz z_b + A_zx x_a + L_qz eps, one coordinate at a time
#pragma unroll
          for (int r = 0; r < D2; ++r) {
            T v = (ok ? (T)azz[r] : T(0)) + s_azx[r];
#pragma unroll
            for (int c = 0; c < D2; ++c) if (c <= r) v += mc.Lqz[r][c] * eps[c];
            zr[0][r] = v;
          }
        }
#pragma unroll
        for (int q = 0; q < DY; ++q) {
          T v = yh[q];
#pragma unroll
          for (int c = 0; c < D2; ++c) v -= mc.LrHz[q][c] * zr[0][c];
          qf += v * v;
        }
        }
        ell[0] = T(-0.5) * qf;
        lmax = ell[0];
      }
      lmax = bmax(lmax, red);
      T ls = T(0);
#pragma unroll
      for (int p = 0; p < PPT; ++p)
        if (tid + p * NT < M) ls += exp2_t((ell[p] - lmax) * LOG2E);
      const T lsum = bsum(ls, red);
      const T llsum = log_t(lsum);
      T* zn = a.z_new + i * M + tid;
#pragma unroll
      for (int p = 0; p < PPT; ++p) {
        if (tid + p * NT < M) {
          lqr[p] = ell[p] - lmax - llsum;
          if (!zstored) {
#pragma unroll
            for (int c = 0; c < D2; ++c) zn[c * NM + p * NT] = zr[p][c];
            if constexpr (D2 > 32) {  // z_t for the z-mean (every gather from the stage is done)
#pragma unroll
              for (int c = 0; c < D2; ++c) zsrc[c * M + tid + p * NT] = zr[p][c];
            }
          }
          a.lq_new[i * M + tid + p * NT] = lqr[p];
        }
      }
      if (tid < D1) a.x_new[i * a.xp + tid] = x[tid];
      sigma = -llsum;  // the largest lq: its ell equals lmax
      SA0 = lsum;      // sum_k exp(lq_k - sigma)
    }

    // ======== look-ahead of step t from (x, z, lq) with y_t ========
    T ep[PPT][DY];  // projected look-ahead noise (chol of H_z Q_z H_z^T) eps
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const int j = tid + p * NT;
      if (j < M) {
        T* rec = kd + j * REC;
        rec[0] = (lqr[p] - sigma) * LOG2E;
        T e2[DY];
        la_z_normals<DY>(a.key, a.t, (uint32_t)i, (uint32_t)j, e2);
        T g_[DY];
#pragma unroll
        for (int q = 0; q < DY; ++q) {
          T e = T(0);
#pragma unroll
          for (int c = 0; c < DY; ++c) if (c <= q) e += mc.Ls[q][c] * e2[c];
          ep[p][q] = e;
          T v = e;
#pragma unroll
          for (int c = 0; c < D1; ++c) v += mc.HzAzx[q][c] * x[c];
          if (zstored) {
            v += gz[q];
          } else {
#pragma unroll
            for (int c = 0; c < D2; ++c) v += mc.HzAzz[q][c] * zr[p][c];
          }
          g_[q] = v;
        }
#pragma unroll
        for (int q = 0; q < DY; ++q) {
          T v = T(0);
#pragma unroll
          for (int c = 0; c < DY; ++c) if (c <= q) v += mc.LrInv[q][c] * g_[c];
          rec[1 + q] = SQ * v;
        }
        if (XZ) {
#pragma unroll
          for (int r = 0; r < D1; ++r) {
            T v = T(0);
#pragma unroll
            for (int c = 0; c < D2; ++c) v += mc.WAxz[r][c] * zr[p][c];
            rec[1 + DY + r] = SQ * v;
          }
        }
      }
    }
    if (XZ) {  // cumulative weights for the categorical draws of the mixture components
      uint32_t cw_[PPT], incl[PPT];
#pragma unroll
      for (int p = 0; p < PPT; ++p)
        cw_[p] = tid + p * NT < M ? (uint32_t)floor(exp2_t((lqr[p] - sigma) * LOG2E) * a.scaleM) : 0u;
      bscan_planes<PPT>(cw_, incl, redU);
#pragma unroll
      for (int p = 0; p < PPT; ++p)
        if (tid + p * NT < M) cum[tid + p * NT] = incl[p];
    }
    __syncthreads();
    // ---- L look-ahead draws xbb^(m) (eq. approx1) ----
    if (tid < L) {
      const int m = tid;
      T mux[D1];
      mu_x(mc, x, a.gcos_cur, mux);
      T e1[D1], xwm[D1];
      normals<D1>(a.key, a.t, (uint32_t)i, P_LA_X, (uint32_t)m, e1);
      int jm = 0;
      if (XZ)
        jm = sys_local_pick(cum, M, cum[M - 1], 1, 0,
                            rand_word(a.key, a.t, (uint32_t)i, P_LA_J, (uint32_t)m));
#pragma unroll
      for (int c = 0; c < D1; ++c) xwm[c] = (XZ ? kd[jm * REC + 1 + DY + c] / SQ : T(0)) + e1[c];
      T xb[D1];
#pragma unroll
      for (int r = 0; r < D1; ++r) {
        T v = mux[r];
#pragma unroll
        for (int c = 0; c < D1; ++c) if (c <= r) v += mc.Lqx[r][c] * xwm[c];
        xb[r] = v;
        a.xbb_new[((long long)i * L + m) * D1 + r] = v;
        xbs[m * D1 + r] = v;
        xw[m * D1 + r] = SQ * xwm[r];
      }
      T hx[DY], res[DY];
      h_x(mc, xb, hx);
#pragma unroll
      for (int q = 0; q < DY; ++q) res[q] = a.y_cur[q] - hx[q];
#pragma unroll
      for (int q = 0; q < DY; ++q) {
        T v = T(0);
#pragma unroll
        for (int c = 0; c < DY; ++c) if (c <= q) v += mc.LrInv[q][c] * res[c];
        cw[m * DY + q] = SQ * v;
      }
    }
    __syncthreads();
    // ---- the L x M weights (eq. weightsMC with alpha of eq. qnobar), log2 units ----
    const int tpm = a.tpm, rows = a.rows, stride = a.stride;
    for (int m0 = 0; m0 < L; m0 += rows) {
      const int m = m0 + tid / tpm;
      const int s = tid % tpm;
      T Sa = T(0), Sal = T(0);
      if (m < L) {
        T cm[DY], xm_[D1];
#pragma unroll
        for (int q = 0; q < DY; ++q) cm[q] = cw[m * DY + q];
#pragma unroll
        for (int c = 0; c < D1; ++c) xm_[c] = xw[m * D1 + c];
        T* Erow = E + m * stride;
#pragma unroll 4
        for (int k2 = s; k2 < M; k2 += tpm) {
          const T* rec = kd + k2 * REC;
          T v = rec[0];
          if (XZ) {
#pragma unroll
            for (int c = 0; c < D1; ++c) {
              const T d = xm_[c] - rec[1 + DY + c];
              v = fma(-d, d, v);
            }
            Sa += exp2_t(v);
          }
#pragma unroll
          for (int q = 0; q < DY; ++q) {
            const T d = cm[q] - rec[1 + q];
            v = fma(-d, d, v);
          }
          const T e = exp2_t(v);
          Sal += e;
          Erow[k2] = e;
        }
      }
      for (int o = tpm >> 1; o > 0; o >>= 1) {
        if (XZ) Sa += __shfl_xor_sync(FULL, Sa, o);
        Sal += __shfl_xor_sync(FULL, Sal, o);
      }
      if (m < L && s == 0) {
        rowS[m] = Sal;
        rowA[m] = XZ ? Sa : SA0;
        shS[m] = T(0);
        shA[m] = T(0);
      }
    }
    __syncthreads();
    // Rows whose sums fell below the normal range are redone with their own maxima.
    const T tiny = sizeof(T) == 4 ? T(1e-30) : T(1e-290);
    if (tid < 32) {
      int fb = 0;
      for (int m = lane; m < L; m += 32) fb |= (rowS[m] < tiny) || (XZ && rowA[m] < tiny);
      fb = __any_sync(FULL, fb);
      if (lane == 0) s_fallback = fb;
    }
    __syncthreads();
    if (s_fallback) {
      for (int m0 = 0; m0 < L; m0 += rows) {
        const int m = m0 + tid / tpm;
        const int s = tid % tpm;
        const bool need = m < L && ((rowS[m] < tiny) || (XZ && rowA[m] < tiny));
        T mxa = NEG, mxs = NEG;
        for (int pass = 0; pass < 2; ++pass) {
          T Sa = T(0), Sal = T(0);
          if (need) {
            for (int k2 = s; k2 < M; k2 += tpm) {
              const T* rec = kd + k2 * REC;
              T v = rec[0];
              if (XZ) {
#pragma unroll
                for (int c = 0; c < D1; ++c) {
                  const T d = xw[m * D1 + c] - rec[1 + DY + c];
                  v = fma(-d, d, v);
                }
              }
              T vl = v;
#pragma unroll
              for (int q = 0; q < DY; ++q) {
                const T d = cw[m * DY + q] - rec[1 + q];
                vl = fma(-d, d, vl);
              }
              if (pass == 0) {
                mxa = fmax(mxa, v);
                mxs = fmax(mxs, vl);
              } else {
                if (XZ) Sa += exp2_t(v - mxa);
                const T e = exp2_t(vl - mxs);
                Sal += e;
                E[m * stride + k2] = e;
              }
            }
          }
          for (int o = tpm >> 1; o > 0; o >>= 1) {
            if (pass == 0) {
              mxa = fmax(mxa, __shfl_xor_sync(FULL, mxa, o));
              mxs = fmax(mxs, __shfl_xor_sync(FULL, mxs, o));
            } else {
              Sa += __shfl_xor_sync(FULL, Sa, o);
              Sal += __shfl_xor_sync(FULL, Sal, o);
            }
          }
          if (pass == 1 && need && s == 0) {
            rowS[m] = Sal;
            shS[m] = mxs;
            if (XZ) {
              rowA[m] = Sa;
              shA[m] = mxa;
            }
          }
        }
      }
      __syncthreads();
    }
    // ---- per-draw weights, the outer weight and the estimator coefficients ----
    if (tid < 32) {
      const T LN2 = (T)LN2_D;
      T lw0 = NEG, lw1 = NEG;
      if (lane < L)
        lw0 = mc.lognorm_y + LN2 * ((log2_t(rowS[lane]) + shS[lane]) - (log2_t(rowA[lane]) + shA[lane]));
      if (lane + 32 < L)
        lw1 = mc.lognorm_y + LN2 * ((log2_t(rowS[lane + 32]) + shS[lane + 32]) -
                                    (log2_t(rowA[lane + 32]) + shA[lane + 32]));
      if (lane < L) a.lwh_new[i * L + lane] = lw0;
      if (lane + 32 < L) a.lwh_new[i * L + lane + 32] = lw1;
      const T mx = warp_max(fmax(lw0, lw1));
      const T p0 = lane < L ? exp_t<T>(lw0 - mx) : T(0);
      const T p1 = lane + 32 < L ? exp_t<T>(lw1 - mx) : T(0);
      const T ps = warp_sum(p0 + p1);
      const T lwi = mx + log_t(ps) - log_t((T)L);
      if (lane < L) coef[lane] = p0 / ps / rowS[lane];
      if (lane + 32 < L) coef[lane + 32] = p1 / ps / rowS[lane + 32];
      // the x part of the filtered mean: every reduction first, then the stores (a store
      // through a generic pointer between them held up the next reduction's loads)
      T xmv[D1];
#pragma unroll
      for (int c = 0; c < D1; ++c) {
        T v = (lane < L ? p0 * xbs[lane * D1 + c] : T(0)) +
              (lane + 32 < L ? p1 * xbs[(lane + 32) * D1 + c] : T(0));
        xmv[c] = warp_sum(v) / ps;
      }
      if (lane == 0) {
#pragma unroll
        for (int c = 0; c < D1; ++c) a.xm[(long long)c * N + i] = xmv[c];
      }
      if (lane == 0) {
        a.lw[i] = lwi;
        if (lwi != lwi) atomicOr(a.err, ERR_NUMERIC);
        const unsigned long long key = order_key(lwi);
        if (lwi == lwi && key > *(volatile unsigned long long*)a.lwmax_key)
          atomicMax(a.lwmax_key, key);
      }
    }
    __syncthreads();
    // ---- z part: beta_k = sum_m coef_m E[m][k]; z-mean = A_zx x + A_zz sum beta z + K sum beta ep ----
    if constexpr (D2 > 32) {
      // wide z: beta to shared memory (the records are no longer read), the z sums one warp
      // a column over the stage's z rows, the DY noise sums over the warps, then one warp a
      // row of [A_zz K] . sums
      T* sbeta = kd;
      T* sbs = (T*)(smem_raw + a.off_sb);
      const T* zmat = (const T*)(smem_raw + a.off_zmat);
      const int w = tid >> 5, nw = NT >> 5;
      T acc[DY];
#pragma unroll
      for (int q = 0; q < DY; ++q) acc[q] = T(0);
#pragma unroll
      for (int p = 0; p < PPT; ++p) {
        const int j = tid + p * NT;
        if (j < M) {
          T beta = T(0);
          for (int m = 0; m < L; ++m) beta += coef[m] * E[m * stride + j];
          sbeta[j] = beta;
#pragma unroll
          for (int q = 0; q < DY; ++q) acc[q] += beta * ep[p][q];
        }
      }
#pragma unroll
      for (int q = 0; q < DY; ++q) acc[q] = warp_sum(acc[q]);
      if (lane == 0) {
#pragma unroll
        for (int q = 0; q < DY; ++q) part[q * 32 + w] = acc[q];
      }
      __syncthreads();
      constexpr int CPW = 8;  // columns (rows below) a warp sums side by side
      for (int c0 = w; c0 < D2; c0 += nw * CPW) {
        T v[CPW];
#pragma unroll
        for (int u = 0; u < CPW; ++u) v[u] = T(0);
        for (int k2 = lane; k2 < M; k2 += 32) {
          const T bk = sbeta[k2];
#pragma unroll
          for (int u = 0; u < CPW; ++u)
            if (c0 + u * nw < D2) v[u] += bk * zsrc[(c0 + u * nw) * M + k2];
        }
#pragma unroll
        for (int u = 0; u < CPW; ++u) v[u] = warp_sum(v[u]);
        if (lane == 0) {
#pragma unroll
          for (int u = 0; u < CPW; ++u)
            if (c0 + u * nw < D2) sbs[c0 + u * nw] = v[u];
        }
      }
      if (tid < DY) {
        T v = T(0);
        for (int q = 0; q < nw; ++q) v += part[tid * 32 + q];
        sbs[D2 + tid] = v;
      }
      __syncthreads();
      for (int r0 = w; r0 < D2; r0 += nw * CPW) {
        T v[CPW];
#pragma unroll
        for (int u = 0; u < CPW; ++u) v[u] = T(0);
        for (int c = lane; c < D2 + DY; c += 32) {
          const T sc = sbs[c];
#pragma unroll
          for (int u = 0; u < CPW; ++u)
            if (r0 + u * nw < D2) v[u] += zmat[(r0 + u * nw) * (D2 + DY) + c] * sc;
        }
#pragma unroll
        for (int u = 0; u < CPW; ++u) v[u] = warp_sum(v[u]);
        if (lane == 0) {
#pragma unroll
          for (int u = 0; u < CPW; ++u) {
            const int r = r0 + u * nw;
            if (r < D2) {
              T zv = v[u];
#pragma unroll
              for (int c = 0; c < D1; ++c) zv += mc.Azx[r][c] * x[c];
              a.zm[(long long)r * N + i] = zv;
            }
          }
        }
      }
      __syncthreads();  // the stage and the work buffers are free for the next group
      if (PF && !pf_issued && tid < 32 && g + gridDim.x < G)
        stage_group<T, D1, D2, true, true>(a, stage0, &bars[0], source_of(g + gridDim.x));
    } else {
      T acc[D2 + DY];
#pragma unroll
      for (int c = 0; c < D2 + DY; ++c) acc[c] = T(0);
#pragma unroll
      for (int p = 0; p < PPT; ++p) {
        const int j = tid + p * NT;
        if (j < M) {
          T beta = T(0);
          for (int m = 0; m < L; ++m) beta += coef[m] * E[m * stride + j];
#pragma unroll
          for (int c = 0; c < D2; ++c) acc[c] += beta * zr[p][c];
#pragma unroll
          for (int q = 0; q < DY; ++q) acc[D2 + q] += beta * ep[p][q];
        }
      }
#pragma unroll
      for (int c = 0; c < D2 + DY; ++c) acc[c] = warp_sum(acc[c]);
      const int w = tid >> 5, nw = NT >> 5;
      if (lane == 0) {
#pragma unroll
        for (int c = 0; c < D2 + DY; ++c) part[c * 32 + w] = acc[c];
      }
      __syncthreads();
      if (tid < D2) {
        const int r = tid;
        T sb[D2 + DY];
#pragma unroll
        for (int c = 0; c < D2 + DY; ++c) {
          T v = T(0);
          for (int q = 0; q < nw; ++q) v += part[c * 32 + q];
          sb[c] = v;
        }
        T v = T(0);
#pragma unroll
        for (int c = 0; c < D1; ++c) v += mc.Azx[r][c] * x[c];
#pragma unroll
        for (int c = 0; c < D2; ++c) v += mc.Azz[r][c] * sb[c];
#pragma unroll
        for (int q = 0; q < DY; ++q) v += mc.K[r][q] * sb[D2 + q];
        a.zm[(long long)r * N + i] = v;
      }
      __syncthreads();  // the stage and the work buffers are free for the next group
      if (PF && !pf_issued && tid < 32 && g + gridDim.x < G)
        stage_group<T, D1, D2, true, true>(a, stage0, &bars[0], source_of(g + gridDim.x));
    }
  }
  if constexpr (TC) {
    tc::fence_before();
    __syncthreads();
    if (tid < 32) tc::tmem_dealloc(taddr, TC_COLS);
  }
}

// The block step with the model constants as a launch parameter.
template <typename T, int D1, int D2, int DY, bool XZ, int PPT, int MAXNT, bool BULK>
__global__ void __launch_bounds__(MAXNT)
    step_kernel(const __grid_constant__ MC<T, D1, D2, DY> mc, const __grid_constant__ StepArgs<T> a) {
  step_body<T, D1, D2, DY, XZ, PPT, BULK, false>(mc, a);
}


// ---- the outer stage's inputs and outputs: evidence, ESS, filtered mean, quantised total ----
template <typename T>
struct OuterArgs {
  const T* lw;
  const T* xm;
  const T* zm;
  long long N;
  int d1, d2;
  unsigned long long* lwmax_key;
  T* lwmax_t;
  unsigned long long* Csum;
  unsigned int* done;
  double* partials;  // one row of 2 + d sums a CTA
  double* stats;     // [logZ_total, logZ_step, ess, s1, mean[d]]
  const int* perm;   // device, d
  double* mean_out;  // optional device outputs
  double* logz_out;
  int* err;
};

}  // namespace dpf
