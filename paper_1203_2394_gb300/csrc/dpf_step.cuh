// The LA-DPF step kernels.
//
// One call t runs three kernels on the context's stream:
//  1. step_kernel (one CTA per outer particle i): the deferred inner step of
//     step t-1 for destination i (the selection of x_{t-1} among the
//     ancestor's look-ahead draws, local systematic resampling of the
//     ancestor's inner set, propagation and the y_{t-1} update of the inner
//     weights; Fig. 4 step 4, DPF step 6, eq. qbar), then the look-ahead of step
//     t on the fresh inner set held in shared memory (Fig. 4 steps 1-2, eqs.
//     approx1, qnobar, weightsMC). The inner set is read once and written once.
//  2. outer_reduce_kernel: evidence, ESS, the filtered mean and the quantised
//     total C of the outer weights (eq. weightsopt).
//  3. global_scan_scatter: global systematic resampling of the outer set
//     (Fig. 4 step 3) with a single-pass decoupled look-back scan.
//
// Device layout (structure of arrays, element type T):
//   z[c][n][j] (d2 x N x M), lq[n][j], x[c][n] (d1 x N)   two slots each
//   lwh[n][m], xbb[n][m][c]                               two slots each
//   lw[n], xm[c][n], zm[c][n], wout[n], anc[n], sel[n]
// Slot parity: after call t the materialised state of step t-1 sits in slot
// (t-1) % 2 and the look-ahead products of step t in slot t % 2.
#pragma once

#include "dpf_common.cuh"
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
  T Hx[DY][D1], Hz[DY][D2], LrInv[DY][DY];
  T HzAzz[DY][D2], HzAzx[DY][D1], Ls[DY][DY];
  T K[D2][DY];     // Q_z H_z^T (H_z Q_z H_z^T)^{-1}
  T m0x[D1], m0z[D2], Lp0x[D1][D1], G0[D2][D1], Lp0c[D2][D2];
  T ga, gb, qc, lognorm_y;
  int growth, quad;
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
};

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
__host__ __device__ inline int rows_tpm(int nt, int L) {
  int tpm = 1;
  while (tpm * 2 <= 32 && tpm * 2 * L <= nt) tpm *= 2;
  return tpm;
}

// Shared-memory carve-up of step_kernel (bytes), identical on host and device.
struct StepSmem {
  size_t zs, cum, ft, gt, lqs, E, xt, ct, xbs, rowS, rowA, shS, shA, coef, red, redU, part, total;
  int stride;
};
template <typename T, int D1, int D2, int DY>
__host__ __device__ inline StepSmem step_smem(int M, int L, int nt) {
  StepSmem s;
  const int tpm = rows_tpm(nt, L);
  int stride = M;
  while (stride % 32 != tpm % 32) ++stride;
  s.stride = stride;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (bytes + 15) & ~(size_t)15;
    return at;
  };
  s.zs = take(sizeof(T) * D2 * M);
  s.cum = take(sizeof(uint32_t) * M);
  s.ft = take(sizeof(T) * D1 * M);
  s.gt = take(sizeof(T) * DY * M);
  s.lqs = take(sizeof(T) * M);
  s.E = take(sizeof(T) * (size_t)L * stride);
  s.xt = take(sizeof(T) * L * D1);
  s.ct = take(sizeof(T) * L * DY);
  s.xbs = take(sizeof(T) * L * D1);
  s.rowS = take(sizeof(T) * L);
  s.rowA = take(sizeof(T) * L);
  s.shS = take(sizeof(T) * L);
  s.shA = take(sizeof(T) * L);
  s.coef = take(sizeof(T) * L);
  s.red = take(sizeof(T) * 32);
  s.redU = take(sizeof(uint32_t) * 32);
  s.part = take(sizeof(T) * 32 * (D2 + DY + 1));
  s.total = o;
  return s;
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
__global__ void init_kernel(const __grid_constant__ MC<T, D1, D2, DY> mc, T* z, T* lq, T* x,
                            long long N, int M, Key key) {
  const long long i = blockIdx.x;
  const int j = threadIdx.x;
  if (j >= M) return;
  T e1[D1], xi[D1];
  normals<D1>(key, 0u, (uint32_t)i, P_INIT_X, 0u, e1);
#pragma unroll
  for (int r = 0; r < D1; ++r) {
    T v = mc.m0x[r];
#pragma unroll
    for (int c = 0; c <= r; ++c) v += mc.Lp0x[r][c] * e1[c];
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
    for (int c = 0; c <= r; ++c) v += mc.Lp0c[r][c] * e2[c];
    z[((long long)r * N + i) * M + j] = v;
  }
  lq[i * M + j] = -log_t((T)M);
  if (j == 0) {
#pragma unroll
    for (int r = 0; r < D1; ++r) x[(long long)r * N + i] = xi[r];
  }
}

template <typename T, int D1, int D2, int DY, bool XZ, int MAXNT>
__global__ void __launch_bounds__(MAXNT)
    step_kernel(const __grid_constant__ MC<T, D1, D2, DY> mc, const __grid_constant__ StepArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NT = blockDim.x;
  const int M = a.M, L = a.L;
  const long long N = a.N;
  const StepSmem lay = step_smem<T, D1, D2, DY>(M, L, NT);
  T* zs = (T*)(smem_raw + lay.zs);
  uint32_t* cum = (uint32_t*)(smem_raw + lay.cum);
  T* ft = (T*)(smem_raw + lay.ft);
  T* gt = (T*)(smem_raw + lay.gt);
  T* lqs = (T*)(smem_raw + lay.lqs);
  T* E = (T*)(smem_raw + lay.E);
  T* xt = (T*)(smem_raw + lay.xt);
  T* ct = (T*)(smem_raw + lay.ct);
  T* xbs = (T*)(smem_raw + lay.xbs);
  T* rowS = (T*)(smem_raw + lay.rowS);
  T* rowA = (T*)(smem_raw + lay.rowA);
  T* shS = (T*)(smem_raw + lay.shS);
  T* shA = (T*)(smem_raw + lay.shA);
  T* coef = (T*)(smem_raw + lay.coef);
  T* red = (T*)(smem_raw + lay.red);
  uint32_t* redU = (uint32_t*)(smem_raw + lay.redU);
  T* part = (T*)(smem_raw + lay.part);
  __shared__ int s_m;
  __shared__ int s_fallback;

  const long long i = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31;
  const int j = tid;
  const bool act = j < M;
  const T NEG = neg_inf<T>();
  if (i == 0 && tid == 0) *a.Csum = 0ull;

  T x[D1];     // x_{t-1}^(i): the group's outer particle
  T zr[D2];    // this thread's inner particle z_{t-1}^(i,j)
  T lqr = NEG; // and its normalised log-weight

  if (a.first) {
#pragma unroll
    for (int c = 0; c < D1; ++c) x[c] = a.x_old[(long long)c * N + i];
    if (act) {
#pragma unroll
      for (int c = 0; c < D2; ++c) zr[c] = a.z_old[((long long)c * N + i) * M + j];
      lqr = a.lq_old[i * M + j];
    }
  } else {
    // ---- selection of x_{t-1}^(i) among the ancestor's look-ahead draws ----
    const int anc = a.anc[i];
    if (tid < 32) {
      const T l0 = lane < L ? a.lwh_old[(long long)anc * L + lane] : NEG;
      const T l1 = lane + 32 < L ? a.lwh_old[(long long)anc * L + lane + 32] : NEG;
      const T mx = warp_max(fmax(l0, l1));
      const int shift = 31 - ceil_log2_i(L);
      const uint32_t c0 = lane < L ? quantize_u32(exp_t<T>(l0 - mx), shift) : 0u;
      const uint32_t c1 = lane + 32 < L ? quantize_u32(exp_t<T>(l1 - mx), shift) : 0u;
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
      const uint32_t u = rand_word(a.key, a.t - 1, (uint32_t)i, P_SEL, 0u);
      const uint64_t rhs = (uint64_t)u * C;
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
    }
    __syncthreads();
    const int msel = s_m;
    T xa[D1];
#pragma unroll
    for (int c = 0; c < D1; ++c) {
      x[c] = a.xbb_old[((long long)anc * L + msel) * D1 + c];
      xa[c] = a.x_old[(long long)c * N + anc];
    }
    // ---- local resampling of the ancestor's inner set (eq. qnobar weights) ----
    T za[D2];
    T alpha = NEG;
    if (act) {
#pragma unroll
      for (int c = 0; c < D2; ++c) {
        za[c] = a.z_old[((long long)c * N + anc) * M + j];
        zs[c * M + j] = za[c];
      }
      alpha = a.lq_old[(long long)anc * M + j];
      if (XZ) {
        T mxa[D1];
        mu_x(mc, xa, a.gcos_prev, mxa);
        T q = T(0);
#pragma unroll
        for (int r = 0; r < D1; ++r) {
          T v = T(0);
#pragma unroll
          for (int c = 0; c <= r; ++c) v += mc.LqxInv[r][c] * (x[c] - mxa[c]);
#pragma unroll
          for (int c = 0; c < D2; ++c) v -= mc.WAxz[r][c] * za[c];
          q += v * v;
        }
        alpha -= T(0.5) * q;
      }
    }
    const T amax = bmax(alpha, red);
    const int shiftM = 31 - ceil_log2_i(M);
    const uint32_t cw = act ? quantize_u32(exp_t<T>(alpha - amax), shiftM) : 0u;
    const uint32_t incl = bscan_u32(cw, redU);
    if (act) cum[j] = incl;
    __syncthreads();
    // ---- propagation and y_{t-1} update (eq. qbar) ----
    T ell = NEG;
    if (act) {
      const uint32_t C = cum[M - 1];
      const uint32_t u = rand_word(a.key, a.t - 1, (uint32_t)i, P_INNER, 0u);
      const int b = sys_local_pick(cum, M, C, M, j, u);
      if (a.dbg_b) a.dbg_b[i * M + j] = b;
      T eps[D2];
      normals<D2>(a.key, a.t - 1, (uint32_t)i, P_PROP, (uint32_t)j, eps);
#pragma unroll
      for (int r = 0; r < D2; ++r) {
        T v = T(0);
#pragma unroll
        for (int c = 0; c < D1; ++c) v += mc.Azx[r][c] * xa[c];
#pragma unroll
        for (int c = 0; c < D2; ++c) v += mc.Azz[r][c] * zs[c * M + b];
#pragma unroll
        for (int c = 0; c <= r; ++c) v += mc.Lqz[r][c] * eps[c];
        zr[r] = v;
      }
      T hx[DY], res[DY];
      h_x(mc, x, hx);
#pragma unroll
      for (int q = 0; q < DY; ++q) {
        T v = a.y_prev[q] - hx[q];
#pragma unroll
        for (int c = 0; c < D2; ++c) v -= mc.Hz[q][c] * zr[c];
        res[q] = v;
      }
      T qf = T(0);
#pragma unroll
      for (int q = 0; q < DY; ++q) {
        T v = T(0);
#pragma unroll
        for (int c = 0; c <= q; ++c) v += mc.LrInv[q][c] * res[c];
        qf += v * v;
      }
      ell = T(-0.5) * qf;
    }
    const T lmax = bmax(ell, red);
    const T lsum = bsum(act ? exp_t<T>(ell - lmax) : T(0), red);
    if (act) {
      lqr = ell - lmax - log_t(lsum);
#pragma unroll
      for (int c = 0; c < D2; ++c) a.z_new[((long long)c * N + i) * M + j] = zr[c];
      a.lq_new[i * M + j] = lqr;
    }
    if (tid == 0) {
#pragma unroll
      for (int c = 0; c < D1; ++c) a.x_new[(long long)c * N + i] = x[c];
    }
  }

  // ======== look-ahead of step t from (x, z, lq) with y_t ========
  T ep[DY];  // projected look-ahead noise Ls eps of this inner particle
  if (act) {
    lqs[j] = lqr;
    if (XZ) {
#pragma unroll
      for (int r = 0; r < D1; ++r) {
        T v = T(0);
#pragma unroll
        for (int c = 0; c < D2; ++c) v += mc.WAxz[r][c] * zr[c];
        ft[r * M + j] = v;
      }
    }
    T e2[DY];
    normals<DY>(a.key, a.t, (uint32_t)i, P_LA_Z, (uint32_t)j, e2);
    T g[DY];
#pragma unroll
    for (int q = 0; q < DY; ++q) {
      T e = T(0);
#pragma unroll
      for (int c = 0; c <= q; ++c) e += mc.Ls[q][c] * e2[c];
      ep[q] = e;
      T v = e;
#pragma unroll
      for (int c = 0; c < D1; ++c) v += mc.HzAzx[q][c] * x[c];
#pragma unroll
      for (int c = 0; c < D2; ++c) v += mc.HzAzz[q][c] * zr[c];
      g[q] = v;
    }
#pragma unroll
    for (int q = 0; q < DY; ++q) {
      T v = T(0);
#pragma unroll
      for (int c = 0; c <= q; ++c) v += mc.LrInv[q][c] * g[c];
      gt[q * M + j] = v;
    }
  }
  // the shift of every exponent: the largest inner log-weight
  const T sigma = bmax(lqr, red);
  const T w_lq = act ? exp_t<T>(lqr - sigma) : T(0);
  T SA0 = T(0);
  if (!XZ) SA0 = bsum(w_lq, red);
  if (XZ) {  // categorical draws of the mixture components need the cumulative weights
    const uint32_t cw = act ? quantize_u32(w_lq, 31 - ceil_log2_i(M)) : 0u;
    const uint32_t incl = bscan_u32(cw, redU);
    if (act) cum[j] = incl;
  }
  __syncthreads();
  // ---- L look-ahead draws xbb^(m) (eq. approx1) ----
  T mux[D1];
  mu_x(mc, x, a.gcos_cur, mux);
  for (int m = tid; m < L; m += NT) {
    T e1[D1], xw[D1];
    normals<D1>(a.key, a.t, (uint32_t)i, P_LA_X, (uint32_t)m, e1);
    int jm = 0;
    if (XZ) jm = sys_local_pick(cum, M, cum[M - 1], 1, 0, rand_word(a.key, a.t, (uint32_t)i, P_LA_J, (uint32_t)m));
#pragma unroll
    for (int c = 0; c < D1; ++c) xw[c] = (XZ ? ft[c * M + jm] : T(0)) + e1[c];
    T xb[D1];
#pragma unroll
    for (int r = 0; r < D1; ++r) {
      T v = mux[r];
#pragma unroll
      for (int c = 0; c <= r; ++c) v += mc.Lqx[r][c] * xw[c];
      xb[r] = v;
      a.xbb_new[((long long)i * L + m) * D1 + r] = v;
      xbs[m * D1 + r] = v;
      xt[m * D1 + r] = xw[r];
    }
    T hx[DY];
    h_x(mc, xb, hx);
    T res[DY];
#pragma unroll
    for (int q = 0; q < DY; ++q) res[q] = a.y_cur[q] - hx[q];
#pragma unroll
    for (int q = 0; q < DY; ++q) {
      T v = T(0);
#pragma unroll
      for (int c = 0; c <= q; ++c) v += mc.LrInv[q][c] * res[c];
      ct[m * DY + q] = v;
    }
  }
  __syncthreads();
  // ---- the L x M weights (eq. weightsMC, alpha of eq. qnobar) ----
  const int tpm = rows_tpm(NT, L);
  const int rows = NT / tpm;
  const int stride = lay.stride;
  for (int m0 = 0; m0 < L; m0 += rows) {
    const int m = m0 + tid / tpm;
    const int s = tid % tpm;
    T Sa = T(0), Sal = T(0);
    if (m < L) {
      T cm[DY], xm_[D1];
#pragma unroll
      for (int q = 0; q < DY; ++q) cm[q] = ct[m * DY + q];
#pragma unroll
      for (int c = 0; c < D1; ++c) xm_[c] = xt[m * D1 + c];
      for (int k = s; k < M; k += tpm) {
        T v = lqs[k] - sigma;
        if (XZ) {
          T q = T(0);
#pragma unroll
          for (int c = 0; c < D1; ++c) {
            const T d = xm_[c] - ft[c * M + k];
            q += d * d;
          }
          v -= T(0.5) * q;
          Sa += exp_t<T>(v);
        }
        T q2 = T(0);
#pragma unroll
        for (int c = 0; c < DY; ++c) {
          const T d = cm[c] - gt[c * M + k];
          q2 += d * d;
        }
        const T e = exp_t<T>(v - T(0.5) * q2);
        Sal += e;
        E[m * stride + k] = e;
      }
    }
    for (int o = tpm >> 1; o > 0; o >>= 1) {
      Sa += __shfl_xor_sync(FULL, Sa, o);
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
  if (tid == 0) {
    int fb = 0;
    for (int m = 0; m < L; ++m) fb |= (rowS[m] < tiny) || (XZ && rowA[m] < tiny);
    s_fallback = fb;
  }
  __syncthreads();
  if (s_fallback) {
    for (int m0 = 0; m0 < L; m0 += rows) {
      const int m = m0 + tid / tpm;
      const int s = tid % tpm;
      const bool need = m < L && ((rowS[m] < tiny) || (XZ && rowA[m] < tiny));
      T mxa = NEG, mxs = NEG;
      if (need) {
        for (int k = s; k < M; k += tpm) {
          T v = lqs[k] - sigma;
          if (XZ) {
            T q = T(0);
#pragma unroll
            for (int c = 0; c < D1; ++c) {
              const T d = xt[m * D1 + c] - ft[c * M + k];
              q += d * d;
            }
            v -= T(0.5) * q;
          }
          T q2 = T(0);
#pragma unroll
          for (int c = 0; c < DY; ++c) {
            const T d = ct[m * DY + c] - gt[c * M + k];
            q2 += d * d;
          }
          mxa = fmax(mxa, v);
          mxs = fmax(mxs, v - T(0.5) * q2);
        }
      }
      for (int o = tpm >> 1; o > 0; o >>= 1) {
        mxa = fmax(mxa, __shfl_xor_sync(FULL, mxa, o));
        mxs = fmax(mxs, __shfl_xor_sync(FULL, mxs, o));
      }
      T Sa = T(0), Sal = T(0);
      if (need) {
        for (int k = s; k < M; k += tpm) {
          T v = lqs[k] - sigma;
          if (XZ) {
            T q = T(0);
#pragma unroll
            for (int c = 0; c < D1; ++c) {
              const T d = xt[m * D1 + c] - ft[c * M + k];
              q += d * d;
            }
            v -= T(0.5) * q;
            Sa += exp_t<T>(v - mxa);
          }
          T q2 = T(0);
#pragma unroll
          for (int c = 0; c < DY; ++c) {
            const T d = ct[m * DY + c] - gt[c * M + k];
            q2 += d * d;
          }
          const T e = exp_t<T>(v - T(0.5) * q2 - mxs);
          Sal += e;
          E[m * stride + k] = e;
        }
      }
      for (int o = tpm >> 1; o > 0; o >>= 1) {
        Sa += __shfl_xor_sync(FULL, Sa, o);
        Sal += __shfl_xor_sync(FULL, Sal, o);
      }
      __syncwarp();
      if (need && s == 0) {
        rowS[m] = Sal;
        shS[m] = mxs;
        if (XZ) {
          rowA[m] = Sa;
          shA[m] = mxa;
        }
      }
    }
    __syncthreads();
  }
  // ---- per-draw weights, the outer weight and the estimator coefficients ----
  if (tid < 32) {
    T lw0 = NEG, lw1 = NEG;
    if (lane < L)
      lw0 = mc.lognorm_y + (log_t(rowS[lane]) + shS[lane]) - (log_t(rowA[lane]) + shA[lane]);
    if (lane + 32 < L)
      lw1 = mc.lognorm_y + (log_t(rowS[lane + 32]) + shS[lane + 32]) -
            (log_t(rowA[lane + 32]) + shA[lane + 32]);
    if (lane < L) a.lwh_new[i * L + lane] = lw0;
    if (lane + 32 < L) a.lwh_new[i * L + lane + 32] = lw1;
    const T mx = warp_max(fmax(lw0, lw1));
    const T p0 = lane < L ? exp_t<T>(lw0 - mx) : T(0);
    const T p1 = lane + 32 < L ? exp_t<T>(lw1 - mx) : T(0);
    const T ps = warp_sum(p0 + p1);
    const T lwi = mx + log_t(ps) - log_t((T)L);
    if (lane < L) coef[lane] = p0 / ps / rowS[lane];
    if (lane + 32 < L) coef[lane + 32] = p1 / ps / rowS[lane + 32];
    // x part of the filtered mean
#pragma unroll
    for (int c = 0; c < D1; ++c) {
      T v = (lane < L ? p0 * xbs[lane * D1 + c] : T(0)) +
            (lane + 32 < L ? p1 * xbs[(lane + 32) * D1 + c] : T(0));
      v = warp_sum(v) / ps;
      if (lane == 0) a.xm[(long long)c * N + i] = v;
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
  T beta = T(0);
  if (act)
    for (int m = 0; m < L; ++m) beta += coef[m] * E[m * stride + j];
  T acc[D2 + DY];
#pragma unroll
  for (int c = 0; c < D2; ++c) acc[c] = act ? beta * zr[c] : T(0);
#pragma unroll
  for (int q = 0; q < DY; ++q) acc[D2 + q] = act ? beta * ep[q] : T(0);
#pragma unroll
  for (int c = 0; c < D2 + DY; ++c) acc[c] = warp_sum(acc[c]);
  const int w = tid >> 5, nw = NT >> 5;
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < D2 + DY; ++c) part[c * 32 + w] = acc[c];
  }
  __syncthreads();
  if (tid < D2 + DY) {
    T v = T(0);
    for (int q = 0; q < nw; ++q) v += part[tid * 32 + q];
    part[tid * 32] = v;
  }
  __syncthreads();
  if (tid < D2) {
    const int r = tid;
    T v = T(0);
#pragma unroll
    for (int c = 0; c < D1; ++c) v += mc.Azx[r][c] * x[c];
#pragma unroll
    for (int c = 0; c < D2; ++c) v += mc.Azz[r][c] * part[c * 32];
#pragma unroll
    for (int q = 0; q < DY; ++q) v += mc.K[r][q] * part[(D2 + q) * 32];
    a.zm[(long long)r * N + i] = v;
  }
}

// ---- outer reduction: evidence, ESS, filtered mean, quantised total ----
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
  double* partials;  // gridDim.x x (4 + d)
  double* stats;     // [logZ_total, logZ_step, ess, s1, mean[d]]
  const int* perm;   // device, d
  double* mean_out;  // optional device outputs
  double* logz_out;
  int* err;
};

constexpr int RED_NT = 256;

template <typename T>
__global__ void __launch_bounds__(RED_NT) outer_reduce_kernel(OuterArgs<T> a) {
  __shared__ double sh[RED_NT / 32][4 + 128];
  __shared__ bool last;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int d = a.d1 + a.d2;
  T lwmax;
  order_decode(*a.lwmax_key, lwmax);
  const int S = 62 - ceil_log2_i(a.N);
  double s1 = 0, s2 = 0;
  double sm[128];
  for (int c = 0; c < d; ++c) sm[c] = 0;
  unsigned long long cc = 0;
  for (long long i = blockIdx.x * (long long)RED_NT + tid; i < a.N; i += (long long)gridDim.x * RED_NT) {
    const T W = exp_t<T>(a.lw[i] - lwmax);
    cc += quantize_u64(W, S);
    const double Wd = (double)W;
    s1 += Wd;
    s2 += Wd * Wd;
    for (int c = 0; c < a.d1; ++c) sm[c] += Wd * (double)a.xm[(long long)c * a.N + i];
    for (int c = 0; c < a.d2; ++c) sm[a.d1 + c] += Wd * (double)a.zm[(long long)c * a.N + i];
  }
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  for (int c = 0; c < d; ++c) sm[c] = warp_sum(sm[c]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cc += __shfl_xor_sync(FULL, cc, o);
  if (lane == 0) {
    sh[w][0] = s1;
    sh[w][1] = s2;
    for (int c = 0; c < d; ++c) sh[w][4 + c] = sm[c];
    if (cc) atomicAdd(a.Csum, cc);
  }
  __syncthreads();
  if (tid < 4 + d && tid != 2 && tid != 3) {
    double v = 0;
    for (int q = 0; q < RED_NT / 32; ++q) v += sh[q][tid];
    a.partials[(long long)blockIdx.x * (4 + d) + tid] = v;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) last = (atomicAdd(a.done, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (tid == 0) {
    double t1 = 0, t2 = 0;
    double mean[128];
    for (int c = 0; c < d; ++c) mean[c] = 0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
      const double* p = a.partials + (long long)b * (4 + d);
      t1 += p[0];
      t2 += p[1];
      for (int c = 0; c < d; ++c) mean[c] += p[4 + c];
    }
    const bool bad = !(lwmax > neg_inf<T>()) || lwmax != lwmax || !(t1 > 0);
    if (bad) atomicOr(a.err, ERR_NUMERIC);
    const double lz = (double)lwmax + log(t1) - log((double)a.N);
    a.stats[0] += lz;
    a.stats[1] = lz;
    a.stats[2] = t1 * t1 / t2;
    a.stats[3] = t1;
    for (int c = 0; c < d; ++c) a.stats[4 + a.perm[c]] = mean[c] / t1;
    *a.lwmax_t = lwmax;
    if (a.mean_out)
      for (int c = 0; c < d; ++c) a.mean_out[c] = a.stats[4 + c];
    if (a.logz_out) *a.logz_out = a.stats[0];
    *a.lwmax_key = 0ull;
    *a.done = 0u;
  }
}

}  // namespace dpf
