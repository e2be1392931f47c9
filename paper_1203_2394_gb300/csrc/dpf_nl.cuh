// The paper's benchmark models (Table 1), whose inner layer is nonlinear in z, with the
// LA-DPF (Fig. 4) and the bootstrap particle filter written for any model of the form
//   s_{t+1} = f(s_t, t) + v,  v ~ N(0, Q);   y_t = h(s_t) + e,  e ~ N(0, R),
// with s = (x, z). The inner draws are conditioned on x through the Gaussian noise:
// x_{t+1} | s_t ~ N(f_x, Q_xx) and z_{t+1} | x_{t+1}, s_t ~ N(f_z + G (x_{t+1} - f_x), S),
// G = Q_zx Q_xx^-1, S = Q_zz - G Q_xz. One CTA a group, one thread an inner particle; the
// look-ahead's L x M pairs are evaluated pair by pair (the inner draw depends on the
// look-ahead draw through G) into shared memory, then a warp a draw reduces both rows and
// the row's softmax-weighted inner draws. The observation is h_x(x) + h_z(z), so h_x is
// taken once a draw and, where G = 0, h_z once an inner particle. The outer stages are the
// filter's.
//
// Readings: the sine and cosine terms take the source step of the transition (as the
// growth map's cosine does); model 2's z_{2,t+1} adds z_{1,t+1}, noise included, so its z
// noise is B v_z with B = [[1, 0], [1, 1]]; s_0 ~ N(0, I) as the table states.
#pragma once

#include "dpf_step.cuh"

namespace dpf {

// Model 1 (2-dimensional): x' = x + z / (1 + z^2), z' = x + 0.5 z + 25 z / (1 + z^2) +
// 8 cos(1.2 t), y = atan(x) + z^2 / 20; Q = [[1, 0.1], [0.1, 1]], R = 1.
struct PaperModel1 {
  static constexpr int D1 = 1, D2 = 1, DY = 1, NT = 1;  // NT: time terms
  __device__ static void fx(const float (&x)[1], const float (&z)[1], const float* tt, float (&o)[1]) {
    o[0] = x[0] + z[0] / (1.f + z[0] * z[0]);
  }
  __device__ static void fz(const float (&x)[1], const float (&z)[1], const float* tt, float (&o)[1]) {
    o[0] = x[0] + 0.5f * z[0] + 25.f * z[0] / (1.f + z[0] * z[0]) + tt[0];
  }
  // y = h_x(x) + h_z(z) + e
  __device__ static float hx(const float (&x)[1]) { return atanf(x[0]); }
  __device__ static float hz(const float (&z)[1]) { return z[0] * z[0] * 0.05f; }  // z^2 / 20
  __device__ static void h(const float (&x)[1], const float (&z)[1], float (&o)[1]) { o[0] = hx(x) + hz(z); }
  static constexpr bool GZERO = false;  // the z draw depends on x_t (G != 0)
  // 8 cos(1.2 s) at the source step s (on the host, in double)
  static void terms(double s, float (&tt)[NT]) { tt[0] = (float)(8.0 * std::cos(1.2 * s)); }
  // chol(Q_xx), its inverse, G, chol(S), R^-1/2, and -1/2 log det(2 pi R)
  __host__ __device__ static constexpr float Lqx(int, int) { return 1.f; }
  __host__ __device__ static constexpr float LqxInv(int, int) { return 1.f; }
  __host__ __device__ static constexpr float G(int, int) { return 0.1f; }
  __host__ __device__ static constexpr float LS(int, int) { return 0.99498743710662f; }  // sqrt(1 - 0.1^2)
  __host__ __device__ static constexpr float LrInv(int, int) { return 1.f; }
  static constexpr float lognorm_y = -0.91893853320467f;  // -log(2 pi) / 2
};

// Model 1 decomposed the other way (Section 4.3's second action): the outer particles carry
// the table's z and the inner ones its x, so here x = z_table and z = x_table; the same
// noise covariance (symmetric in the two coordinates).
struct PaperModel1Swap {
  static constexpr int D1 = 1, D2 = 1, DY = 1, NT = 1;
  __device__ static void fx(const float (&x)[1], const float (&z)[1], const float* tt, float (&o)[1]) {
    o[0] = z[0] + 0.5f * x[0] + 25.f * x[0] / (1.f + x[0] * x[0]) + tt[0];
  }
  __device__ static void fz(const float (&x)[1], const float (&z)[1], const float* tt, float (&o)[1]) {
    o[0] = z[0] + x[0] / (1.f + x[0] * x[0]);
  }
  __device__ static float hx(const float (&x)[1]) { return x[0] * x[0] * 0.05f; }
  __device__ static float hz(const float (&z)[1]) { return atanf(z[0]); }
  __device__ static void h(const float (&x)[1], const float (&z)[1], float (&o)[1]) { o[0] = hx(x) + hz(z); }
  static constexpr bool GZERO = false;
  static void terms(double s, float (&tt)[NT]) { tt[0] = (float)(8.0 * std::cos(1.2 * s)); }
  __host__ __device__ static constexpr float Lqx(int, int) { return 1.f; }
  __host__ __device__ static constexpr float LqxInv(int, int) { return 1.f; }
  __host__ __device__ static constexpr float G(int, int) { return 0.1f; }
  __host__ __device__ static constexpr float LS(int, int) { return 0.99498743710662f; }
  __host__ __device__ static constexpr float LrInv(int, int) { return 1.f; }
  static constexpr float lognorm_y = -0.91893853320467f;
};

// Model 2 (4-dimensional): x1' = 0.5 x1 + 8 sin t, x2' = 0.4 x1 + 0.5 x2, z1' = z1 + z2 /
// (1 + z2^2), z2' = z1' + 0.5 z2 + 25 z2 / (1 + z2^2) + 8 cos(1.2 t),
// y = (x1 + x2) / (1 + x1^2) + atan(z1) + z2^2 / 20; the noise of x is N(0, I), of
// (z1, z2) before the composition N(0, [[1, 0.1], [0.1, 10]]), R = 1.
struct PaperModel2 {
  static constexpr int D1 = 2, D2 = 2, DY = 1, NT = 2;
  __device__ static void fx(const float (&x)[2], const float (&z)[2], const float* tt, float (&o)[2]) {
    o[0] = 0.5f * x[0] + tt[0];
    o[1] = 0.4f * x[0] + 0.5f * x[1];
  }
  __device__ static void fz(const float (&x)[2], const float (&z)[2], const float* tt, float (&o)[2]) {
    const float z1 = z[0] + z[1] / (1.f + z[1] * z[1]);
    o[0] = z1;
    o[1] = z1 + 0.5f * z[1] + 25.f * z[1] / (1.f + z[1] * z[1]) + tt[1];
  }
  __device__ static float hx(const float (&x)[2]) { return (x[0] + x[1]) / (1.f + x[0] * x[0]); }
  __device__ static float hz(const float (&z)[2]) { return atanf(z[0]) + z[1] * z[1] * 0.05f; }
  __device__ static void h(const float (&x)[2], const float (&z)[2], float (&o)[1]) { o[0] = hx(x) + hz(z); }
  static constexpr bool GZERO = true;  // x and z noises independent: the z draw is free of x_t
  static void terms(double s, float (&tt)[NT]) {
    tt[0] = (float)(8.0 * std::sin(s));
    tt[1] = (float)(8.0 * std::cos(1.2 * s));
  }
  __host__ __device__ static constexpr float Lqx(int r, int c) { return r == c ? 1.f : 0.f; }
  __host__ __device__ static constexpr float LqxInv(int r, int c) { return r == c ? 1.f : 0.f; }
  __host__ __device__ static constexpr float G(int, int) { return 0.f; }
  // chol([[1, 1.1], [1.1, 11.2]]): the covariance of B v_z (sqrt(11.2 - 1.21) = 3.1607)
  __host__ __device__ static constexpr float LS(int r, int c) {
    return r == 0 ? (c == 0 ? 1.f : 0.f) : (c == 0 ? 1.1f : 3.16069612585582f);
  }
  __host__ __device__ static constexpr float LrInv(int, int) { return 1.f; }
  static constexpr float lognorm_y = -0.91893853320467f;
};

struct NLArgs {
  const float* z_old;
  const float* lq_old;
  const float* x_old;
  float* z_new;
  float* lq_new;
  float* x_new;
  const float* lwh_old;
  const float* xbb_old;
  float* lwh_new;
  float* xbb_new;
  const int32_t* anc;
  int32_t* sel;
  float* lw;
  float* xm;
  float* zm;
  const float* y_prev;
  const float* y_cur;
  unsigned long long* lwmax_key;
  unsigned long long* Csum;
  int* err;
  long long N;
  int M, L, xp;
  uint32_t t;
  Key key;
  float tt_prev[2];  // the model's time terms of the transition into step t-1
  float tt_cur[2];   // ... into step t
  float scaleM, scaleL, logL;
  int first;
  int32_t* dbg_b;  // debug (or null): the local resampling indices of the inner update, N x M
  int32_t* dbg_j;  // debug (or null): the mixture component of each look-ahead draw, N x L
};

// log N(r; 0, Q_xx) up to the constant: -|L_qx^-1 r|^2 / 2
template <class Mod>
__device__ __forceinline__ float nl_quad_x(const float (&r)[Mod::D1]) {
  float q = 0.f;
#pragma unroll
  for (int a = 0; a < Mod::D1; ++a) {
    float v = 0.f;
#pragma unroll
    for (int c = 0; c < Mod::D1; ++c)
      if (c <= a) v += Mod::LqxInv(a, c) * r[c];
    q += v * v;
  }
  return -0.5f * q;
}

template <class Mod>
__device__ __forceinline__ float nl_loglik(const float (&x)[Mod::D1], const float (&z)[Mod::D2], const float* y) {
  float hv[Mod::DY], r[Mod::DY];
  Mod::h(x, z, hv);
#pragma unroll
  for (int q = 0; q < Mod::DY; ++q) r[q] = y[q] - hv[q];
  float qf = 0.f;
#pragma unroll
  for (int a = 0; a < Mod::DY; ++a) {
    float v = 0.f;
#pragma unroll
    for (int c = 0; c < Mod::DY; ++c)
      if (c <= a) v += Mod::LrInv(a, c) * r[c];
    qf += v * v;
  }
  return Mod::lognorm_y - 0.5f * qf;
}

// z' = f_z + G (x' - f_x) + chol(S) e
template <class Mod>
__device__ __forceinline__ void nl_zdraw(const float (&fzv)[Mod::D2], const float (&fxv)[Mod::D1],
                                         const float (&xn)[Mod::D1], const float (&e)[Mod::D2],
                                         float (&zn)[Mod::D2]) {
#pragma unroll
  for (int r = 0; r < Mod::D2; ++r) {
    float v = fzv[r];
#pragma unroll
    for (int c = 0; c < Mod::D1; ++c) v += Mod::G(r, c) * (xn[c] - fxv[c]);
#pragma unroll
    for (int c = 0; c < Mod::D2; ++c)
      if (c <= r) v += Mod::LS(r, c) * e[c];
    zn[r] = v;
  }
}

// Initial draw (s_0 ~ N(0, I)): x_0 from the normals (0, i, INIT_X, 0), z_0^(i,j) from
// (0, i, INIT_Z, j), lq = -log M. One CTA a group.
template <class Mod>
__global__ void nl_init_kernel(float* z, float* lq, float* x, long long N, int M, int xp, Key key) {
  const long long i = blockIdx.x;
  const long long NM = N * (long long)M;
  if (threadIdx.x == 0) {
    float e[Mod::D1];
    normals<Mod::D1>(key, 0u, (uint32_t)i, P_INIT_X, 0u, e);
    for (int c = 0; c < xp; ++c) x[i * xp + c] = c < Mod::D1 ? e[c < Mod::D1 ? c : 0] : 0.f;
  }
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    float e[Mod::D2];
    normals<Mod::D2>(key, 0u, (uint32_t)i, P_INIT_Z, (uint32_t)j, e);
#pragma unroll
    for (int c = 0; c < Mod::D2; ++c) z[c * NM + i * M + j] = e[c];
    lq[i * M + j] = -logf((float)M);
  }
}

// Bytes of shared memory of nl_step_kernel: the group's per-inner-particle arrays (z, lq,
// f_x, the draw's base, h_z), the two L x M pair arrays, the per-draw arrays (two draws of
// d1, h_x, the ancestor's weights, the two row log-sum-exps, the z row means), cum
// (max(M, L) words) and the reductions (32 floats, 64 words).
__host__ __device__ constexpr size_t nl_smem_bytes(int D1, int D2, int M, int L) {
  return 4 * ((size_t)(2 * D2 + D1 + 2) * M + 2 * (size_t)L * M + (size_t)(2 * D1 + D2 + 4) * L +
              (size_t)((((M > L ? M : L) + 3) & ~3)) + 32 + 64) + 16;
}

// One call t: the inner update of step t-1 (t >= 2), then the look-ahead of step t.
template <class Mod>
__global__ void __launch_bounds__(1024) nl_step_kernel(const __grid_constant__ NLArgs a) {
  constexpr int D1 = Mod::D1, D2 = Mod::D2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int M = a.M, L = a.L, tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  const bool act = tid < M;
  const long long N = a.N, NM = N * (long long)M;
  static_assert(Mod::DY == 1, "the look-ahead's pair loop takes a scalar observation");
  float* zs = (float*)smem_raw;  // [D2][M] the ancestor's z
  float* lqs = zs + D2 * M;      // [M] the ancestor's lq, then the group's own
  float* fxk = lqs + M;          // [D1][M] f_x(x, z_k) of the look-ahead
  float* bk = fxk + D1 * M;      // [D2][M] f_z(x, z_k) + chol(S) e_k: the draw's base
  float* hzk = bk + D2 * M;      // [M] h_z of the base (models with G = 0)
  float* E1 = hzk + M;           // [L][M] alpha + ell of the pairs (log2 units)
  float* E2 = E1 + L * M;        // [L][M] alpha (log2 units)
  float* xbs = E2 + L * M;       // [L][D1] the look-ahead draws
  float* hxs = xbs + L * D1;     // [L] h_x of the draws
  float* lwhs = hxs + L;         // [L] the ancestor's per-draw weights
  float* xbbs = lwhs + L;        // [L][D1] the ancestor's draws
  float* rowm = xbbs + L * D1;   // [2L] LSE_k of alpha + ell and of alpha per draw
  float* zrow = rowm + 2 * L;    // [L][D2] sum_k softmax_k(alpha + ell) zhat per draw
  uint32_t* cum = (uint32_t*)(zrow + L * D2);  // [max(M, L)]
  float* red = (float*)(cum + (((M > L ? M : L) + 3) & ~3));
  uint32_t* redU = (uint32_t*)(red + 32);
  const float NEG = neg_inf<float>();
  const float LOG2E = (float)LOG2E_D;
  if (blockIdx.x == 0 && tid == 0) *a.Csum = 0ull;
  for (long long i = blockIdx.x; i < N; i += gridDim.x) {
    float x[D1], zk[D2];
    float lqk = NEG;
#pragma unroll
    for (int c = 0; c < D2; ++c) zk[c] = 0.f;
    if (a.first) {
#pragma unroll
      for (int c = 0; c < D1; ++c) x[c] = a.x_old[i * a.xp + c];
      if (act) {
#pragma unroll
        for (int c = 0; c < D2; ++c) zk[c] = a.z_old[c * NM + i * M + tid];
        lqk = a.lq_old[i * M + tid];
      }
    } else {
      const long long g = a.anc[i];
      if (act) {
#pragma unroll
        for (int c = 0; c < D2; ++c) zs[c * M + tid] = a.z_old[c * NM + g * M + tid];
        lqs[tid] = a.lq_old[g * M + tid];
      }
      if (tid < L) {
        lwhs[tid] = a.lwh_old[g * L + tid];
#pragma unroll
        for (int c = 0; c < D1; ++c) xbbs[tid * D1 + c] = a.xbb_old[(g * L + tid) * D1 + c];
      }
      float xa[D1];
#pragma unroll
      for (int c = 0; c < D1; ++c) xa[c] = a.x_old[g * a.xp + c];
      // ---- x_{t-1}: one of the ancestor's look-ahead draws, by its weight ----
      {
        const float l = tid < L ? lwhs[tid] : NEG;
        const float mx = bmax(l, red);
        uint32_t cw[1] = {tid < L ? (uint32_t)floor(exp2f((l - mx) * LOG2E) * a.scaleL) : 0u}, incl[1];
        bscan_planes<1>(cw, incl, redU);
        if (tid < L) cum[tid] = incl[0];
        __syncthreads();
        const uint32_t C = cum[L - 1];
        int m = sys_local_pick(cum, L, C, 1, 0, rand_word(a.key, a.t - 1, (uint32_t)i, P_SEL, 0u));
        if (C == 0 || m >= L) {
          if (tid == 0) atomicOr(a.err, ERR_NUMERIC);
          m = L - 1;
        }
        if (tid == 0) a.sel[i] = m;
#pragma unroll
        for (int c = 0; c < D1; ++c) x[c] = xbbs[m * D1 + c];
      }
      // ---- local resampling by lq + log p(x_{t-1} | x_{t-2}, z) ----
      float alpha = NEG;
      if (act) {
        float zz[D2], fxv[D1], r[D1];
#pragma unroll
        for (int c = 0; c < D2; ++c) zz[c] = zs[c * M + tid];
        Mod::fx(xa, zz, a.tt_prev, fxv);
#pragma unroll
        for (int c = 0; c < D1; ++c) r[c] = x[c] - fxv[c];
        alpha = lqs[tid] + nl_quad_x<Mod>(r);
      }
      const float amax = bmax(alpha, red);  // its barriers end the reads of cum above
      {
        uint32_t cw[1] = {act ? (uint32_t)floor(exp2f((alpha - amax) * LOG2E) * a.scaleM) : 0u}, incl[1];
        bscan_planes<1>(cw, incl, redU);
        if (act) cum[tid] = incl[0];
      }
      __syncthreads();
      const uint32_t C = cum[M - 1];
      const uint32_t uin = rand_word(a.key, a.t - 1, (uint32_t)i, P_INNER, 0u);
      // ---- propagation given x_{t-1} and the update by y_{t-1} ----
      float ell = NEG;
      if (act) {
        const int b = sys_local_pick(cum, M, C, M, tid, uin);
        if (a.dbg_b) a.dbg_b[i * M + tid] = b;
        float zb[D2], fxb[D1], fzb[D2], e[D2];
#pragma unroll
        for (int c = 0; c < D2; ++c) zb[c] = zs[c * M + b];
        Mod::fx(xa, zb, a.tt_prev, fxb);
        Mod::fz(xa, zb, a.tt_prev, fzb);
        normals<D2>(a.key, a.t - 1, (uint32_t)i, P_PROP, (uint32_t)tid, e);
        nl_zdraw<Mod>(fzb, fxb, x, e, zk);
        ell = nl_loglik<Mod>(x, zk, a.y_prev);
      }
      const float lmax = bmax(ell, red);
      const float lsum = bsum(act ? expf(ell - lmax) : 0.f, red);
      const float lse = lmax + logf(lsum);
      if (act) {
        lqk = ell - lse;
#pragma unroll
        for (int c = 0; c < D2; ++c) a.z_new[c * NM + i * M + tid] = zk[c];
        a.lq_new[i * M + tid] = lqk;
      }
      if (tid < D1) a.x_new[i * a.xp + tid] = x[tid < D1 ? tid : 0];
      __syncthreads();  // every gather from the ancestor's rows is done
    }
    // ======== look-ahead of step t from (x, z, lq) with y_t ========
    // per inner particle k: f_x, the base f_z + chol(S) e_k of its draw (the noise e_k shared
    // by the L draws) and, when the draw is free of x_t, h_z of it
    if (act) {
      float fxv[D1], fzv[D2], ek[D2], zb[D2];
      Mod::fx(x, zk, a.tt_cur, fxv);
      Mod::fz(x, zk, a.tt_cur, fzv);
      normals<D2>(a.key, a.t, (uint32_t)i, P_LA_Z, (uint32_t)tid, ek);
#pragma unroll
      for (int r = 0; r < D2; ++r) {
        float v = fzv[r];
#pragma unroll
        for (int c = 0; c < D2; ++c)
          if (c <= r) v += Mod::LS(r, c) * ek[c];
        zb[r] = v;
        bk[r * M + tid] = v;
      }
#pragma unroll
      for (int c = 0; c < D1; ++c) fxk[c * M + tid] = fxv[c];
      if (Mod::GZERO) hzk[tid] = Mod::hz(zb);
      lqs[tid] = lqk;
    }
    {
      const float mx = bmax(lqk, red);
      uint32_t cw[1] = {act ? (uint32_t)floor(exp2f((lqk - mx) * LOG2E) * a.scaleM) : 0u}, incl[1];
      bscan_planes<1>(cw, incl, redU);
      if (act) cum[tid] = incl[0];
    }
    __syncthreads();
    if (tid < L) {  // draw m from the mixture: a component by qbar, then the Gaussian
      const int m = tid;
      const int jm = sys_local_pick(cum, M, cum[M - 1], 1, 0, rand_word(a.key, a.t, (uint32_t)i, P_LA_J, (uint32_t)m));
      if (a.dbg_j) a.dbg_j[i * L + m] = jm;
      float e1[D1], xb[D1];
      normals<D1>(a.key, a.t, (uint32_t)i, P_LA_X, (uint32_t)m, e1);
#pragma unroll
      for (int r = 0; r < D1; ++r) {
        float v = fxk[r * M + jm];
#pragma unroll
        for (int c = 0; c < D1; ++c)
          if (c <= r) v += Mod::Lqx(r, c) * e1[c];
        xb[r] = v;
        xbs[m * D1 + r] = v;
        a.xbb_new[((long long)i * L + m) * D1 + r] = v;
      }
      hxs[m] = Mod::hx(xb);
    }
    __syncthreads();
    // the L x M pairs, a thread an inner particle k: alpha = lq_k + log p(xbb_m | x, z_k),
    // zhat = base_k + G (xbb_m - f_x,k), ell = log p(y_t | xbb_m, zhat)
    if (act) {
      float fxv[D1], zb[D2];
#pragma unroll
      for (int c = 0; c < D1; ++c) fxv[c] = fxk[c * M + tid];
#pragma unroll
      for (int c = 0; c < D2; ++c) zb[c] = bk[c * M + tid];
      const float hz0 = Mod::GZERO ? hzk[tid] : 0.f;
      const float y0 = a.y_cur[0];
      for (int m = 0; m < L; ++m) {
        float r[D1], zh[D2];
#pragma unroll
        for (int c = 0; c < D1; ++c) r[c] = xbs[m * D1 + c] - fxv[c];
        const float al = lqk + nl_quad_x<Mod>(r);
        float hzv = hz0;
        if (!Mod::GZERO) {
#pragma unroll
          for (int q = 0; q < D2; ++q) {
            float v = zb[q];
#pragma unroll
            for (int c = 0; c < D1; ++c) v += Mod::G(q, c) * r[c];
            zh[q] = v;
          }
          hzv = Mod::hz(zh);
        }
        const float res = (y0 - hxs[m] - hzv) * Mod::LrInv(0, 0);
        E1[m * M + tid] = (al + Mod::lognorm_y - 0.5f * res * res) * LOG2E;  // log2 units
        E2[m * M + tid] = al * LOG2E;
      }
    }
    __syncthreads();
    // a warp a draw: the log-sum-exps of both rows and the softmax-weighted zhat of row 1
    for (int m = w; m < L; m += nw) {
      float m1 = NEG, m2 = NEG;
      for (int k = lane; k < M; k += 32) {
        m1 = fmaxf(m1, E1[m * M + k]);
        m2 = fmaxf(m2, E2[m * M + k]);
      }
      m1 = warp_max(m1);
      m2 = warp_max(m2);
      float xb[D1];
#pragma unroll
      for (int c = 0; c < D1; ++c) xb[c] = xbs[m * D1 + c];
      float s1 = 0.f, s2 = 0.f, za[D2];
#pragma unroll
      for (int c = 0; c < D2; ++c) za[c] = 0.f;
      for (int k = lane; k < M; k += 32) {
        const float e = exp2_t(E1[m * M + k] - m1);
        s1 += e;
        s2 += exp2_t(E2[m * M + k] - m2);
        float r[D1];
#pragma unroll
        for (int c = 0; c < D1; ++c) r[c] = xb[c] - fxk[c * M + k];
#pragma unroll
        for (int q = 0; q < D2; ++q) {
          float v = bk[q * M + k];
#pragma unroll
          for (int c = 0; c < D1; ++c) v += Mod::G(q, c) * r[c];
          za[q] += e * v;
        }
      }
      s1 = warp_sum(s1);
      s2 = warp_sum(s2);
#pragma unroll
      for (int c = 0; c < D2; ++c) za[c] = warp_sum(za[c]);
      if (lane == 0) {  // back to natural-log units
        rowm[2 * m] = (m1 + log2f(s1)) * (float)LN2_D;
        rowm[2 * m + 1] = (m2 + log2f(s2)) * (float)LN2_D;
#pragma unroll
        for (int c = 0; c < D2; ++c) zrow[m * D2 + c] = za[c] / s1;
      }
    }
    __syncthreads();
    if (tid < 32) {  // per-draw weights, the outer weight and the filtered mean (L <= 32)
      const float lwm = tid < L ? rowm[2 * tid] - rowm[2 * tid + 1] : NEG;
      if (tid < L) a.lwh_new[i * L + tid] = lwm;
      const float mx = warp_max(lwm);
      const float p = tid < L ? expf(lwm - mx) : 0.f;
      const float ps = warp_sum(p);
#pragma unroll
      for (int c = 0; c < D1; ++c) {
        const float v = warp_sum(tid < L ? p * xbs[tid * D1 + c] : 0.f) / ps;
        if (tid == 0) a.xm[c * N + i] = v;
      }
#pragma unroll
      for (int c = 0; c < D2; ++c) {
        const float v = warp_sum(tid < L ? p * zrow[tid * D2 + c] : 0.f) / ps;
        if (tid == 0) a.zm[c * N + i] = v;
      }
      if (tid == 0) {
        const float lwi = mx + logf(ps) - a.logL;
        a.lw[i] = lwi;
        if (lwi != lwi) atomicOr(a.err, ERR_NUMERIC);
        const unsigned long long key = order_key(lwi);
        if (lwi == lwi && key > *(volatile unsigned long long*)a.lwmax_key) atomicMax(a.lwmax_key, key);
      }
    }
    __syncthreads();  // the group's arrays are free for the next group
  }
}

// The bootstrap particle filter for these models: one thread a particle.
template <class Mod>
__global__ void __launch_bounds__(256) nl_pf_kernel(const __grid_constant__ NLArgs a) {
  constexpr int D1 = Mod::D1, D2 = Mod::D2;
  const long long N = a.N;
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.Csum = 0ull;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long s = a.first ? i : (long long)a.anc[i];
    float x[D1], z[D2], fxv[D1], fzv[D2], ex[D1], ez[D2], xn[D1], zn[D2];
#pragma unroll
    for (int c = 0; c < D1; ++c) x[c] = a.x_old[s * a.xp + c];
#pragma unroll
    for (int c = 0; c < D2; ++c) z[c] = a.z_old[c * N + s];
    Mod::fx(x, z, a.tt_cur, fxv);
    Mod::fz(x, z, a.tt_cur, fzv);
    normals<D1>(a.key, a.t, (uint32_t)i, P_PF_X, 0u, ex);
    normals<D2>(a.key, a.t, (uint32_t)i, P_PF_Z, 0u, ez);
#pragma unroll
    for (int r = 0; r < D1; ++r) {
      float v = fxv[r];
#pragma unroll
      for (int c = 0; c < D1; ++c)
        if (c <= r) v += Mod::Lqx(r, c) * ex[c];
      xn[r] = v;
    }
    nl_zdraw<Mod>(fzv, fxv, xn, ez, zn);
    const float lwi = nl_loglik<Mod>(xn, zn, a.y_cur);
#pragma unroll
    for (int c = 0; c < D1; ++c) {
      a.x_new[i * a.xp + c] = xn[c];
      a.xm[c * N + i] = xn[c];
    }
#pragma unroll
    for (int c = 0; c < D2; ++c) {
      a.z_new[c * N + i] = zn[c];
      a.zm[c * N + i] = zn[c];
    }
    a.lw[i] = lwi;
    const unsigned long long key = order_key(lwi);
    if (lwi == lwi && key > *(volatile unsigned long long*)a.lwmax_key) atomicMax(a.lwmax_key, key);
  }
}

// Bytes of shared memory of nl_std_kernel: the ancestor's z, f_x and f_z per inner
// particle, cum (M words) and the reductions (32 floats, 64 words).
__host__ __device__ constexpr size_t nl_std_smem_bytes(int D1, int D2, int M) {
  return 4 * ((size_t)(2 * D2 + D1) * M + (size_t)((M + 3) & ~3) + 32 + 64) + 16;
}

// The DPF without look-ahead for these models (the paper's Fig. dpf with the prior as both
// proposals), call t for each outer particle i with ancestor a (i itself at t = 1):
//   x_t ~ sum_j qbar_j N(f_x(x_a, z_aj), Q_xx): the component by the one-draw local rule
//         (word (t, i, LA_J, 0)), then the Gaussian draw (normals (t, i, LA_X, 0)); with the
//         Gaussian approximation (Section 4.2) the mixture's moment-matched Gaussian instead,
//         mean sum_j qbar_j f_x,j and covariance Q_xx + sum_j qbar_j (f_x,j - mu)(f_x,j - mu)^T;
//   b = local resampling by lq_aj + log N(x_t; f_x,j, Q_xx) (word (t, i, INNER, 0));
//   z_t^j = f_z,b + G (x_t - f_x,b) + chol(S) e_j (normals (t, i, PROP, j));
//   lq = ell - LSE ell, ell = log p(y_t | x_t, z_t^j); log w = LSE ell - log M.
template <class Mod>
__global__ void __launch_bounds__(1024) nl_std_kernel(const __grid_constant__ NLArgs a, int gauss) {
  constexpr int D1 = Mod::D1, D2 = Mod::D2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int M = a.M, tid = threadIdx.x;
  const bool act = tid < M;
  const long long N = a.N, NM = N * (long long)M;
  float* zs = (float*)smem_raw;  // [D2][M] the ancestor's z
  float* fxs = zs + D2 * M;      // [D1][M]
  float* fzs = fxs + D1 * M;     // [D2][M]
  uint32_t* cum = (uint32_t*)(fzs + D2 * M);  // [M]
  float* red = (float*)(cum + ((M + 3) & ~3));
  uint32_t* redU = (uint32_t*)(red + 32);
  const float NEG = neg_inf<float>();
  const float LOG2E = (float)LOG2E_D;
  if (blockIdx.x == 0 && tid == 0) *a.Csum = 0ull;
  for (long long i = blockIdx.x; i < N; i += gridDim.x) {
    const long long g = a.first ? i : (long long)a.anc[i];
    float xa[D1], fxj[D1], fzj[D2];
#pragma unroll
    for (int c = 0; c < D1; ++c) xa[c] = a.x_old[g * a.xp + c];
    float lqj = NEG;
#pragma unroll
    for (int c = 0; c < D1; ++c) fxj[c] = 0.f;
    if (act) {
      float zj[D2];
#pragma unroll
      for (int c = 0; c < D2; ++c) {
        zj[c] = a.z_old[c * NM + g * M + tid];
        zs[c * M + tid] = zj[c];
      }
      lqj = a.lq_old[g * M + tid];
      Mod::fx(xa, zj, a.tt_cur, fxj);
      Mod::fz(xa, zj, a.tt_cur, fzj);
#pragma unroll
      for (int c = 0; c < D1; ++c) fxs[c * M + tid] = fxj[c];
#pragma unroll
      for (int c = 0; c < D2; ++c) fzs[c * M + tid] = fzj[c];
    }
    // ---- x_t from the mixture prior ----
    const float mx = bmax(lqj, red);
    {
      uint32_t cw[1] = {act ? (uint32_t)floor(exp2f((lqj - mx) * LOG2E) * a.scaleM) : 0u}, incl[1];
      bscan_planes<1>(cw, incl, redU);
      if (act) cum[tid] = incl[0];
    }
    __syncthreads();
    float e1[D1], xt[D1];
    normals<D1>(a.key, a.t, (uint32_t)i, P_LA_X, 0u, e1);
    if (gauss) {
      if (a.dbg_j && tid == 0) a.dbg_j[i] = -1;
      const float qj = act ? expf(lqj - mx) : 0.f;
      const float qs = bsum(qj, red);
      float mu[D1];
#pragma unroll
      for (int r = 0; r < D1; ++r) mu[r] = bsum(qj * fxj[r], red) / qs;
      float C[D1][D1];
#pragma unroll
      for (int r = 0; r < D1; ++r)
#pragma unroll
        for (int c = 0; c < D1; ++c)
          if (c <= r) {
            float q = 0.f;  // Q_xx = L_qx L_qx^T
#pragma unroll
            for (int k = 0; k < D1; ++k) q += Mod::Lqx(r, k) * Mod::Lqx(c, k);
            C[r][c] = bsum(qj * (fxj[r] - mu[r]) * (fxj[c] - mu[c]), red) / qs + q;
          }
      // Cholesky of the covariance in place (lower triangle), the same in every thread
#pragma unroll
      for (int c = 0; c < D1; ++c) {
        float d = C[c][c];
#pragma unroll
        for (int k = 0; k < D1; ++k)
          if (k < c) d -= C[c][k] * C[c][k];
        d = sqrtf(d);
        C[c][c] = d;
#pragma unroll
        for (int r = 0; r < D1; ++r) {
          if (r > c) {
            float v = C[r][c];
#pragma unroll
            for (int k = 0; k < D1; ++k)
              if (k < c) v -= C[r][k] * C[c][k];
            C[r][c] = v / d;
          }
        }
      }
#pragma unroll
      for (int r = 0; r < D1; ++r) {
        float v = mu[r];
#pragma unroll
        for (int c = 0; c < D1; ++c)
          if (c <= r) v += C[r][c] * e1[c];
        xt[r] = v;
      }
    } else {
      const int jm = sys_local_pick(cum, M, cum[M - 1], 1, 0, rand_word(a.key, a.t, (uint32_t)i, P_LA_J, 0u));
      if (a.dbg_j && tid == 0) a.dbg_j[i] = jm;
#pragma unroll
      for (int r = 0; r < D1; ++r) {
        float v = fxs[r * M + jm];
#pragma unroll
        for (int c = 0; c < D1; ++c)
          if (c <= r) v += Mod::Lqx(r, c) * e1[c];
        xt[r] = v;
      }
    }
    // ---- local resampling by q = qbar p(x_t | x_{t-1}, z) ----
    float alpha = NEG;
    if (act) {
      float r[D1];
#pragma unroll
      for (int c = 0; c < D1; ++c) r[c] = xt[c] - fxj[c];
      alpha = lqj + nl_quad_x<Mod>(r);
    }
    const float amax = bmax(alpha, red);  // its barriers also end every read of cum above
    {
      uint32_t cw[1] = {act ? (uint32_t)floor(exp2f((alpha - amax) * LOG2E) * a.scaleM) : 0u}, incl[1];
      bscan_planes<1>(cw, incl, redU);
      if (act) cum[tid] = incl[0];
    }
    __syncthreads();
    const uint32_t C = cum[M - 1];
    const uint32_t uin = rand_word(a.key, a.t, (uint32_t)i, P_INNER, 0u);
    // ---- propagation given x_t and the weights of y_t ----
    float zn[D2];
    float ell = NEG;
#pragma unroll
    for (int c = 0; c < D2; ++c) zn[c] = 0.f;
    if (act) {
      const int b = sys_local_pick(cum, M, C, M, tid, uin);
      if (a.dbg_b) a.dbg_b[i * M + tid] = b;
      float fxb[D1], fzb[D2], e[D2];
#pragma unroll
      for (int c = 0; c < D1; ++c) fxb[c] = fxs[c * M + b];
#pragma unroll
      for (int c = 0; c < D2; ++c) fzb[c] = fzs[c * M + b];
      normals<D2>(a.key, a.t, (uint32_t)i, P_PROP, (uint32_t)tid, e);
      nl_zdraw<Mod>(fzb, fxb, xt, e, zn);
      ell = nl_loglik<Mod>(xt, zn, a.y_cur);
    }
    const float lmax = bmax(ell, red);
    const float lsum = bsum(act ? expf(ell - lmax) : 0.f, red);
    const float lse = lmax + logf(lsum);
    const float W = act ? expf(ell - lse) : 0.f;
    if (act) {
#pragma unroll
      for (int c = 0; c < D2; ++c) a.z_new[c * NM + i * M + tid] = zn[c];
      a.lq_new[i * M + tid] = ell - lse;
    }
#pragma unroll
    for (int c = 0; c < D2; ++c) {
      const float v = bsum(W * zn[c], red);
      if (tid == 0) a.zm[c * N + i] = v;
    }
    if (tid == 0) {
      const float lwi = lse - a.logL;  // logL carries log M here
#pragma unroll
      for (int c = 0; c < D1; ++c) {
        a.x_new[i * a.xp + c] = xt[c];
        a.xm[c * N + i] = xt[c];
      }
      a.lw[i] = lwi;
      if (lwi != lwi) atomicOr(a.err, ERR_NUMERIC);
      const unsigned long long key = order_key(lwi);
      if (lwi == lwi && key > *(volatile unsigned long long*)a.lwmax_key) atomicMax(a.lwmax_key, key);
    }
    __syncthreads();  // the staged rows are free for the next group
  }
}

}  // namespace dpf

#include "dpf_variant.cuh"

namespace dpf {

// A paper model as a filter variant (FP32): the LA-DPF step, the bootstrap particle filter's
// step and the shared outer stage.
template <class Mod>
struct PaperVariant {
  static constexpr int D1 = Mod::D1, D2 = Mod::D2, DY = Mod::DY;
  static int xpad() { return (D1 * 4 + 15) / 16 * 16 / 4; }
  static dpf_status make_const(const HostModel&, std::vector<unsigned char>& out) {
    out.clear();
    return DPF_OK;
  }
  static size_t smem(int M, int L, bool, int) {
    return L > 32 ? (size_t)1 << 40 : nl_smem_bytes(D1, D2, M, L);  // L <= 32: one warp's draws
  }
  static dpf_status init(Ctx& x) {
    const Key key{(uint32_t)x.seed, (uint32_t)(x.seed >> 32)};
    nl_init_kernel<Mod><<<(unsigned)x.N, threads_for(x.M), 0, x.stream>>>(
        (float*)x.z[0], (float*)x.lq[0], (float*)x.x[0], x.N, x.M, x.xp, key);
    return cuda_error(cudaGetLastError(), "init kernel launch");
  }
  static void terms(long long s, float (&tt)[2]) {
    float v[Mod::NT];
    Mod::terms((double)s, v);
    tt[0] = v[0];
    tt[1] = Mod::NT > 1 ? v[Mod::NT > 1 ? 1 : 0] : 0.f;
  }
  static dpf_status step(Ctx& x, int) {
    const long long t = x.t + 1;
    const int so = (int)((t + 2) % 2), sn = (int)((t + 1) % 2);
    const bool first = t == 1;
    NLArgs a{};
    a.z_old = (const float*)x.z[first ? sn : so];
    a.lq_old = (const float*)x.lq[first ? sn : so];
    a.x_old = (const float*)x.x[first ? sn : so];
    a.z_new = (float*)x.z[sn];
    a.lq_new = (float*)x.lq[sn];
    a.x_new = (float*)x.x[sn];
    a.lwh_old = (const float*)x.lwh[(t + 1) % 2];
    a.xbb_old = (const float*)x.xbb[(t + 1) % 2];
    a.lwh_new = (float*)x.lwh[t % 2];
    a.xbb_new = (float*)x.xbb[t % 2];
    a.anc = x.anc;
    a.sel = x.sel;
    a.lw = (float*)x.lw;
    a.xm = (float*)x.xm;
    a.zm = (float*)x.zm;
    a.y_prev = (const float*)x.yb + ((t + 1) % 2) * x.dy;
    a.y_cur = (const float*)x.yb + (t % 2) * x.dy;
    a.lwmax_key = x.lwmax_key;
    a.Csum = x.Csum;
    a.err = x.err;
    a.N = x.N;
    a.M = x.M;
    a.L = x.L;
    a.xp = x.xp;
    a.t = (uint32_t)t;
    a.key = Key{(uint32_t)x.seed, (uint32_t)(x.seed >> 32)};
    terms(t - 2, a.tt_prev);
    terms(t - 1, a.tt_cur);
    a.scaleM = (float)std::ldexp(1.0, 31 - ceil_log2_i(x.M));
    a.scaleL = (float)std::ldexp(1.0, 31 - ceil_log2_i(x.L));
    a.logL = (float)std::log((double)x.L);
    a.first = first ? 1 : 0;
    a.dbg_b = x.debug ? x.dbg_b : nullptr;
    a.dbg_j = x.debug ? x.dbg_j : nullptr;
    const int big = x.M > x.L ? x.M : x.L;
    const int nt = (big < 32 ? 32 : (big + 31) / 32 * 32);
    const size_t sm = nl_smem_bytes(D1, D2, x.M, x.L);
    auto k = nl_step_kernel<Mod>;
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
    }
    // a persistent grid: every SM filled with as many CTAs as fit at once
    int occ = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, nt, sm);
    const long long fill = (long long)std::max(occ, 1) * std::max(sms, 1);
    const unsigned blocks = (unsigned)std::min<long long>(x.N, fill);
    k<<<blocks, nt, sm, x.stream>>>(a);
    return cuda_error(cudaGetLastError(), "paper-model step launch");
  }
  static dpf_status pf_step(Ctx& x) {
    const long long t = x.t + 1;
    const int so = (int)((t + 1) % 2), sn = (int)(t % 2);
    NLArgs a{};
    a.x_old = (const float*)x.x[so];
    a.z_old = (const float*)x.z[so];
    a.x_new = (float*)x.x[sn];
    a.z_new = (float*)x.z[sn];
    a.lw = (float*)x.lw;
    a.xm = (float*)x.xm;
    a.zm = (float*)x.zm;
    a.anc = x.anc;
    a.y_cur = (const float*)x.yb + (t % 2) * x.dy;
    a.lwmax_key = x.lwmax_key;
    a.Csum = x.Csum;
    a.err = x.err;
    a.N = x.N;
    a.M = 1;
    a.xp = x.xp;
    a.t = (uint32_t)t;
    a.key = Key{(uint32_t)x.seed, (uint32_t)(x.seed >> 32)};
    terms(t - 1, a.tt_cur);
    a.first = t == 1 ? 1 : 0;
    const unsigned blocks = (unsigned)std::min<long long>((x.N + 255) / 256, 152 * 8);
    nl_pf_kernel<Mod><<<blocks, 256, 0, x.stream>>>(a);
    return cuda_error(cudaGetLastError(), "paper-model particle filter launch");
  }
  static dpf_status std_step(Ctx& x) {
    const long long t = x.t + 1;
    const int so = (int)((t + 1) % 2), sn = (int)(t % 2);
    NLArgs a{};
    a.x_old = (const float*)x.x[so];
    a.z_old = (const float*)x.z[so];
    a.lq_old = (const float*)x.lq[so];
    a.x_new = (float*)x.x[sn];
    a.z_new = (float*)x.z[sn];
    a.lq_new = (float*)x.lq[sn];
    a.lw = (float*)x.lw;
    a.xm = (float*)x.xm;
    a.zm = (float*)x.zm;
    a.anc = x.anc;
    a.y_cur = (const float*)x.yb + (t % 2) * x.dy;
    a.lwmax_key = x.lwmax_key;
    a.Csum = x.Csum;
    a.err = x.err;
    a.N = x.N;
    a.M = x.M;
    a.xp = x.xp;
    a.t = (uint32_t)t;
    a.key = Key{(uint32_t)x.seed, (uint32_t)(x.seed >> 32)};
    terms(t - 1, a.tt_cur);
    a.scaleM = (float)std::ldexp(1.0, 31 - ceil_log2_i(x.M));
    a.logL = (float)std::log((double)x.M);
    a.first = t == 1 ? 1 : 0;
    a.dbg_b = x.debug ? x.dbg_b : nullptr;
    a.dbg_j = x.debug ? x.dbg_j : nullptr;
    const int nt = (x.M + 31) / 32 * 32;
    const size_t sm = nl_std_smem_bytes(D1, D2, x.M);
    auto k = nl_std_kernel<Mod>;
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
    }
    const unsigned blocks = (unsigned)std::min<long long>(x.N, 152 * 8);
    k<<<blocks, nt, sm, x.stream>>>(a, x.std_gauss ? 1 : 0);
    return cuda_error(cudaGetLastError(), "paper-model DPF step launch");
  }
  static dpf_status outer(Ctx& x, double* mean_out, double* logz_out, cudaStream_t st) {
    return outer_stage<float, D1, D2>(x, mean_out, logz_out, st);
  }
  static Variant make() {
    Variant v;
    v.prec = DPF_F32;
    v.d1 = D1;
    v.d2 = D2;
    v.dy = DY;
    v.make_const = &make_const;
    v.init = &init;
    v.step = &step;
    v.outer = &outer;
    v.pf_step = &pf_step;
    v.std_step = &std_step;
    v.outer_args = nullptr;
    v.outer_batch = nullptr;
    v.scan_batch = nullptr;
    v.step_smem = &smem;
    v.xpad = &xpad;
    v.batch_args = nullptr;
    v.region_bytes = nullptr;
    v.batch_launch = nullptr;
    v.use_xz = nullptr;
    v.ppl_for = nullptr;
    v.args_size = sizeof(NLArgs);
    v.const_size = 0;
    v.oargs_size = sizeof(FusedOuterArgs<float>);
    v.max_m = 1024;
    v.xz_supported = true;
    return v;
  }
};

}  // namespace dpf
