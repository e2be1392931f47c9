// The decentralized particle filter without look-ahead (the paper's Fig. dpf, after
// Chen et al. 2011), with the prior as both proposals, the filter the LA-DPF extends.
// Call t, for each outer particle i (one CTA a group, one thread an inner particle):
//   a = the ancestor the outer resampling of call t-1 gave i (i itself at t = 1);
//   x_t^i ~ sum_j qbar^(a,j) p(x_t | x_{t-1}^a, z_{t-1}^(a,j))      (step 4: the mixture prior;
//          the component by the one-draw local systematic rule, the Gaussian draw after it);
//   q^(j) proportional to qbar^(a,j) p(x_t^i | x_{t-1}^a, z_{t-1}^(a,j))   (step 5);
//   b = local systematic resampling of j by q                          (step 6);
//   z_t^(i,j) = A_zx x_{t-1}^a + A_zz z_{t-1}^(a,b_j) + chol(Q_z) e     (step 7, r = 1);
//   ell^(i,j) = log p(y_t | x_t^i, z_t^(i,j)); log w^i = LSE_j ell - log M   (step 1);
//   qbar^(i,j) = exp(ell - LSE_j ell)                                  (step 3).
// The outer resampling of step 2 is the filter's global scan after the kernel, which
// also gives the evidence and the weighted mean. Random words: the component (t, i,
// LA_J, 0), the x noise (t, i, LA_X, 0), the local resampling (t, i, INNER, 0), the z
// noise (t, i, PROP, j). With the Gaussian approximation of the mixture (Section 4.2),
// step 4 draws x_t from the Gaussian with the mixture's mean and covariance instead, with
// the same normals.
#pragma once

#include "dpf_step.cuh"

namespace dpf {

template <typename T>
struct StdArgs {
  const T* x_old;  // [N][xp]
  const T* z_old;  // [D2][N M]
  const T* lq_old;  // [N][M] normalised inner log-weights (log qbar)
  T* x_new;
  T* z_new;
  T* lq_new;
  T* lw;  // [N]
  T* xm;  // [D1][N]
  T* zm;  // [D2][N]: sum_j qbar z
  const int32_t* anc;
  const T* y;  // [DY] y_t
  unsigned long long* lwmax_key;
  unsigned long long* Csum;
  int* err;
  long long N;
  int M, xp;
  uint32_t t;
  Key key;
  T gcos;     // growth cosine term of the transition into step t
  T scaleM;   // 2^(31 - ceil(log2 M)): the local rule's quantisation
  T logM;
  int first;  // t == 1: no ancestors yet
  int gauss;  // draw x_t from the moment-matched Gaussian of the mixture (Section 4.2)
  int32_t* dbg_b;  // debug (or null): the local resampling indices, N x M
  int32_t* dbg_j;  // debug (or null): the mixture component of x_t (-1 for the Gaussian form), N
};

template <typename T, int D1, int D2, int DY, bool XZ>
__global__ void __launch_bounds__(1024)
    std_dpf_kernel(const __grid_constant__ MC<T, D1, D2, DY> mc, const __grid_constant__ StdArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int M = a.M, tid = threadIdx.x, j = tid;
  const bool act = j < M;
  const long long N = a.N, NM = N * (long long)M;
  T* zs = (T*)smem_raw;                         // [D2][M] the ancestor group's z
  uint32_t* cum = (uint32_t*)(zs + D2 * M);     // [M]
  T* red = (T*)(cum + M + (M & 1));             // [32] block reductions
  uint32_t* redU = (uint32_t*)(red + 32);       // [64]
  const T NEG = neg_inf<T>();
  const T LOG2E = (T)LOG2E_D;
  if (blockIdx.x == 0 && tid == 0) *a.Csum = 0ull;
  for (long long i = blockIdx.x; i < N; i += gridDim.x) {
    const long long g = a.first ? i : (long long)a.anc[i];
    T xp_[D1];
#pragma unroll
    for (int c = 0; c < D1; ++c) xp_[c] = a.x_old[g * a.xp + c];
    T lqj = NEG;
    if (act) {
#pragma unroll
      for (int c = 0; c < D2; ++c) zs[c * M + j] = a.z_old[c * NM + g * M + j];
      lqj = a.lq_old[g * M + j];
    }
    // ---- x_t from the mixture: the component, then the Gaussian draw ----
    const T mx = bmax(lqj, red);
    {
      uint32_t cw[1] = {act ? (uint32_t)floor(exp2_t((lqj - mx) * LOG2E) * a.scaleM) : 0u}, incl[1];
      bscan_planes<1>(cw, incl, redU);
      if (act) cum[j] = incl[0];
    }
    __syncthreads();  // the staged rows and the component weights are complete
    const int jm = sys_local_pick(cum, M, cum[M - 1], 1, 0, rand_word(a.key, a.t, (uint32_t)i, P_LA_J, 0u));
    if (a.dbg_j && j == 0) a.dbg_j[i] = (XZ && a.gauss) ? -1 : jm;
    T e1[D1];
    normals<D1>(a.key, a.t, (uint32_t)i, P_LA_X, 0u, e1);
    T mux[D1];
    mu_x(mc, xp_, a.gcos, mux);
    T xt[D1];
    {
      T w[D1];
      if (XZ && a.gauss) {
        // the mixture's moment-matched Gaussian, in the coordinates whitened by L_qx: with
        // u_j = L_qx^-1 A_xz z_j, mean ubar = sum_j qbar_j u_j and covariance I + C,
        // C = sum_j qbar_j (u_j - ubar)(u_j - ubar)^T; w = ubar + chol(I + C) e
        T uj[D1];
#pragma unroll
        for (int r = 0; r < D1; ++r) {
          T v = T(0);
          if (act) {
#pragma unroll
            for (int c = 0; c < D2; ++c) v += mc.WAxz[r][c] * zs[c * M + j];
          }
          uj[r] = v;
        }
        const T qj = act ? exp_t<T>(lqj - mx) : T(0);
        const T qs = bsum(qj, red);
        T ub[D1];
#pragma unroll
        for (int r = 0; r < D1; ++r) ub[r] = bsum(qj * uj[r], red) / qs;
        T G[D1][D1];
#pragma unroll
        for (int r = 0; r < D1; ++r)
#pragma unroll
          for (int c = 0; c < D1; ++c)
            if (c <= r) G[r][c] = bsum(qj * (uj[r] - ub[r]) * (uj[c] - ub[c]), red) / qs + (r == c ? T(1) : T(0));
        // Cholesky of I + C in place (lower triangle), the same in every thread
#pragma unroll
        for (int c = 0; c < D1; ++c) {
          T d = G[c][c];
#pragma unroll
          for (int k = 0; k < D1; ++k)
            if (k < c) d -= G[c][k] * G[c][k];
          d = sqrt(d);
          G[c][c] = d;
#pragma unroll
          for (int r = 0; r < D1; ++r) {
            if (r > c) {
              T v = G[r][c];
#pragma unroll
              for (int k = 0; k < D1; ++k)
                if (k < c) v -= G[r][k] * G[c][k];
              G[r][c] = v / d;
            }
          }
        }
#pragma unroll
        for (int r = 0; r < D1; ++r) {
          T v = ub[r];
#pragma unroll
          for (int c = 0; c < D1; ++c)
            if (c <= r) v += G[r][c] * e1[c];
          w[r] = v;
        }
      } else {
#pragma unroll
        for (int r = 0; r < D1; ++r) {
          T v = e1[r];
          if (XZ) {
#pragma unroll
            for (int c = 0; c < D2; ++c) v += mc.WAxz[r][c] * zs[c * M + jm];
          }
          w[r] = v;
        }
      }
#pragma unroll
      for (int r = 0; r < D1; ++r) {
        T v = mux[r];
#pragma unroll
        for (int c = 0; c < D1; ++c)
          if (c <= r) v += mc.Lqx[r][c] * w[c];
        xt[r] = v;
      }
    }
    // ---- local resampling by q = qbar p(x_t | x_{t-1}, z) ----
    T alpha = lqj;
    if (XZ && act) {
      T wres[D1];  // L_qx^-1 (x_t - mu_x): the z-free part of the whitened residual
#pragma unroll
      for (int r = 0; r < D1; ++r) {
        T v = T(0);
#pragma unroll
        for (int c = 0; c < D1; ++c)
          if (c <= r) v += mc.LqxInv[r][c] * (xt[c] - mux[c]);
        wres[r] = v;
      }
      T q = T(0);
#pragma unroll
      for (int r = 0; r < D1; ++r) {
        T v = wres[r];
#pragma unroll
        for (int c = 0; c < D2; ++c) v -= mc.WAxz[r][c] * zs[c * M + j];
        q += v * v;
      }
      alpha -= T(0.5) * q;
    }
    const T amax = bmax(act ? alpha : NEG, red);  // its barriers also end every read of cum above
    {
      uint32_t cw[1] = {act ? (uint32_t)floor(exp2_t((alpha - amax) * LOG2E) * a.scaleM) : 0u}, incl[1];
      bscan_planes<1>(cw, incl, redU);
      if (act) cum[j] = incl[0];
    }
    __syncthreads();
    const uint32_t C = cum[M - 1];
    const uint32_t uin = rand_word(a.key, a.t, (uint32_t)i, P_INNER, 0u);
    // ---- propagation from the prior and the weights of y_t ----
    T yh[DY];
    {
      T hx[DY], res[DY];
      h_x(mc, xt, hx);
#pragma unroll
      for (int q = 0; q < DY; ++q) res[q] = a.y[q] - hx[q];
#pragma unroll
      for (int q = 0; q < DY; ++q) {
        T v = T(0);
#pragma unroll
        for (int c = 0; c < DY; ++c)
          if (c <= q) v += mc.LrInv[q][c] * res[c];
        yh[q] = v;
      }
    }
    T zn[D2];
    T ell = NEG;
    if (act) {
      const int b = sys_local_pick(cum, M, C, M, j, uin);
      if (a.dbg_b) a.dbg_b[i * M + j] = b;
      T eps[D2];
      normals<D2>(a.key, a.t, (uint32_t)i, P_PROP, (uint32_t)j, eps);
#pragma unroll
      for (int r = 0; r < D2; ++r) {
        T v = T(0);
#pragma unroll
        for (int c = 0; c < D1; ++c) v += mc.Azx[r][c] * xp_[c];
#pragma unroll
        for (int c = 0; c < D2; ++c) v += mc.Azz[r][c] * zs[c * M + b];
#pragma unroll
        for (int c = 0; c < D2; ++c)
          if (c <= r) v += mc.Lqz[r][c] * eps[c];
        zn[r] = v;
      }
      T qf = T(0);
#pragma unroll
      for (int q = 0; q < DY; ++q) {
        T v = yh[q];
#pragma unroll
        for (int c = 0; c < D2; ++c) v -= mc.LrHz[q][c] * zn[c];
        qf += v * v;
      }
      ell = mc.lognorm_y - T(0.5) * qf;
    }
    const T lmax = bmax(ell, red);
    const T lsum = bsum(act ? exp_t<T>(ell - lmax) : T(0), red);
    const T lse = lmax + log_t(lsum);
    const T lqn = ell - lse;
    T W = act ? exp_t<T>(lqn) : T(0);
    if (act) {
#pragma unroll
      for (int c = 0; c < D2; ++c) a.z_new[c * NM + i * M + j] = zn[c];
      a.lq_new[i * M + j] = lqn;
    }
    // the group's z-mean sum_j qbar z_t, one coordinate at a time
#pragma unroll
    for (int c = 0; c < D2; ++c) {
      const T s = bsum(act ? W * zn[c] : T(0), red);
      if (tid == 0) a.zm[c * N + i] = s;
    }
    if (tid == 0) {
      const T lwi = lse - a.logM;
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
