// The bootstrap particle filter over the full state s = (x, z), the baseline the
// paper compares the decentralized filters with (Section 4.1, "PF"): every particle
// is propagated from its resampled ancestor by the model's transition and weighted
// by the likelihood of y_t. One thread a particle. The outer stages of the filter
// (the evidence, the weighted mean and the global systematic resampling) serve it
// unchanged, with one "group" a particle: lw is the particle's log-weight and
// (xm, zm) its state.
//
// Transition (no x/z cross-covariance in Q, as for the filter):
//   x_t = mu_x(x_{t-1}) + A_xz z_{t-1} + L_qx e_x,   z_t = A_zx x_{t-1} + A_zz z_{t-1} + L_qz e_z,
// with e_x the Philox normals of purpose PF_X and e_z those of PF_Z at counter
// (t, i, purpose, 0). Weight: log w_i = log N(y_t; h_x(x_t) + H_z z_t, R).
#pragma once

#include "dpf_step.cuh"

namespace dpf {

template <typename T>
struct PFArgs {
  const T* x_old;  // [N][xp]: the particles of step t-1 (t = 1: the initial draw)
  const T* z_old;  // [D2][N]
  T* x_new;
  T* z_new;
  T* lw;           // [N] log-weights of step t
  T* xm;           // [D1][N] the particles' x, for the weighted mean
  T* zm;           // [D2][N]
  const int32_t* anc;  // [N] ancestors from the last resampling (t >= 2)
  const T* y;          // [DY] y_t
  unsigned long long* lwmax_key;
  unsigned long long* Csum;  // reset here for this step's outer reduction
  long long N;
  int xp;
  uint32_t t;
  Key key;
  T gcos;     // growth cosine term of the transition into step t
  int first;  // t == 1: the particles are the initial draw, no ancestors yet
};

template <typename T, int D1, int D2, int DY, bool XZ>
__global__ void __launch_bounds__(256)
    pf_kernel(const __grid_constant__ MC<T, D1, D2, DY> mc, const __grid_constant__ PFArgs<T> a) {
  const RoundKeys rk = round_keys(a.key);
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.Csum = 0ull;
  const long long N = a.N;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long s = a.first ? i : (long long)a.anc[i];
    T x[D1], z[D2];
#pragma unroll
    for (int c = 0; c < D1; ++c) x[c] = a.x_old[s * a.xp + c];
#pragma unroll
    for (int c = 0; c < D2; ++c) z[c] = a.z_old[c * N + s];
    T ex[D1], ez[D2];
    normals_rk<D1>(rk, a.t, (uint32_t)i, P_PF_X, 0u, ex);
    normals_rk<D2>(rk, a.t, (uint32_t)i, P_PF_Z, 0u, ez);
    // x_t = mu_x + L_qx (L_qx^-1 A_xz z + e_x)
    T mux[D1];
    mu_x(mc, x, a.gcos, mux);
    T wx[D1];
#pragma unroll
    for (int r = 0; r < D1; ++r) {
      T v = ex[r];
      if (XZ) {
#pragma unroll
        for (int c = 0; c < D2; ++c) v += mc.WAxz[r][c] * z[c];
      }
      wx[r] = v;
    }
    T xn[D1];
#pragma unroll
    for (int r = 0; r < D1; ++r) {
      T v = mux[r];
#pragma unroll
      for (int c = 0; c < D1; ++c)
        if (c <= r) v += mc.Lqx[r][c] * wx[c];
      xn[r] = v;
    }
    // z_t = A_zx x + A_zz z + L_qz e_z
    T zn[D2];
#pragma unroll
    for (int r = 0; r < D2; ++r) {
      T v = T(0);
#pragma unroll
      for (int c = 0; c < D1; ++c) v += mc.Azx[r][c] * x[c];
#pragma unroll
      for (int c = 0; c < D2; ++c) v += mc.Azz[r][c] * z[c];
      if (mc.diag_qz) {
        v += mc.Lqz[r][r] * ez[r];
      } else {
#pragma unroll
        for (int c = 0; c < D2; ++c)
          if (c <= r) v += mc.Lqz[r][c] * ez[c];
      }
      zn[r] = v;
    }
    // log N(y_t; h_x(x_t) + H_z z_t, R): whitened residual L_r^-1 (y - h_x) - L_r^-1 H_z z
    T hx[DY], res[DY];
    h_x(mc, xn, hx);
#pragma unroll
    for (int q = 0; q < DY; ++q) res[q] = a.y[q] - hx[q];
    T qf = T(0);
#pragma unroll
    for (int q = 0; q < DY; ++q) {
      T v = T(0);
#pragma unroll
      for (int c = 0; c < DY; ++c)
        if (c <= q) v += mc.LrInv[q][c] * res[c];
#pragma unroll
      for (int c = 0; c < D2; ++c) v -= mc.LrHz[q][c] * zn[c];
      qf += v * v;
    }
    const T lwi = mc.lognorm_y - T(0.5) * qf;
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

}  // namespace dpf
