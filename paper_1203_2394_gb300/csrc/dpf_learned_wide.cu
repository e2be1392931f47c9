// The outer-amortised learned proposal at the wide size (d1 = 8, d2 = 56, dy = 8):
// the inner update of a step (Fig. 4, step 4) with the network's per-group affine map
// of the prior draws in place of the plain prior proposal.
//
// Three stages per step, all on the filter's stream:
//   1. oaw_prepare_kernel, one CTA per outer particle, one inner particle a thread:
//      the SIR selection among the ancestor's look-ahead draws and the local
//      systematic resampling of its inner set (the plain rule, bit for bit), then the
//      prior means mu_j = A_zx x_{t-1} + A_zz z_{t-1}^(b_j) (kept in device memory,
//      d2 planes of N M floats, for stage 3) and the group features (x_{t-1}, x_t,
//      y_t, mean and variance of mu over j);
//   2. the network over the N feature rows (proposal_forward_rows: four products on
//      the tensor cores, BF16 operands and FP32 accumulation);
//   3. oaw_update_kernel, one CTA per outer particle: the prior draw
//      zhat = mu + L_qz eps, the map z = k + c + s (zhat - k) about the centre k (the
//      group's mean prior mean m, or the particle's own mu), and the importance
//      weight log N(z; mu, Q_z) - log N(zhat; mu, Q_z) + sum log s + log p(y_t | x_t, z)
//      normalised over the group.
// Stage 1 forms A_zz z_b either on the CUDA cores, from the ancestor's inner set (56 rows
// of M values) and A_zz^T staged in shared memory, or at M = 256 on the tensor cores
// (oaw_prepare_tc_kernel). The other model constants (A_zx, L_qz, H_z, L_R^-1) sit in
// this translation unit's constant bank and are read as uniform constant-bank operands.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <utility>
#include <vector>

#include "dpf_learned.h"
#include "dpf_tc.cuh"
#include "dpf_variant.cuh"

namespace dpf {

namespace {

constexpr int OW_D1 = 8, OW_D2 = 56, OW_DY = 8;
constexpr int OW_DIN = 2 * OW_D1 + OW_DY + 2 * OW_D2;  // group features
constexpr int OW_DOUT = 2 * OW_D2;                      // raw log s, c
typedef MC<float, OW_D1, OW_D2, OW_DY> OwConst;

// 52 KB of this module's 64 KB constant bank; copied from the context's device copy
// before the stages of every step, in stream order.
__constant__ OwConst c_ow;

// The ancestor's inner set z_{t-1}^(src, .) into sz[c * M + j] (M threads).
__device__ __forceinline__ void ow_stage(const float* __restrict__ z_old, long long NM, long long src, int M,
                                         float* sz) {
  const int j = threadIdx.x;
#pragma unroll 8
  for (int c = 0; c < OW_D2; ++c) sz[c * M + j] = z_old[c * NM + src * M + j];
}

// A_zz^T in shared memory (sAt[c * 56 + r]), copied once per CTA: the 12.5 KB matrix is
// read as warp-uniform 16-byte loads (a broadcast), where constant-bank operands of
// that size would miss the constant cache.
constexpr int OW_AT_FLOATS = OW_D2 * OW_D2;
__device__ __forceinline__ void ow_load_at(float* sAt) {
  for (int e = threadIdx.x; e < OW_AT_FLOATS; e += blockDim.x) {
    const int c = e / OW_D2, r = e % OW_D2;
    sAt[e] = c_ow.Azz[r][c];
  }
}

// mu = A_zx xa + A_zz z_b, z_b the staged column b (column by column: one load of
// z_b[c] and fourteen 16-byte loads of A_zz's column c, then 56 FMAs).
__device__ __forceinline__ void ow_prior_mean(const float (&xa)[OW_D1], const float* sz, const float* sAt, int M,
                                              int b, float (&mu)[OW_D2]) {
#pragma unroll
  for (int r = 0; r < OW_D2; ++r) {
    float v = 0.f;
#pragma unroll
    for (int c = 0; c < OW_D1; ++c) v += c_ow.Azx[r][c] * xa[c];
    mu[r] = v;
  }
#pragma unroll 2
  for (int c = 0; c < OW_D2; ++c) {
    const float zc = sz[c * M + b];
    const float4* col = reinterpret_cast<const float4*>(sAt + c * OW_D2);
#pragma unroll
    for (int q = 0; q < OW_D2 / 4; ++q) {
      const float4 a4 = col[q];
      mu[4 * q + 0] += a4.x * zc;
      mu[4 * q + 1] += a4.y * zc;
      mu[4 * q + 2] += a4.z * zc;
      mu[4 * q + 3] += a4.w * zc;
    }
  }
}

// Mean and variance over the group of every coordinate of mu (two passes, the
// variance about the mean); mu is written over the staged set, which every thread
// has finished reading. Results in s_m[56], s_v[56].
__device__ __forceinline__ void ow_group_moments(const float (&mu)[OW_D2], float* sz, int M, float* s_m,
                                                 float* s_v) {
  const int j = threadIdx.x, lane = j & 31, w = j >> 5, nw = blockDim.x >> 5;
  __syncthreads();  // every gather from the staged set is done
#pragma unroll
  for (int r = 0; r < OW_D2; ++r) sz[r * M + j] = mu[r];
  __syncthreads();
  const float invM = 1.f / (float)M;
  for (int d = w; d < OW_D2; d += nw) {
    float s = 0.f;
    for (int k = lane; k < M; k += 32) s += sz[d * M + k];
    const float m = warp_sum(s) * invM;
    float q = 0.f;
    for (int k = lane; k < M; k += 32) {
      const float e = sz[d * M + k] - m;
      q += e * e;
    }
    const float v = warp_sum(q) * invM;
    if (lane == 0) {
      s_m[d] = m;
      s_v[d] = v;
    }
  }
  __syncthreads();
}

// Half h (rows 28 h .. 28 h + 27) of mu = A_zx xa + A_zz z_b, written to mu_out (d2
// planes of N M floats) and to smu[rr * M + j]; 28 accumulators, so that two CTAs of 256
// threads fit an SM.
constexpr int OW_H = OW_D2 / 2;
__device__ __forceinline__ void ow_prior_mean_half(int h, const float (&xa)[OW_D1], const float* sz,
                                                   const float* sAt, int M, int b, float* mu_out, long long NM,
                                                   float* smu) {
  const int j = threadIdx.x;
  float acc[OW_H];
#pragma unroll
  for (int rr = 0; rr < OW_H; ++rr) {
    float v = 0.f;
#pragma unroll
    for (int c = 0; c < OW_D1; ++c) v += c_ow.Azx[h * OW_H + rr][c] * xa[c];
    acc[rr] = v;
  }
#pragma unroll 2
  for (int c = 0; c < OW_D2; ++c) {
    const float zc = sz[c * M + b];
    const float4* col = reinterpret_cast<const float4*>(sAt + c * OW_D2 + h * OW_H);
#pragma unroll
    for (int q = 0; q < OW_H / 4; ++q) {
      const float4 a4 = col[q];
      acc[4 * q + 0] += a4.x * zc;
      acc[4 * q + 1] += a4.y * zc;
      acc[4 * q + 2] += a4.z * zc;
      acc[4 * q + 3] += a4.w * zc;
    }
  }
#pragma unroll
  for (int rr = 0; rr < OW_H; ++rr) {
    mu_out[(long long)(h * OW_H + rr) * NM] = acc[rr];
    smu[rr * M + j] = acc[rr];
  }
}

// Mean and variance over the group of rows 28 h .. 28 h + 27 of mu, from smu (all
// threads have written it) into s_m, s_v.
__device__ __forceinline__ void ow_half_moments(int h, const float* smu, int M, float* s_m, float* s_v) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const float invM = 1.f / (float)M;
  for (int rr = w; rr < OW_H; rr += nw) {
    float s = 0.f;
    for (int k = lane; k < M; k += 32) s += smu[rr * M + k];
    const float m = warp_sum(s) * invM;
    float q = 0.f;
    for (int k = lane; k < M; k += 32) {
      const float e = smu[rr * M + k] - m;
      q += e * e;
    }
    const float v = warp_sum(q) * invM;
    if (lane == 0) {
      s_m[h * OW_H + rr] = m;
      s_v[h * OW_H + rr] = v;
    }
  }
}

struct OwShared {
  uint32_t cum[256];
  uint32_t redU[32];
  float red[8];
  float s_m[OW_D2], s_v[OW_D2], s_s[OW_D2], s_c[OW_D2], s_rl[OW_D2];
  float s_xa[OW_D1], s_xt[OW_D1];
  float s_sumls;
  int s_msel;
  uint32_t s_uin;
};

// The plain rule's selection of x_{t-1}^(i) among the ancestor's look-ahead draws and
// the local systematic resampling of the ancestor's inner set (its own weights: the x
// transition is free of z); writes sel, x_new, the indices (and the debug copy) and
// returns this thread's parent b. Every thread of the CTA (one a particle) calls it.
__device__ __forceinline__ int ow_select_resample(const StepArgs<float>& a, long long i, long long anc,
                                                  int32_t* __restrict__ bidx_out, OwShared& sh) {
  const int M = a.M, j = threadIdx.x, lane = j & 31;
  const float NEG = -INFINITY;
  const float LOG2E = (float)LOG2E_D;
  if (j < 32) {
    const int L = a.L;
    const float l0 = lane < L ? a.lwh_old[anc * L + lane] : NEG;
    const float l1 = lane + 32 < L ? a.lwh_old[anc * L + lane + 32] : NEG;
    const float mx = warp_max(fmaxf(l0, l1));
    const uint32_t c0 = lane < L ? (uint32_t)floorf(exp2_t((l0 - mx) * LOG2E) * a.scaleL) : 0u;
    const uint32_t c1 = lane + 32 < L ? (uint32_t)floorf(exp2_t((l1 - mx) * LOG2E) * a.scaleL) : 0u;
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
    const uint32_t wsel = philox(ctr(a.t - 1, (uint32_t)i, lane == 0 ? P_SEL : P_INNER, 0u, 0u), a.key).x;
    const uint32_t usel = __shfl_sync(FULL, wsel, 0);
    const uint64_t rhs = (uint64_t)usel * C;
    const unsigned b0 = __ballot_sync(FULL, ((uint64_t)s0 << 32) > rhs);
    const unsigned b1 = __ballot_sync(FULL, ((uint64_t)(s1 + tot0) << 32) > rhs);
    if (lane == 0) {
      int m = b0 ? __ffs(b0) - 1 : (b1 ? 32 + __ffs(b1) - 1 : L - 1);
      if (C == 0 || m >= L) {
        atomicOr(a.err, ERR_NUMERIC);
        m = L - 1;
      }
      sh.s_msel = m;
      a.sel[i] = m;
    }
    if (lane == 1) sh.s_uin = wsel;
  }
  __syncthreads();
  const int msel = sh.s_msel;
  if (j < a.xp) a.x_new[i * a.xp + j] = j < OW_D1 ? a.xbb_old[(anc * a.L + msel) * OW_D1 + j] : 0.f;
  const float al = a.lq_old[anc * M + j];
  const float amax = bmax(al, sh.red);
  uint32_t cw[1] = {(uint32_t)floorf(exp2_t((al - amax) * LOG2E) * a.scaleM)}, incl[1];
  bscan_planes<1>(cw, incl, sh.redU);
  sh.cum[j] = incl[0];
  __syncthreads();
  const uint32_t C = sh.cum[M - 1];
  if (C == 0 && j == 0) atomicOr(a.err, ERR_NUMERIC);
  const int b = sys_local_pick(sh.cum, M, C, M, j, sh.s_uin);
  bidx_out[i * M + j] = b;
  if (a.dbg_b) a.dbg_b[i * M + j] = b;
  return b;
}

// The group's feature row (x_{t-1} of the ancestor, x_t, y_t, m, v) once the moments
// are in sh.
__device__ __forceinline__ void ow_features(const StepArgs<float>& a, long long i, long long anc,
                                            float* __restrict__ feat, const OwShared& sh) {
  const int j = threadIdx.x;
  float* f = feat + i * OW_DIN;
  if (j < OW_D1) {
    f[j] = a.x_old[anc * a.xp + j];
    f[OW_D1 + j] = a.xbb_old[(anc * a.L + sh.s_msel) * OW_D1 + j];
  }
  if (j < OW_DY) f[2 * OW_D1 + j] = a.y_prev[j];
  if (j < OW_D2) {
    f[2 * OW_D1 + OW_DY + j] = sh.s_m[j];
    f[2 * OW_D1 + OW_DY + OW_D2 + j] = sh.s_v[j];
  }
}

// Stage 1: selection, local resampling, prior means and the group features (two CTAs
// of 256 threads an SM: at most 128 registers a thread).
__global__ void __launch_bounds__(256, 2)
    oaw_prepare_kernel(const __grid_constant__ StepArgs<float> a, int32_t* __restrict__ bidx_out,
                       float* __restrict__ feat, float* __restrict__ mu_out) {
  // [A_zz^T (56 x 56)][the staged set (56 x M)][half of mu (28 x M)]
  extern __shared__ __align__(16) float ow_sz[];
  __shared__ OwShared sh;
  const int M = a.M, j = threadIdx.x;
  const long long NM = a.N * (long long)M;
  float* sAt = ow_sz;
  float* sz = ow_sz + OW_AT_FLOATS;
  float* smu = sz + OW_D2 * M;
  ow_load_at(sAt);
  for (long long i = blockIdx.x; i < a.N; i += gridDim.x) {
    const long long anc = a.anc[i];
    ow_stage(a.z_old, NM, anc, M, sz);
    float xa[OW_D1];
#pragma unroll
    for (int c = 0; c < OW_D1; ++c) xa[c] = a.x_old[anc * a.xp + c];
    const int b = ow_select_resample(a, i, anc, bidx_out, sh);
    // ---- prior means and the group features ----
    for (int h = 0; h < 2; ++h) {
      ow_prior_mean_half(h, xa, sz, sAt, M, b, mu_out + i * M + j, NM, smu);
      __syncthreads();
      ow_half_moments(h, smu, M, sh.s_m, sh.s_v);
      __syncthreads();  // smu is rewritten by the next half
    }
    ow_features(a, i, anc, feat, sh);
    __syncthreads();  // the staged set and the shared words are reused by the next group
  }
}

// Stage 1 with the product A_zz z_b on the tensor cores (M = 128 or 256; used at 256). Per group the
// gathered parents z_b form the A operand (one row a particle; K = the 56 coordinates,
// padded to 64, in two chunks of 32), A_zz the B operand (N = 56 padded to 64, staged
// once per CTA), 3xTF32 (kind::tf32: A_lo B_hi + A_hi B_lo + A_hi B_hi) into an FP32
// accumulator in TMEM, 64 columns a 128-row tile; thread j then reads its row. Operands
// are K-major without swizzle (the layout of dpf_tc.cuh). A wait that gives up sets
// ERR_TIMEOUT, waits once more for the MMAs in flight, releases the TMEM and returns.
constexpr int OWT_KC16 = 8;                  // 16-byte chunks of one 128-byte operand row (32 TF32)
constexpr int OWT_SPIN = 1 << 22;
constexpr uint32_t OWT_B_BYTES = 64u * 128u;  // one K chunk of B: 64 rows x 128 bytes
constexpr uint32_t OWT_TILE_BYTES = 128u * 128u;  // one K chunk of a 128-row A tile

__global__ void __launch_bounds__(256, 2)
    oaw_prepare_tc_kernel(const __grid_constant__ StepArgs<float> a, int32_t* __restrict__ bidx_out,
                          float* __restrict__ feat, float* __restrict__ mu_out) {
  // [A hi (M rows x 128 B)][A lo][B hi (2 chunks x 64 rows x 128 B)][B lo]; the A region
  // doubles as the staging tile of the group moments once the MMAs have completed
  extern __shared__ __align__(1024) unsigned char owt_sm[];
  __shared__ OwShared sh;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_taddr;
  const int M = a.M, j = threadIdx.x, w = j >> 5;
  const long long NM = a.N * (long long)M;
  const uint32_t a_bytes = (uint32_t)M * 128u;
  unsigned char* a_hi = owt_sm;
  unsigned char* a_lo = owt_sm + a_bytes;
  unsigned char* b_hi = owt_sm + 2 * a_bytes;
  unsigned char* b_lo = b_hi + 2 * OWT_B_BYTES;
  const uint32_t ncols = (uint32_t)(M / 128) * 64u;
  if (w == 0) {
    tc::tmem_alloc(&s_taddr, ncols);
    tc::tmem_relinquish();
  }
  if (j == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  for (int e = j; e < 64 * 64; e += blockDim.x) {  // B = A_zz, zero-padded to 64 x 64
    const int n = e >> 6, k = e & 63;
    const float v = (n < OW_D2 && k < OW_D2) ? c_ow.Azz[n][k] : 0.f;
    float h, l;
    tc::split_tf32(v, h, l);
    const uint32_t off = (uint32_t)(k >> 5) * OWT_B_BYTES + tc::kmajor_offset(n, 4 * (k & 31), OWT_KC16);
    *(float*)(b_hi + off) = h;
    *(float*)(b_lo + off) = l;
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = s_taddr;
  const uint32_t idesc = tc::instr_desc(tc::FMT_TF32, 128, 64);
  uint32_t phase = 0;
  int ok = 1;
  for (long long i = blockIdx.x; i < a.N; i += gridDim.x) {
    const long long anc = a.anc[i];
    float xa[OW_D1];
#pragma unroll
    for (int c = 0; c < OW_D1; ++c) xa[c] = a.x_old[anc * a.xp + c];
    const int b = ow_select_resample(a, i, anc, bidx_out, sh);
    const float* zp = a.z_old + anc * M + b;  // the parent's coordinate c at zp[c NM]
    for (int q = 0; q < 2 && ok; ++q) {
      // this thread's operand row of chunk q: coordinates 32 q .. 32 q + 31 (zeros past 55)
#pragma unroll
      for (int c4 = 0; c4 < 8; ++c4) {
        const int c0 = 32 * q + 4 * c4;
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = c0 + u < OW_D2 ? zp[(long long)(c0 + u) * NM] : 0.f;
        float4 hi, lo;
        tc::split_tf32(v[0], hi.x, lo.x);
        tc::split_tf32(v[1], hi.y, lo.y);
        tc::split_tf32(v[2], hi.z, lo.z);
        tc::split_tf32(v[3], hi.w, lo.w);
        const uint32_t off = tc::kmajor_offset(j, 16 * c4, OWT_KC16);
        *(float4*)(a_hi + off) = hi;
        *(float4*)(a_lo + off) = lo;
      }
      tc::fence_proxy_async();
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
      if (j == 0) {
        const uint32_t sbh = smem_addr(b_hi) + (uint32_t)q * OWT_B_BYTES;
        const uint32_t sbl = smem_addr(b_lo) + (uint32_t)q * OWT_B_BYTES;
        for (int t = 0; t < M / 128; ++t) {
          const uint32_t sah = smem_addr(a_hi) + (uint32_t)t * OWT_TILE_BYTES;
          const uint32_t sal = smem_addr(a_lo) + (uint32_t)t * OWT_TILE_BYTES;
          const uint32_t d = taddr + (uint32_t)(64 * t);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t off = (uint32_t)ks * 256u;
            const uint32_t acc = (q > 0 || ks > 0) ? 1u : 0u;
            tc::mma_tf32(d, tc::smem_desc(sal + off, OWT_KC16), tc::smem_desc(sbh + off, OWT_KC16), idesc, acc);
            tc::mma_tf32(d, tc::smem_desc(sah + off, OWT_KC16), tc::smem_desc(sbl + off, OWT_KC16), idesc, 1);
            tc::mma_tf32(d, tc::smem_desc(sah + off, OWT_KC16), tc::smem_desc(sbh + off, OWT_KC16), idesc, 1);
          }
        }
        tc::commit(&bar);
      }
      const bool done = tc::bar_wait(&bar, phase, OWT_SPIN);
      phase ^= 1u;
      tc::fence_after();
      ok = __syncthreads_and(done ? 1 : 0);  // every thread saw the MMAs finish before the tiles change
    }
    if (!ok) break;
    // this thread's row of mu: the accumulator, then + A_zx x_{t-1}
    float mu[OW_D2];
    {
      const uint32_t row = taddr + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(64 * (j >> 7));
      float v[16];
#pragma unroll
      for (int c0 = 0; c0 < 48; c0 += 16) {
        tc::ld16(row + (uint32_t)c0, v);
#pragma unroll
        for (int u = 0; u < 16; ++u) mu[c0 + u] = v[u];
      }
      float v8[8];
      tc::ld8(row + 48u, v8);
#pragma unroll
      for (int u = 0; u < 8; ++u) mu[48 + u] = v8[u];
    }
#pragma unroll
    for (int r = 0; r < OW_D2; ++r) {
#pragma unroll
      for (int c = 0; c < OW_D1; ++c) mu[r] += c_ow.Azx[r][c] * xa[c];
      mu_out[r * NM + i * M + j] = mu[r];
    }
    tc::fence_before();  // the TMEM reads are ordered before the barriers that follow
    ow_group_moments(mu, (float*)owt_sm, M, sh.s_m, sh.s_v);
    ow_features(a, i, anc, feat, sh);
    __syncthreads();  // the A region and the shared words are reused by the next group
  }
  if (!ok) {
    if (j == 0) atomicOr(a.err, ERR_TIMEOUT);
    tc::bar_wait(&bar, phase ^ 1u, OWT_SPIN);  // a second bound for MMAs still in flight
  }
  tc::fence_before();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(taddr, ncols);
}

// Stage 3: the mapped draws and their normalised importance weights. DIAG: Q_z is
// diagonal (the normals are consumed as they come; two CTAs an SM).
template <bool DIAG>
__global__ void __launch_bounds__(256, DIAG ? 2 : 1)
    oaw_update_kernel(const __grid_constant__ StepArgs<float> a, const float* __restrict__ mu_in,
                      const float* __restrict__ feat, const float* __restrict__ out, int centre) {
  __shared__ OwShared sh;
  const int M = a.M, j = threadIdx.x, lane = j & 31;
  const long long NM = a.N * (long long)M;
  for (long long i = blockIdx.x; i < a.N; i += gridDim.x) {
    if (j < OW_D2) {
      const float ls = fminf(fmaxf(out[i * OW_DOUT + j], kLogSigMin), kLogSigMax);
      sh.s_s[j] = expf(ls);
      sh.s_c[j] = out[i * OW_DOUT + OW_D2 + j];
      sh.s_m[j] = feat[i * OW_DIN + 2 * OW_D1 + OW_DY + j];
      sh.s_rl[j] = 1.f / c_ow.Lqz[j][j];
    }
    if (j < 32) {  // sum of the clamped log-scales
      float v = 0.f;
      for (int d = lane; d < OW_D2; d += 32) v += fminf(fmaxf(out[i * OW_DOUT + d], kLogSigMin), kLogSigMax);
      v = warp_sum(v);
      if (lane == 0) sh.s_sumls = v;
    }
    if (j < OW_D1) sh.s_xt[j] = a.x_new[i * a.xp + j];
    __syncthreads();
    float xt[OW_D1];
#pragma unroll
    for (int c = 0; c < OW_D1; ++c) xt[c] = sh.s_xt[c];
    const float* mup = mu_in + i * M + j;
    float* zn = a.z_new + i * M + j;
    float hz[OW_DY];
#pragma unroll
    for (int q = 0; q < OW_DY; ++q) hz[q] = 0.f;
    float e2 = 0.f, lpz = 0.f;
    if constexpr (DIAG) {
      // diagonal Q_z: coordinate by coordinate as the normals come, four a Philox block
      // (the same words and order as normals<56>); the prior means are all loaded first
      float muv[OW_D2];
#pragma unroll
      for (int r = 0; r < OW_D2; ++r) muv[r] = mup[r * NM];
#pragma unroll
      for (int bk = 0; bk < OW_D2 / 4; ++bk) {
        const uint4 w = philox(ctr(a.t - 1, (uint32_t)i, P_PROP, (uint32_t)j, (uint32_t)bk), a.key);
        float ev[4];
        box_muller(w.x, w.y, ev[0], ev[1]);
        box_muller(w.z, w.w, ev[2], ev[3]);
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          const int r = 4 * bk + q4;
          const float eps = ev[q4], lrr = c_ow.Lqz[r][r];
          e2 += eps * eps;
          const float mu = muv[r], k = centre ? mu : sh.s_m[r];
          const float z = k + sh.s_c[r] + sh.s_s[r] * (mu + eps * lrr - k);
          zn[r * NM] = z;
#pragma unroll
          for (int q = 0; q < OW_DY; ++q) hz[q] += c_ow.Hz[q][r] * z;
          const float u = (z - mu) * sh.s_rl[r];
          lpz += u * u;
        }
      }
    } else {  // a full Q_z: L_qz eps, then forward substitution
      float le[OW_D2];  // eps, then L_qz eps, then z - mu, then L_qz^-1 (z - mu)
      normals<OW_D2>(a.key, a.t - 1, (uint32_t)i, P_PROP, (uint32_t)j, le);
#pragma unroll
      for (int r = 0; r < OW_D2; ++r) e2 += le[r] * le[r];
#pragma unroll
      for (int r = OW_D2 - 1; r >= 0; --r) {  // row r reads eps_0 .. eps_r, not yet overwritten
        float v = 0.f;
#pragma unroll
        for (int c = 0; c <= r; ++c) v += c_ow.Lqz[r][c] * le[c];
        le[r] = v;
      }
#pragma unroll
      for (int r = 0; r < OW_D2; ++r) {
        const float mu = mup[r * NM], k = centre ? mu : sh.s_m[r];
        const float z = k + sh.s_c[r] + sh.s_s[r] * (mu + le[r] - k);
        zn[r * NM] = z;
#pragma unroll
        for (int q = 0; q < OW_DY; ++q) hz[q] += c_ow.Hz[q][r] * z;
        le[r] = z - mu;
      }
#pragma unroll
      for (int r = 0; r < OW_D2; ++r) {  // forward substitution in place
        float v = le[r];
#pragma unroll
        for (int c = 0; c < r; ++c) v -= c_ow.Lqz[r][c] * le[c];
        le[r] = v / c_ow.Lqz[r][r];
        lpz += le[r] * le[r];
      }
    }
    float hx[OW_DY];
    h_x(c_ow, xt, hx);
    float res[OW_DY];
#pragma unroll
    for (int q = 0; q < OW_DY; ++q) res[q] = a.y_prev[q] - hx[q] - hz[q];
    float lpy = 0.f;
#pragma unroll
    for (int q = 0; q < OW_DY; ++q) {
      float v = 0.f;
#pragma unroll
      for (int c = 0; c <= q; ++c) v += c_ow.LrInv[q][c] * res[c];
      lpy += v * v;
    }
    const float lr = -0.5f * lpz + 0.5f * e2 + sh.s_sumls - 0.5f * lpy;
    const float lmax = bmax(lr, sh.red);
    const float se = bsum(expf(lr - lmax), sh.red);
    const float lq = lr - (lmax + logf(se));
    a.lq_new[i * M + j] = lq;
    if (!(lq == lq)) atomicOr(a.err, ERR_NUMERIC);
    __syncthreads();  // the shared words are reused by the next group
  }
}

// Training rows from the last inner update: per inner particle the group features,
// (z_t, mu, m) and w = exp(lq_t) / N.
struct OwRecord {
  const float *x_old, *x_new, *z_old, *z_new, *lq_new, *y_prev;
  const int32_t *anc_prev, *bidx;
  long long N, i0, n_outer;
  int M, xp;
  float *G, *Z, *w;
};

__global__ void __launch_bounds__(256) oaw_record_kernel(const __grid_constant__ OwRecord r) {
  extern __shared__ __align__(16) float ow_sz[];  // [A_zz^T][the staged set]
  __shared__ OwShared sh;
  const int M = r.M, j = threadIdx.x;
  const long long NM = r.N * (long long)M;
  float* sAt = ow_sz;
  float* sz = ow_sz + OW_AT_FLOATS;
  ow_load_at(sAt);
  for (long long q = blockIdx.x; q < r.n_outer; q += gridDim.x) {
    const long long i = r.i0 + q;
    const long long anc = r.anc_prev[i];
    ow_stage(r.z_old, NM, anc, M, sz);
    if (j < OW_D1) {
      sh.s_xa[j] = r.x_old[anc * r.xp + j];
      sh.s_xt[j] = r.x_new[i * r.xp + j];
    }
    __syncthreads();
    float xa[OW_D1];
#pragma unroll
    for (int c = 0; c < OW_D1; ++c) xa[c] = sh.s_xa[c];
    float mu[OW_D2];
    ow_prior_mean(xa, sz, sAt, M, r.bidx[i * M + j], mu);
    ow_group_moments(mu, sz, M, sh.s_m, sh.s_v);
    const long long e = q * M + j;
    float* g = r.G + e * OW_DIN;
#pragma unroll
    for (int c = 0; c < OW_D1; ++c) {
      g[c] = sh.s_xa[c];
      g[OW_D1 + c] = sh.s_xt[c];
    }
#pragma unroll
    for (int c = 0; c < OW_DY; ++c) g[2 * OW_D1 + c] = r.y_prev[c];
    float* zr = r.Z + e * 3 * OW_D2;
#pragma unroll 8
    for (int d = 0; d < OW_D2; ++d) {
      g[2 * OW_D1 + OW_DY + d] = sh.s_m[d];
      g[2 * OW_D1 + OW_DY + OW_D2 + d] = sh.s_v[d];
      zr[d] = r.z_new[d * NM + i * M + j];
      zr[OW_D2 + d] = mu[d];
      zr[2 * OW_D2 + d] = sh.s_m[d];
    }
    r.w[e] = expf(r.lq_new[i * M + j]) / (float)r.N;
    __syncthreads();
  }
}

// The dynamic shared memory a launch of k needs: raised per kernel (never lowered, so
// that a launch already made with more keeps its size), the largest request remembered
// per kernel function (kernels of one signature share no cache).
template <typename K>
cudaError_t ow_attr(K k, size_t smem) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, size_t>> set;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& e : set)
    if (e.first == (const void*)k) {
      if (smem <= e.second) return cudaSuccess;
      const cudaError_t r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (r == cudaSuccess) e.second = smem;
      return r;
    }
  const cudaError_t r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (r == cudaSuccess) set.emplace_back((const void*)k, smem);
  return r;
}

// A persistent grid: as many CTAs as fit on the device at once (each copies A_zz^T
// once), at most one a group.
template <typename K>
cudaError_t ow_grid(K k, int nt, size_t smem, long long n, unsigned* grid) {
  int nb = 0, dev = 0, nsm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, nt, smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  *grid = (unsigned)std::min<long long>(n, (long long)std::max(nb, 1) * nsm);
  return cudaSuccess;
}

}  // namespace

bool oa_wide_shape(const Ctx& x) {
  return x.prec == DPF_F32 && x.d1 == OW_D1 && x.d2 == OW_D2 && x.dy == OW_DY && !x.hm.xz && x.M % 32 == 0 &&
         x.M >= 32 && x.M <= 256;
}

dpf_status oa_wide_step(Ctx& x, dpf_proposal& p) {
  if (p.din != OW_DIN || p.dout != OW_DOUT)
    return set_error(DPF_E_INVALID, "amortised wide step: the proposal's sizes do not match (8, 56, 8)");
  StepArgs<float> a{};
  VariantImpl<float, OW_D1, OW_D2, OW_DY, 0>::fill_args(x, a);
  a.xp = x.xp;
  cudaError_t e = cudaMemcpyToSymbolAsync(c_ow, x.d_mconst, sizeof(OwConst), 0, cudaMemcpyDeviceToDevice, x.stream);
  if (e != cudaSuccess) return cuda_error(e, "amortised wide step: model constants");
  unsigned grid = 0, grid_u = 0;
  // A_zz z_b on the tensor cores at M = 256 (as fast as the CUDA-core form there: the pass
  // is bound by its per-group chain of dependent steps, not by the product; at M = 128 the
  // tensor-core form, three CTAs an SM, was the slower)
  if (x.tensor_cores && x.M == 256) {
    const size_t sm = 2 * (size_t)x.M * 128 + 4 * (size_t)OWT_B_BYTES;
    e = ow_attr(oaw_prepare_tc_kernel, sm);
    if (e == cudaSuccess) e = ow_grid(oaw_prepare_tc_kernel, x.M, sm, x.N, &grid);
    if (e != cudaSuccess) return cuda_error(e, "amortised wide step: launch shape");
    oaw_prepare_tc_kernel<<<grid, x.M, sm, x.stream>>>(a, (int32_t*)x.oa_bidx, (float*)x.oa_feat,
                                                      (float*)x.oa_mu);
  } else {
    const size_t sm = sizeof(float) * ((size_t)(OW_D2 + OW_H) * x.M + OW_AT_FLOATS);
    e = ow_attr(oaw_prepare_kernel, sm);
    if (e == cudaSuccess) e = ow_grid(oaw_prepare_kernel, x.M, sm, x.N, &grid);
    if (e != cudaSuccess) return cuda_error(e, "amortised wide step: launch shape");
    oaw_prepare_kernel<<<grid, x.M, sm, x.stream>>>(a, (int32_t*)x.oa_bidx, (float*)x.oa_feat, (float*)x.oa_mu);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "amortised wide prepare launch");
  dpf_status st = proposal_forward_rows(p, (const float*)x.oa_feat, x.N, (float*)x.oa_hidden, (float*)x.oa_out,
                                        x.err, x.stream);
  if (st) return st;
  const bool diag = reinterpret_cast<const OwConst*>(x.mconst.data())->diag_qz != 0;
  auto upd = diag ? oaw_update_kernel<true> : oaw_update_kernel<false>;
  e = ow_grid(upd, x.M, 0, x.N, &grid_u);
  if (e != cudaSuccess) return cuda_error(e, "amortised wide step: launch shape");
  upd<<<grid_u, x.M, 0, x.stream>>>(
      a, (const float*)x.oa_mu, (const float*)x.oa_feat, (const float*)x.oa_out, p.centre);
  return cuda_error(cudaGetLastError(), "amortised wide update launch");
}

dpf_status oa_wide_record(Ctx& x, long long i0, long long n_outer, float* G, float* Z, float* w) {
  const long long t = x.t;
  OwRecord r{};
  r.x_old = (const float*)x.x[t % 2];
  r.x_new = (const float*)x.x[(t + 1) % 2];
  r.z_old = (const float*)x.z[t % 2];
  r.z_new = (const float*)x.z[(t + 1) % 2];
  r.lq_new = (const float*)x.lq[(t + 1) % 2];
  r.y_prev = (const float*)x.yb + ((t + 1) % 2) * x.dy;
  r.anc_prev = x.anc_prev;
  r.bidx = x.dbg_b;
  r.N = x.N;
  r.i0 = i0;
  r.n_outer = n_outer;
  r.M = x.M;
  r.xp = x.xp;
  r.G = G;
  r.Z = Z;
  r.w = w;
  cudaError_t e = cudaMemcpyToSymbolAsync(c_ow, x.d_mconst, sizeof(OwConst), 0, cudaMemcpyDeviceToDevice, x.stream);
  if (e != cudaSuccess) return cuda_error(e, "amortised wide record: model constants");
  const size_t sm = sizeof(float) * ((size_t)OW_D2 * x.M + OW_AT_FLOATS);
  e = ow_attr(oaw_record_kernel, sm);
  unsigned grid = 0;
  if (e == cudaSuccess) e = ow_grid(oaw_record_kernel, x.M, sm, n_outer, &grid);
  if (e != cudaSuccess) return cuda_error(e, "amortised wide record: launch shape");
  oaw_record_kernel<<<grid, x.M, sm, x.stream>>>(r);
  return cuda_error(cudaGetLastError(), "amortised wide record launch");
}

}  // namespace dpf
