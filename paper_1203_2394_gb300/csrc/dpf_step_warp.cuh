// The step kernel in its warp-per-group form (M <= 256): one warp owns one
// outer particle i at a time and each lane owns PPL of its inner particles
// (k = lane + 32 p) in registers, so every reduction and scan of the step is a
// warp shuffle and no block-wide barrier is needed. The warps are persistent;
// each has one shared-memory stage into which the next group's source rows are
// bulk-copied (cp.async.bulk + mbarrier) as soon as the current group has
// consumed them, overlapping the gather with the look-ahead arithmetic.
//
// The arithmetic is that of step_kernel (the same Fig. 4 steps, the same
// random-number keys and resampling rules). For a model whose x transition does
// not depend on z, the z-mean weights simplify: with alpha = lq + const_m the
// outer-and-draw weight of draw m is S_m / sum_m' S_m' (S_m = sum_k e^(m,k)), so
// beta_k = sum_m pi_m e^(m,k) / S_m = sum_m e^(m,k) / sum_(m,k) e^(m,k), one pass.
#pragma once

#include <cstring>
#include <type_traits>

#include "dpf_step.cuh"

namespace dpf {

constexpr int WARPS_PER_CTA = 4;
// Row stride (elements) of the lane-partials table part[row][PART_STRIDE]: rows start on
// 16 bytes (vector loads of a row) and a row's 32 lane entries fall on distinct banks.
constexpr int PART_STRIDE = 36;

// CTAs per SM the register allocation aims for: 4 (128 registers a thread)
// unless a lane holds many coordinates of many particles, where 2 (255) avoids
// spilling them.
template <int PPL, int D2>
constexpr int warp_min_blocks() { return PPL * D2 >= 48 ? 2 : 4; }

// Per-warp shared-memory carve-up (bytes from the warp's region), on the host.
template <typename T, int D1, int D2, int DY, bool XZ>
inline size_t warp_geometry(int M, int L, StepArgs<T>* a, bool first = false) {
  auto r16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
  const int xp = (int)((D1 * sizeof(T) + 15) / 16 * 16 / sizeof(T));
  size_t so = 0;
  const uint32_t sz = (uint32_t)so; so += r16(sizeof(T) * D2 * M);
  const uint32_t slq = (uint32_t)so; so += r16(sizeof(T) * M);
  const uint32_t sx = (uint32_t)so; so += r16(sizeof(T) * xp);
  const uint32_t slwh = (uint32_t)so; so += r16(sizeof(T) * L);
  const uint32_t sxbb = (uint32_t)so; so += r16(sizeof(T) * L * D1);
  size_t o = so;  // the stage comes first
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += r16(bytes);
    return (uint32_t)at;
  };
  const uint32_t cum = take(sizeof(uint32_t) * M), fs = take(XZ ? sizeof(T) * D1 * M : 0),
                 xw = take(sizeof(T) * L * D1), cw = take(sizeof(T) * L * DY),
                 xbs = take(sizeof(T) * L * D1), row = take(sizeof(T) * L * 5),
                 part = take(sizeof(T) * 2 * PART_STRIDE * L),
                 zrow = take(sizeof(T) * D2 * (D1 + D2 + DY));
  const size_t warp_bytes = r16(o);
  if (a) {
    a->xp = xp;
    a->stage_bytes = (uint32_t)warp_bytes;  // per-warp region size
    a->stage_tx = (uint32_t)(sizeof(T) * (D2 * M + M + xp + (first ? 0 : L + L * D1)));
    a->off_stage = 0; a->off_sz = sz; a->off_slq = slq; a->off_sx = sx; a->off_slwh = slwh;
    a->off_sxbb = sxbb;
    a->off_cum = cum; a->off_kd = fs; a->off_xw = xw; a->off_cw = cw; a->off_xbs = xbs;
    a->off_row = row; a->off_part = part; a->off_zrow = zrow;
  }
  return warp_bytes * WARPS_PER_CTA;
}

// log2 for the per-group scalar math: the hardware approximation in FP32 (absolute
// error about 2^-22, far inside the log-weight tolerance), the accurate one in FP64.
__device__ __forceinline__ float log2_fast(float x) { return lg2_approx(x); }
__device__ __forceinline__ double log2_fast(double x) { return log2(x); }

// Vector moves of P consecutive elements (16-byte chunks where possible). float and
// double move as float4 / float2 / double2; 32-bit integers as uint4 / uint2 (the casts
// between uint32_t and int32_t keep the bits).
template <typename T, int P>
__device__ __forceinline__ void vld(const T* src, T (&out)[P]) {
  if constexpr (std::is_same<T, float>::value && P % 4 == 0) {
#pragma unroll
    for (int q = 0; q < P / 4; ++q) {
      const float4 v = reinterpret_cast<const float4*>(src)[q];
      out[4 * q + 0] = v.x;
      out[4 * q + 1] = v.y;
      out[4 * q + 2] = v.z;
      out[4 * q + 3] = v.w;
    }
  } else if constexpr (std::is_same<T, float>::value && P == 2) {
    const float2 v = *reinterpret_cast<const float2*>(src);
    out[0] = v.x;
    out[1] = v.y;
  } else if constexpr (std::is_same<T, double>::value && P % 2 == 0) {
#pragma unroll
    for (int q = 0; q < P / 2; ++q) {
      const double2 v = reinterpret_cast<const double2*>(src)[q];
      out[2 * q + 0] = v.x;
      out[2 * q + 1] = v.y;
    }
  } else if constexpr (std::is_integral<T>::value && sizeof(T) == 4 && P % 4 == 0) {
#pragma unroll
    for (int q = 0; q < P / 4; ++q) {
      const uint4 v = reinterpret_cast<const uint4*>(src)[q];
      out[4 * q + 0] = (T)v.x;
      out[4 * q + 1] = (T)v.y;
      out[4 * q + 2] = (T)v.z;
      out[4 * q + 3] = (T)v.w;
    }
  } else if constexpr (std::is_integral<T>::value && sizeof(T) == 4 && P == 2) {
    const uint2 v = *reinterpret_cast<const uint2*>(src);
    out[0] = (T)v.x;
    out[1] = (T)v.y;
  } else {
#pragma unroll
    for (int q = 0; q < P; ++q) out[q] = src[q];
  }
}
template <typename T, int P>
__device__ __forceinline__ void vst(T* dst, const T (&in)[P]) {
  if constexpr (std::is_same<T, float>::value && P % 4 == 0) {
#pragma unroll
    for (int q = 0; q < P / 4; ++q)
      reinterpret_cast<float4*>(dst)[q] = make_float4(in[4 * q], in[4 * q + 1], in[4 * q + 2], in[4 * q + 3]);
  } else if constexpr (std::is_same<T, float>::value && P == 2) {
    *reinterpret_cast<float2*>(dst) = make_float2(in[0], in[1]);
  } else if constexpr (std::is_same<T, double>::value && P % 2 == 0) {
#pragma unroll
    for (int q = 0; q < P / 2; ++q) reinterpret_cast<double2*>(dst)[q] = make_double2(in[2 * q], in[2 * q + 1]);
  } else if constexpr (std::is_integral<T>::value && sizeof(T) == 4 && P % 4 == 0) {
#pragma unroll
    for (int q = 0; q < P / 4; ++q)
      reinterpret_cast<uint4*>(dst)[q] = make_uint4((uint32_t)in[4 * q], (uint32_t)in[4 * q + 1],
                                                    (uint32_t)in[4 * q + 2], (uint32_t)in[4 * q + 3]);
  } else if constexpr (std::is_integral<T>::value && sizeof(T) == 4 && P == 2) {
    *reinterpret_cast<uint2*>(dst) = make_uint2((uint32_t)in[0], (uint32_t)in[1]);
  } else {
#pragma unroll
    for (int q = 0; q < P; ++q) dst[q] = in[q];
  }
}

// Local systematic resampling of M particles into M by offspring ranges. With the
// integer rule out[j] = min{ k : cum_k M 2^16 > (j 2^16 + u16) C }, source k is
// chosen by the destinations j in [J(cum_{k-1}), J(cum_k)), where
//   J(c) = #{ j in [0, M) : (j 2^16 + u16) C < c M 2^16 }
// counts the systematic points below the cumulative weight c. J is estimated in
// single precision (within one of the count: c M / C <= M carries a relative error
// of a few 2^-24) and settled by one exact 64-bit comparison on each side.
__device__ __forceinline__ int sys_points_below(uint32_t c, uint32_t C, int M, uint32_t u16,
                                                float m_over_C, float u_frac) {
  int J = __float2int_ru(fmaf(__uint2float_rn(c), m_over_C, -u_frac));
  J = min(max(J, 0), M);
  const uint64_t R = ((uint64_t)c * (uint32_t)M) << 16;
  if (J > 0 && ((((uint64_t)(J - 1)) << 16) + u16) * C >= R)
    --J;
  else if (J < M && ((((uint64_t)J) << 16) + u16) * C < R)
    ++J;
  return J;
}

// The ancestors bidx of this lane's destinations j = k0 .. k0 + P - 1, from the
// inclusive cumulative weights loc of its sources k0 .. k0 + P - 1 (the same k).
// Source k marks slot J(cum_k) with k + 1 when it is the last source with that count;
// out[j] = #{ k : J(cum_k) <= j } is then the running maximum of the slots. `slot`
// is M words of the warp's shared memory. Warp-wide; every lane takes part.
template <int P>
__device__ __forceinline__ void sys_local_offspring(const uint32_t (&loc)[P], uint32_t C, int M,
                                                    uint32_t u16, int k0, bool act, int lane,
                                                    int* slot, int (&bidx)[P]) {
  const float m_over_C = __fdividef((float)M, __uint2float_rn(C));
  const float u_frac = (float)u16 * 0x1p-16f;
  int J[P];
#pragma unroll
  for (int p = 0; p < P; ++p) J[p] = act ? sys_points_below(loc[p], C, M, u16, m_over_C, u_frac) : M;
  int Jn = __shfl_down_sync(FULL, J[0], 1);
  if (lane == 31) Jn = M;
  int zero[P];
#pragma unroll
  for (int p = 0; p < P; ++p) zero[p] = 0;
  if (act) vst<int, P>(slot + k0, zero);
  __syncwarp();
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int nxt = p + 1 < P ? J[p + 1] : Jn;
    if (J[p] < nxt && J[p] < M) slot[J[p]] = k0 + p + 1;
  }
  __syncwarp();
  int s[P];
  if (act) vld<int, P>(slot + k0, s);
  else {
#pragma unroll
    for (int p = 0; p < P; ++p) s[p] = 0;
  }
#pragma unroll
  for (int p = 1; p < P; ++p) s[p] = max(s[p], s[p - 1]);
  int v = s[P - 1];  // inclusive warp max-scan of the lanes' running maxima
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v = max(v, n);
  }
  int before = __shfl_up_sync(FULL, v, 1);
  if (lane == 0) before = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) bidx[p] = min(max(s[p], before), M - 1);
}

// acc[p] += a * x[p] for all p: packed FP32x2 FMAs on float pairs, scalar otherwise.
template <typename T, int P>
__device__ __forceinline__ void axpy(T a, const T (&x)[P], T (&acc)[P]) {
  if constexpr (sizeof(T) == 4 && P % 2 == 0) {
#pragma unroll
    for (int p = 0; p < P; p += 2) {
      const float2 r = __ffma2_rn(make_float2(a, a), make_float2(x[p], x[p + 1]),
                                  make_float2(acc[p], acc[p + 1]));
      acc[p] = r.x;
      acc[p + 1] = r.y;
    }
  } else {
#pragma unroll
    for (int p = 0; p < P; ++p) acc[p] = fma(a, x[p], acc[p]);
  }
}
// acc[p] -= d[p]^2 with d[p] = c + g[p] (c broadcast): the quadratic-form step
template <typename T, int P>
__device__ __forceinline__ void sub_sq(T c, const T (&g)[P], T (&acc)[P]) {
  if constexpr (sizeof(T) == 4 && P % 2 == 0) {
#pragma unroll
    for (int p = 0; p < P; p += 2) {
      const float2 d = __fadd2_rn(make_float2(c, c), make_float2(g[p], g[p + 1]));
      const float2 r = __ffma2_rn(make_float2(-d.x, -d.y), d, make_float2(acc[p], acc[p + 1]));
      acc[p] = r.x;
      acc[p + 1] = r.y;
    }
  } else {
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const T d = c + g[p];
      acc[p] = fma(-d, d, acc[p]);
    }
  }
}

// acc[p] += x[p] (packed FP32x2 adds on float pairs)
template <typename T, int P>
__device__ __forceinline__ void add_to(const T (&x)[P], T (&acc)[P]) {
  if constexpr (sizeof(T) == 4 && P % 2 == 0) {
#pragma unroll
    for (int p = 0; p < P; p += 2) {
      const float2 r = __fadd2_rn(make_float2(acc[p], acc[p + 1]), make_float2(x[p], x[p + 1]));
      acc[p] = r.x;
      acc[p + 1] = r.y;
    }
  } else {
#pragma unroll
    for (int p = 0; p < P; ++p) acc[p] += x[p];
  }
}
// Sum of P values as a pairwise tree (halves added element by element, packed on float
// pairs), P a power of two.
template <typename T, int P>
__device__ __forceinline__ T tree_sum(const T (&x)[P]) {
  if constexpr (P == 1) {
    return x[0];
  } else {
    T h[P / 2];
#pragma unroll
    for (int p = 0; p < P / 2; ++p) h[p] = x[p];
    T u[P / 2];
#pragma unroll
    for (int p = 0; p < P / 2; ++p) u[p] = x[P / 2 + p];
    add_to<T, P / 2>(u, h);
    return tree_sum<T, P / 2>(h);
  }
}
// Largest of P values as a pairwise tree, P a power of two.
template <typename T, int P>
__device__ __forceinline__ T tree_max(const T (&x)[P]) {
  if constexpr (P == 1) {
    return x[0];
  } else {
    T h[P / 2];
#pragma unroll
    for (int p = 0; p < P / 2; ++p) h[p] = fmax(x[p], x[P / 2 + p]);
    return tree_max<T, P / 2>(h);
  }
}
// Reduce each row m < L of the 32 lane partials part[m][0..31] (stride PART_STRIDE) to
// out[m], by their maximum (MAXR) or sum: for L <= 16 lanes m and m + 16 each take half of
// row m (vector loads) and combine by one shuffle, else lane m takes all of row m.
template <typename T, bool MAXR>
__device__ __forceinline__ void reduce_rows(const T* part, int L, int lane, T* out) {
  if (L <= 16) {
    const int m = lane & 15, h = lane >> 4;
    T r = MAXR ? neg_inf<T>() : T(0);
    if (m < L) {
      T x[16];
      vld<T, 16>(part + m * PART_STRIDE + 16 * h, x);
      r = MAXR ? tree_max<T, 16>(x) : tree_sum<T, 16>(x);
    }
    const T o = __shfl_xor_sync(FULL, r, 16);
    r = MAXR ? fmax(r, o) : r + o;
    if (h == 0 && m < L) out[m] = r;
  } else {
    for (int m = lane; m < L; m += 32) {
      T x[16];
      vld<T, 16>(part + m * PART_STRIDE, x);
      const T lo = MAXR ? tree_max<T, 16>(x) : tree_sum<T, 16>(x);
      vld<T, 16>(part + m * PART_STRIDE + 16, x);
      const T hi = MAXR ? tree_max<T, 16>(x) : tree_sum<T, 16>(x);
      out[m] = MAXR ? fmax(lo, hi) : lo + hi;
    }
  }
}

// Issue the bulk copies of one group's source rows into a warp's stage (lane 0).
template <typename T, int D1, int D2>
__device__ __forceinline__ void warp_stage(const StepArgs<T>& a, unsigned char* st, uint64_t* bar,
                                           long long src, int lane) {
  // warp-wide: lane 0 arms the barrier with the stage's bytes, one lane a copy
  const int M = a.M, L = a.L;
  const long long NM = a.N * (long long)M;
  if (lane == 0) mbar_arrive_tx(bar, a.stage_tx);
  for (int e = lane; e < D2 + 4; e += 32) {
    if (e < D2) {
      bulk_load(st + a.off_sz + (size_t)e * M * sizeof(T), a.z_old + e * NM + src * M,
                (uint32_t)(M * sizeof(T)), bar);
    } else if (e == D2) {
      bulk_load(st + a.off_slq, a.lq_old + src * M, (uint32_t)(M * sizeof(T)), bar);
    } else if (e == D2 + 1) {
      bulk_load(st + a.off_sx, a.x_old + src * a.xp, (uint32_t)(a.xp * sizeof(T)), bar);
    } else if (!a.first) {
      if (e == D2 + 2)
        bulk_load(st + a.off_slwh, a.lwh_old + src * L, (uint32_t)(L * sizeof(T)), bar);
      else
        bulk_load(st + a.off_sxbb, a.xbb_old + src * L * D1, (uint32_t)(L * D1 * sizeof(T)), bar);
    }
  }
}

// Steps groups gfirst, gfirst + W, ... (< gend) of one filter with one warp:
// `mc` and `a` may live in kernel parameters or in global memory; `ws` is the
// warp's shared-memory region, `bar` its stage barrier, `phase` its parity.
// MF = 32 PPL when the launch has M = 32 PPL (every lane holds PPL particles: M is a
// compile-time constant and no lane is idle), else 0 (M from the arguments).
template <typename T, int D1, int D2, int DY, bool XZ, int PPL, int MF = 0>
__device__ __forceinline__ void warp_run(const MC<T, D1, D2, DY>& mc, const StepArgs<T>& a,
                                         long long gfirst, long long gend, long long W,
                                         unsigned char* ws, uint64_t* bar, uint32_t& phase) {
  static_assert(MF == 0 || MF == 32 * PPL, "MF is 0 or 32 PPL");
  const int lane = threadIdx.x & 31;
  const int M = MF ? MF : a.M, L = a.L;
  const long long N = a.N;
  const long long NM = N * (long long)M;
  T* sz = (T*)(ws + a.off_sz);
  T* slq = (T*)(ws + a.off_slq);
  T* sx = (T*)(ws + a.off_sx);
  T* slwh = (T*)(ws + a.off_slwh);
  T* sxbb = (T*)(ws + a.off_sxbb);
  uint32_t* cum = (uint32_t*)(ws + a.off_cum);
  T* fs = (T*)(ws + a.off_kd);
  T* xw = (T*)(ws + a.off_xw);
  T* cw = (T*)(ws + a.off_cw);
  T* xbs = (T*)(ws + a.off_xbs);
  T* rowS = (T*)(ws + a.off_row);
  T* rowA = rowS + L;
  T* shS = rowA + L;
  T* shA = shS + L;
  T* coef = shA + L;
  T* part = (T*)(ws + a.off_part);  // [2L][PART_STRIDE] lane partials
  // the rows [A_zx A_zz K] of the model, for the z-mean (lane r reads row r: shared memory
  // serves the lanes' different rows at once, where the constant bank would serialise them)
  constexpr int ZW = D1 + D2 + DY;
  T* zrow = (T*)(ws + a.off_zrow);
  for (int e = lane; e < D2 * ZW; e += 32) {
    const int r = e / ZW, c = e % ZW;
    zrow[e] = c < D1 ? mc.Azx[r][c] : (c < D1 + D2 ? mc.Azz[r][c - D1] : mc.K[r][c - D1 - D2]);
  }
  __syncwarp();
  const T NEG = neg_inf<T>();
  const T LOG2E = (T)LOG2E_D, SQ = (T)SQ_D, LN2 = (T)LN2_D;
  const RoundKeys rk = round_keys(a.key);
  // this lane's inner particles are k0 .. k0 + PPL - 1 (consecutive)
  const int k0 = PPL * lane;
  const bool act = MF ? true : k0 < M;
  if (gfirst == 0 && lane == 0) *a.Csum = 0ull;  // the outer reduction of this step sums into it

  long long g = gfirst;
  long long src_next = -1;  // the same in every lane
  if (a.glist) {
    const long long G = group_count(a);
    if (G < gend) gend = G;
  }
  if (g < gend) {
    const long long i0 = group_at(a, g);
    warp_stage<T, D1, D2>(a, ws, bar, a.first ? i0 : (long long)a.anc[i0], lane);
    if (g + W < gend) {
      const long long i1 = group_at(a, g + W);
      src_next = a.first ? i1 : (long long)a.anc[i1];
    }
  }
  __syncwarp();
  for (; g < gend; g += W, phase ^= 1u) {
    const long long i = group_at(a, g);
    {  // wait for this group's rows (bounded)
      int spins = 0;
      while (!mbar_test(bar, phase)) {
        if (++spins > MBAR_SPIN_LIMIT) {
          if (lane == 0) atomicOr(a.err, ERR_TIMEOUT);
          break;
        }
      }
    }
    if (a.gskip && a.gskip[i]) {  // a group left untouched: pass its stage on
      __syncwarp();
      if (g + W < gend) {
        warp_stage<T, D1, D2>(a, ws, bar, src_next, lane);
        const long long g2 = g + 2 * W;
        if (g2 < gend) {
          const long long i2 = group_at(a, g2);
          src_next = a.first ? i2 : (long long)a.anc[i2];
        }
      }
      continue;
    }
    T x[D1];
    T zr[D2][PPL];  // this lane's inner particles z_{t-1}^(i, k0 + p)
    T lqr[PPL];     // and their normalised log-weights
    T sigma, SA0;

    if (a.first) {
#pragma unroll
      for (int c = 0; c < D1; ++c) x[c] = sx[c];
#pragma unroll
      for (int p = 0; p < PPL; ++p) lqr[p] = NEG;
      // lanes past M hold zeros: their z enters the look-ahead's projections, whose
      // weights are then masked, and an undefined register there could be a NaN
#pragma unroll
      for (int c = 0; c < D2; ++c)
#pragma unroll
        for (int p = 0; p < PPL; ++p) zr[c][p] = T(0);
      if (act) {
#pragma unroll
        for (int c = 0; c < D2; ++c) vld<T, PPL>(sz + c * M + k0, zr[c]);
        vld<T, PPL>(slq + k0, lqr);
      }
      if (a.la_only) {  // the state's own weights: largest lq and sum exp(lq - largest)
        T mx = NEG;
#pragma unroll
        for (int p = 0; p < PPL; ++p) mx = fmax(mx, lqr[p]);
        sigma = warp_max(mx);
        T se = T(0);
#pragma unroll
        for (int p = 0; p < PPL; ++p) se += act ? exp2_t((lqr[p] - sigma) * LOG2E) : T(0);
        SA0 = warp_sum(se);
      } else {
        sigma = -a.logM;
        SA0 = (T)M;
      }
    } else {
      // ---- selection of x_{t-1}^(i) among the ancestor's look-ahead draws ----
      int msel;
      uint32_t uin;
      {
        // draws m = lane and (when L > 32, a warp-uniform branch) m = lane + 32
        const bool two = L > 32;
        const T l0 = lane < L ? slwh[lane] : NEG;
        const T l1 = two && lane + 32 < L ? slwh[lane + 32] : NEG;
        const T mx = warp_max(fmax(l0, l1));
        const uint32_t c0 = lane < L ? (uint32_t)floor(exp2_t((l0 - mx) * LOG2E) * a.scaleL) : 0u;
        uint32_t s0 = c0, s1 = 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t n0 = __shfl_up_sync(FULL, s0, o);
          if (lane >= o) s0 += n0;
        }
        if (two) {
          s1 = lane + 32 < L ? (uint32_t)floor(exp2_t((l1 - mx) * LOG2E) * a.scaleL) : 0u;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t n1 = __shfl_up_sync(FULL, s1, o);
            if (lane >= o) s1 += n1;
          }
        }
        const uint32_t tot0 = __shfl_sync(FULL, s0, 31), tot1 = two ? __shfl_sync(FULL, s1, 31) : 0u;
        const uint64_t C = (uint64_t)tot0 + tot1;
        const uint32_t w =
            philox_rk(ctr(a.t - 1, (uint32_t)i, lane == 0 ? P_SEL : P_INNER, 0u, 0u), rk).x;
        const uint32_t usel = __shfl_sync(FULL, w, 0);
        uin = __shfl_sync(FULL, w, 1);
        const uint64_t rhs = (uint64_t)usel * C;
        const unsigned b0 = __ballot_sync(FULL, ((uint64_t)s0 << 32) > rhs);
        const unsigned b1 = two ? __ballot_sync(FULL, ((uint64_t)(s1 + tot0) << 32) > rhs) : 0u;
        msel = b0 ? __ffs(b0) - 1 : (b1 ? 32 + __ffs(b1) - 1 : L - 1);
        if (C == 0 || msel >= L) {
          if (lane == 0) atomicOr(a.err, ERR_NUMERIC);
          msel = L - 1;
        }
        if (lane == 0) a.sel[i] = msel;
      }
      T xa[D1];
#pragma unroll
      for (int c = 0; c < D1; ++c) {
        x[c] = sxbb[msel * D1 + c];
        xa[c] = sx[c];
      }
      // ---- local resampling of the ancestor's inner set (eq. qnobar weights) ----
      T alpha[PPL];
#pragma unroll
      for (int p = 0; p < PPL; ++p) alpha[p] = NEG;
      if (act) {
        vld<T, PPL>(slq + k0, alpha);
        if (XZ) {
          T mxa[D1], wres[D1];
          mu_x(mc, xa, a.gcos_prev, mxa);
#pragma unroll
          for (int r = 0; r < D1; ++r) {
            T v = T(0);
#pragma unroll
            for (int c = 0; c < D1; ++c) if (c <= r) v += mc.LqxInv[r][c] * (x[c] - mxa[c]);
            wres[r] = v;
          }
          T res[D1][PPL];
#pragma unroll
          for (int r = 0; r < D1; ++r)
#pragma unroll
            for (int p = 0; p < PPL; ++p) res[r][p] = wres[r];
#pragma unroll
          for (int c = 0; c < D2; ++c) {
            T zc[PPL];
            vld<T, PPL>(sz + c * M + k0, zc);
#pragma unroll
            for (int r = 0; r < D1; ++r) axpy<T, PPL>(-mc.WAxz[r][c], zc, res[r]);
          }
#pragma unroll
          for (int r = 0; r < D1; ++r)
#pragma unroll
            for (int p = 0; p < PPL; ++p) alpha[p] -= T(0.5) * res[r][p] * res[r][p];
        }
      }
      T amax = NEG;
#pragma unroll
      for (int p = 0; p < PPL; ++p) amax = fmax(amax, alpha[p]);
      amax = warp_max(amax);
      // ancestors of the lane's destinations by offspring ranges (sys_local_offspring)
      int bidx[PPL];
      {
        uint32_t loc[PPL];
        uint32_t run = 0;
#pragma unroll
        for (int p = 0; p < PPL; ++p) {
          run += act ? (uint32_t)floor(exp2_t((alpha[p] - amax) * LOG2E) * a.scaleM) : 0u;
          loc[p] = run;
        }
        uint32_t v = run;  // inclusive warp scan of the lane totals
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t n = __shfl_up_sync(FULL, v, o);
          if (lane >= o) v += n;
        }
        const uint32_t base = v - run;
#pragma unroll
        for (int p = 0; p < PPL; ++p) loc[p] += base;
        const uint32_t C = __shfl_sync(FULL, v, 31);
        if (C == 0u && lane == 0) atomicOr(a.err, ERR_NUMERIC);
        sys_local_offspring<PPL>(loc, C, M, uin >> 16, k0, act, lane, (int*)cum, bidx);
      }
      // ---- propagation and the y_{t-1} update (eq. qbar) ----
      T azx[D2];
#pragma unroll
      for (int r = 0; r < D2; ++r) {
        T v = T(0);
#pragma unroll
        for (int c = 0; c < D1; ++c) v += mc.Azx[r][c] * xa[c];
        azx[r] = v;
      }
      T yh[DY];
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
      if (a.dbg_b && act) vst<int, PPL>(a.dbg_b + i * M + k0, bidx);
      // z_t = A_zz z_anc + (A_zx x + ...) + L_qz eps, column by column so that only
      // one column of the ancestors' z, or one block of four normals a particle,
      // is live beside the result; each row keeps its order of accumulation
#pragma unroll
      for (int r = 0; r < D2; ++r)
#pragma unroll
        for (int p = 0; p < PPL; ++p) zr[r][p] = azx[r];
#pragma unroll
      for (int c = 0; c < D2; ++c) {
        T zc[PPL];
#pragma unroll
        for (int p = 0; p < PPL; ++p) zc[p] = sz[c * M + bidx[p]];
#pragma unroll
        for (int r = 0; r < D2; ++r) axpy<T, PPL>(mc.Azz[r][c], zc, zr[r]);
      }
#pragma unroll
      for (int b = 0; b < (D2 + 3) / 4; ++b) {
        T e4[4][PPL];
#pragma unroll
        for (int p = 0; p < PPL; ++p) {
          T e[4];
          normal_block_rk(rk, a.t - 1, (uint32_t)i, P_PROP, (uint32_t)(k0 + p), b, D2 - 4 * b, e);
#pragma unroll
          for (int j = 0; j < 4; ++j) e4[j][p] = e[j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = 4 * b + j;
          if (c < D2) {
            if (mc.diag_qz) {
              axpy<T, PPL>(mc.Lqz[c][c], e4[j], zr[c]);
            } else {
              // constant bounds (not r = c ..) so that the loop unrolls before c is known
              // and zr stays in registers
#pragma unroll
              for (int r = 0; r < D2; ++r)
                if (r >= c) axpy<T, PPL>(mc.Lqz[r][c], e4[j], zr[r]);
            }
          }
        }
      }
      T ell[PPL];
#pragma unroll
      for (int p = 0; p < PPL; ++p) ell[p] = T(0);
#pragma unroll
      for (int q = 0; q < DY; ++q) {
        T rq[PPL];
#pragma unroll
        for (int p = 0; p < PPL; ++p) rq[p] = yh[q];
#pragma unroll
        for (int c = 0; c < D2; ++c) axpy<T, PPL>(-mc.LrHz[q][c], zr[c], rq);
#pragma unroll
        for (int p = 0; p < PPL; ++p) ell[p] = fma(rq[p], rq[p], ell[p]);
      }
      T lmax = NEG;
#pragma unroll
      for (int p = 0; p < PPL; ++p) {
        ell[p] = act ? T(-0.5) * ell[p] : NEG;
        lmax = fmax(lmax, ell[p]);
      }
      lmax = warp_max(lmax);
      T ls = T(0);
#pragma unroll
      for (int p = 0; p < PPL; ++p) ls += act ? exp2_t((ell[p] - lmax) * LOG2E) : T(0);
      const T lsum = warp_sum(ls);
      const T llsum = LN2 * log2_fast(lsum);
#pragma unroll
      for (int p = 0; p < PPL; ++p) lqr[p] = ell[p] - lmax - llsum;
      if (act) {
#pragma unroll
        for (int c = 0; c < D2; ++c) vst<T, PPL>(a.z_new + c * NM + i * M + k0, zr[c]);
        vst<T, PPL>(a.lq_new + i * M + k0, lqr);
      }
      {  // lane c < D1 stores x[c] (a select chain: a register array indexed by the lane
         // would be placed in local memory)
        T xo = x[0];
#pragma unroll
        for (int c = 1; c < D1; ++c)
          if (lane == c) xo = x[c];
        if (lane < D1) a.x_new[i * a.xp + lane] = xo;
      }
      sigma = -llsum;
      SA0 = lsum;
    }
    // the stage is consumed: prefetch the next group's rows into it
    __syncwarp();
    if (g + W < gend) {
      warp_stage<T, D1, D2>(a, ws, bar, src_next, lane);
      const long long g2 = g + 2 * W;
      if (g2 < gend) {
        const long long i2 = group_at(a, g2);
        src_next = a.first ? i2 : (long long)a.anc[i2];
      }
    }

    // ======== look-ahead of step t from (x, z, lq) with y_t ========
    T ak[PPL];      // (lq - sigma) log2(e)
    T ngk[DY][PPL]; // minus the scaled whitened projected draws
    T ep[DY][PPL];  // projected look-ahead noise
    T nfk[D1][PPL]; // minus the scaled whitened A_xz z (x transition depends on z)
#pragma unroll
    for (int p = 0; p < PPL; ++p) ak[p] = act ? (lqr[p] - sigma) * LOG2E : NEG;
    {
      T e2[DY][PPL];
      if constexpr (DY <= 2 && PPL % 2 == 0) {
        // the lane's particles k0 + p, k0 + p + 1 (k0 + p even) share one Philox block
        // (la_z_normals): its first word pair for the first, its second for the other
#pragma unroll
        for (int p = 0; p < PPL; p += 2) {
          const uint4 w = philox_rk(ctr(a.t, (uint32_t)i, P_LA_Z, (uint32_t)(k0 + p) >> 1, 0u), rk);
          T n0, n1, n2, n3;
          box_muller(w.x, w.y, n0, n1);
          box_muller(w.z, w.w, n2, n3);
          e2[0][p] = n0;
          e2[0][p + 1] = n2;
          if constexpr (DY > 1) {
            e2[1][p] = n1;
            e2[1][p + 1] = n3;
          }
        }
      } else if constexpr (DY <= 2) {
#pragma unroll
        for (int p = 0; p < PPL; ++p) {
          const uint32_t k = (uint32_t)(k0 + p);
          const uint4 w = philox_rk(ctr(a.t, (uint32_t)i, P_LA_Z, k >> 1, 0u), rk);
          T n0, n1;
          box_muller((k & 1u) ? w.z : w.x, (k & 1u) ? w.w : w.y, n0, n1);
          e2[0][p] = n0;
          if constexpr (DY > 1) e2[1][p] = n1;
        }
      } else {
#pragma unroll
        for (int p = 0; p < PPL; ++p) {
          T e[DY];
          normals_rk<DY>(rk, a.t, (uint32_t)i, P_LA_Z, (uint32_t)(k0 + p), e);
#pragma unroll
          for (int q = 0; q < DY; ++q) e2[q][p] = e[q];
        }
      }
      T gg[DY][PPL];
#pragma unroll
      for (int q = 0; q < DY; ++q) {
        T hx = T(0);
#pragma unroll
        for (int c = 0; c < D1; ++c) hx += mc.HzAzx[q][c] * x[c];
#pragma unroll
        for (int p = 0; p < PPL; ++p) ep[q][p] = T(0);
#pragma unroll
        for (int c = 0; c < DY; ++c) if (c <= q) axpy<T, PPL>(mc.Ls[q][c], e2[c], ep[q]);
#pragma unroll
        for (int p = 0; p < PPL; ++p) gg[q][p] = ep[q][p] + hx;
#pragma unroll
        for (int c = 0; c < D2; ++c) axpy<T, PPL>(mc.HzAzz[q][c], zr[c], gg[q]);
      }
#pragma unroll
      for (int q = 0; q < DY; ++q) {
#pragma unroll
        for (int p = 0; p < PPL; ++p) ngk[q][p] = T(0);
#pragma unroll
        for (int c = 0; c < DY; ++c) if (c <= q) axpy<T, PPL>(-SQ * mc.LrInv[q][c], gg[c], ngk[q]);
      }
      if (XZ) {
#pragma unroll
        for (int r = 0; r < D1; ++r) {
          T f[PPL];
#pragma unroll
          for (int p = 0; p < PPL; ++p) f[p] = T(0);
#pragma unroll
          for (int c = 0; c < D2; ++c) axpy<T, PPL>(mc.WAxz[r][c], zr[c], f);
          if (act) vst<T, PPL>(fs + r * M + k0, f);
#pragma unroll
          for (int p = 0; p < PPL; ++p) nfk[r][p] = -SQ * f[p];
        }
      }
    }
    if (XZ) {  // cumulative weights for the categorical draws of the mixture components
      uint32_t loc[PPL];
      uint32_t run = 0;
#pragma unroll
      for (int p = 0; p < PPL; ++p) {
        run += act ? (uint32_t)floor(exp2_t(ak[p]) * a.scaleM) : 0u;
        loc[p] = run;
      }
      uint32_t v = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t n = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += n;
      }
      const uint32_t base = v - run;
#pragma unroll
      for (int p = 0; p < PPL; ++p) loc[p] += base;
      if (act) vst<uint32_t, PPL>(cum + k0, loc);
    }
    __syncwarp();
    // ---- L look-ahead draws xbb^(m) (eq. approx1) ----
    {
      T mux[D1];
      mu_x(mc, x, a.gcos_cur, mux);
      for (int m = lane; m < L; m += 32) {
        T e1[D1], xwm[D1];
        normals_rk<D1>(rk, a.t, (uint32_t)i, P_LA_X, (uint32_t)m, e1);
        int jm = 0;
        if (XZ)
          jm = sys_local_pick(cum, M, cum[M - 1], 1, 0,
                              philox_rk(ctr(a.t, (uint32_t)i, P_LA_J, (uint32_t)m, 0u), rk).x);
#pragma unroll
        for (int c = 0; c < D1; ++c) xwm[c] = (XZ ? fs[c * M + jm] : T(0)) + e1[c];
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
    }
    __syncwarp();
    // ---- the L x M weights (eq. weightsMC with alpha of eq. qnobar), log2 units ----
    T B[PPL];  // beta_k up to normalisation
#pragma unroll
    for (int p = 0; p < PPL; ++p) B[p] = T(0);
    bool general = XZ;
    if (!XZ) {
      // one pass: e(m,k) = 2^(a_k - |c'_m - g'_k|^2), S_m = sum_k e, B_k = sum_m e
#pragma unroll 4
      for (int m = 0; m < L; ++m) {
        T v[PPL];
#pragma unroll
        for (int p = 0; p < PPL; ++p) v[p] = ak[p];
#pragma unroll
        for (int q = 0; q < DY; ++q) sub_sq<T, PPL>(cw[m * DY + q], ngk[q], v);
        T e[PPL];
#pragma unroll
        for (int p = 0; p < PPL; ++p) e[p] = exp2_t(v[p]);
        add_to<T, PPL>(e, B);
        part[m * PART_STRIDE + lane] = tree_sum<T, PPL>(e);
      }
      __syncwarp();
      // row sums of the 32 lane partials: for L <= 16 lanes m and m + 16 each add half of
      // row m (vector loads) and combine by one shuffle; else lane m adds all of row m
      if (L <= 16) {
        const int m = lane & 15, h = lane >> 4;
        T sum = T(0);
        if (m < L) {
          T r[16];
          vld<T, 16>(part + m * PART_STRIDE + 16 * h, r);
          sum = tree_sum<T, 16>(r);
        }
        sum += __shfl_xor_sync(FULL, sum, 16);
        if (h == 0 && m < L) {
          rowS[m] = sum;
          rowA[m] = SA0;
          shS[m] = T(0);
          shA[m] = T(0);
        }
      } else {
        for (int m = lane; m < L; m += 32) {
          T r[16];
          vld<T, 16>(part + m * PART_STRIDE, r);
          const T lo = tree_sum<T, 16>(r);
          vld<T, 16>(part + m * PART_STRIDE + 16, r);
          rowS[m] = lo + tree_sum<T, 16>(r);
          rowA[m] = SA0;
          shS[m] = T(0);
          shA[m] = T(0);
        }
      }
      __syncwarp();
      const T tiny = sizeof(T) == 4 ? T(1e-30) : T(1e-290);
      bool bad = false;
      for (int m = lane; m < L; m += 32) bad |= rowS[m] < tiny;
      general = __any_sync(FULL, bad);
    }
    T gmax = T(0);  // the largest row maximum (robust path without x-z coupling; else 0)
    if (general && !XZ) {
      // robust path of a model whose x transition does not depend on z (a row
      // underflowed): the alpha sums are then the same for every draw (SA0, whose largest
      // term is 2^0), so only the rows of e need their maxima. Pass 0 takes the row
      // maxima h_m; pass 1 the row sums relative to them and, since pi_m / S_m is then
      // proportional to 2^(h_m), beta_k up to normalisation as sum_m 2^(h_m - gmax) e'(m,k)
      // (the same weights as the fast path's sum_m e(m,k), relative to the largest row)
#pragma unroll
      for (int p = 0; p < PPL; ++p) B[p] = T(0);
      for (int pass = 0; pass < 2; ++pass) {
#pragma unroll 4
        for (int m = 0; m < L; ++m) {
          const T hs = pass ? shS[m] : T(0);
          const T wm = pass ? exp2_t(hs - gmax) : T(0);
          T vl[PPL];
#pragma unroll
          for (int p = 0; p < PPL; ++p) vl[p] = ak[p];
#pragma unroll
          for (int q = 0; q < DY; ++q) sub_sq<T, PPL>(cw[m * DY + q], ngk[q], vl);
          T ps = pass ? T(0) : NEG;
          if (act) {
#pragma unroll
            for (int p = 0; p < PPL; ++p) {
              if (pass) {
                const T e = exp2_t(vl[p] - hs);
                ps += e;
                B[p] = fma(wm, e, B[p]);
              } else {
                ps = fmax(ps, vl[p]);
              }
            }
          }
          part[m * PART_STRIDE + lane] = ps;
        }
        __syncwarp();
        if (pass == 0) {
          reduce_rows<T, true>(part, L, lane, shS);
          __syncwarp();
          T g = NEG;
          for (int m = lane; m < L; m += 32) g = fmax(g, shS[m]);
          gmax = warp_max(g);
        } else {
          reduce_rows<T, false>(part, L, lane, rowS);
          for (int m = lane; m < L; m += 32) {
            rowA[m] = SA0;
            shA[m] = T(0);
          }
        }
        __syncwarp();
      }
    } else if (general) {
      // robust path (x transition depends on z): row maxima, row sums relative to them,
      // then beta with the coefficients pi_m / S_m
      for (int pass = 0; pass < 2; ++pass) {
        for (int m = 0; m < L; ++m) {
          const T ha = pass ? shA[m] : T(0), hs = pass ? shS[m] : T(0);
          T v[PPL];
#pragma unroll
          for (int p = 0; p < PPL; ++p) v[p] = ak[p];
          if (XZ) {
#pragma unroll
            for (int c = 0; c < D1; ++c) sub_sq<T, PPL>(xw[m * D1 + c], nfk[c], v);
          }
          T vl[PPL];
#pragma unroll
          for (int p = 0; p < PPL; ++p) vl[p] = v[p];
#pragma unroll
          for (int q = 0; q < DY; ++q) sub_sq<T, PPL>(cw[m * DY + q], ngk[q], vl);
          T pa = pass ? T(0) : NEG, ps = pass ? T(0) : NEG;
          if (act) {
#pragma unroll
            for (int p = 0; p < PPL; ++p) {
              if (pass == 0) {
                pa = fmax(pa, v[p]);
                ps = fmax(ps, vl[p]);
              } else {
                pa += exp2_t(v[p] - ha);
                ps += exp2_t(vl[p] - hs);
              }
            }
          }
          part[m * PART_STRIDE + lane] = pa;
          part[(L + m) * PART_STRIDE + lane] = ps;
        }
        __syncwarp();
        for (int m = lane; m < L; m += 32) {
          T ra = pass ? T(0) : NEG, rs = pass ? T(0) : NEG;
          for (int l = 0; l < 32; ++l) {
            if (pass == 0) {
              ra = fmax(ra, part[m * PART_STRIDE + l]);
              rs = fmax(rs, part[(L + m) * PART_STRIDE + l]);
            } else {
              ra += part[m * PART_STRIDE + l];
              rs += part[(L + m) * PART_STRIDE + l];
            }
          }
          if (pass == 0) {
            shA[m] = ra;
            shS[m] = rs;
          } else {
            rowA[m] = ra;
            rowS[m] = rs;
          }
        }
        __syncwarp();
      }
    }
    // ---- per-draw weights, the outer weight and the x part of the filtered mean ----
    // draws m = lane and (L > 32, a warp-uniform branch) m = lane + 32
    const bool two = L > 32;
    T lw0 = NEG, lw1 = NEG;
    if (lane < L) {
      lw0 = mc.lognorm_y + LN2 * ((log2_fast(rowS[lane]) + shS[lane]) - (log2_fast(rowA[lane]) + shA[lane]));
      a.lwh_new[i * L + lane] = lw0;
    }
    if (two && lane + 32 < L) {
      lw1 = mc.lognorm_y + LN2 * ((log2_fast(rowS[lane + 32]) + shS[lane + 32]) -
                                  (log2_fast(rowA[lane + 32]) + shA[lane + 32]));
      a.lwh_new[i * L + lane + 32] = lw1;
    }
    const T mx = warp_max(two ? fmax(lw0, lw1) : lw0);
    const T p0 = lane < L ? exp2_t((lw0 - mx) * LOG2E) : T(0);
    const T p1 = two && lane + 32 < L ? exp2_t((lw1 - mx) * LOG2E) : T(0);
    const T psum = warp_sum(p0 + p1);
    const T lwi = mx + LN2 * log2_fast(psum) - a.logL;
    const T ipsum = T(1) / psum;
#pragma unroll
    for (int c = 0; c < D1; ++c) {
      T v = lane < L ? p0 * xbs[lane * D1 + c] : T(0);
      if (two && lane + 32 < L) v += p1 * xbs[(lane + 32) * D1 + c];
      v = warp_sum(v) * ipsum;
      if (lane == 0) a.xm[(long long)c * N + i] = v;
    }
    if (lane == 0) {
      a.lw[i] = lwi;
      if (lwi != lwi) atomicOr(a.err, ERR_NUMERIC);
      const unsigned long long key = order_key(lwi);
      if (lwi == lwi && key > *(volatile unsigned long long*)a.lwmax_key)
        atomicMax(a.lwmax_key, key);
    }
    // ---- z part of the filtered mean: beta_k = sum_m pi_m e(m,k) / S_m ----
    if (general && XZ) {
#pragma unroll
      for (int p = 0; p < PPL; ++p) B[p] = T(0);
      if (lane < L) coef[lane] = p0 / psum / rowS[lane];
      if (lane + 32 < L) coef[lane + 32] = p1 / psum / rowS[lane + 32];
      __syncwarp();
      for (int m = 0; m < L; ++m) {
        const T cf = coef[m], hs = shS[m];
        T v[PPL];
#pragma unroll
        for (int p = 0; p < PPL; ++p) v[p] = ak[p];
        if (XZ) {
#pragma unroll
          for (int c = 0; c < D1; ++c) sub_sq<T, PPL>(xw[m * D1 + c], nfk[c], v);
        }
#pragma unroll
        for (int q = 0; q < DY; ++q) sub_sq<T, PPL>(cw[m * DY + q], ngk[q], v);
#pragma unroll
        for (int p = 0; p < PPL; ++p) B[p] += act ? cf * exp2_t(v[p] - hs) : T(0);
      }
    } else {
      // normalise sum_m e(m,k) by sum_(m,k) e(m,k), both relative to the largest row
      // (gmax = 0 and every shS = 0 on the fast path)
      T tot = T(0);
      for (int m = lane; m < L; m += 32) tot += general ? rowS[m] * exp2_t(shS[m] - gmax) : rowS[m];
      tot = warp_sum(tot);
      const T inv = T(1) / tot;
#pragma unroll
      for (int p = 0; p < PPL; ++p) B[p] *= inv;
    }
    T acc[D2 + DY];
#pragma unroll
    for (int c = 0; c < D2; ++c) {
      T v = T(0);
#pragma unroll
      for (int p = 0; p < PPL; ++p) v = fma(B[p], zr[c][p], v);
      acc[c] = act ? v : T(0);
    }
#pragma unroll
    for (int q = 0; q < DY; ++q) {
      T v = T(0);
#pragma unroll
      for (int p = 0; p < PPL; ++p) v = fma(B[p], ep[q][p], v);
      acc[D2 + q] = act ? v : T(0);
    }
#pragma unroll
    for (int c = 0; c < D2 + DY; ++c) acc[c] = warp_sum(acc[c]);
    if (lane < D2) {
      const int r = lane;
      const T* row = zrow + r * ZW;
      T v = T(0);
#pragma unroll
      for (int c = 0; c < D1; ++c) v += row[c] * x[c];
#pragma unroll
      for (int c = 0; c < D2; ++c) v += row[D1 + c] * acc[c];
#pragma unroll
      for (int q = 0; q < DY; ++q) v += row[D1 + D2 + q] * acc[D2 + q];
      a.zm[(long long)r * N + i] = v;
    }
    __syncwarp();
  }
}


template <typename T, int D1, int D2, int DY, bool XZ, int PPL, int MF>
__global__ void __launch_bounds__(WARPS_PER_CTA * 32, warp_min_blocks<PPL, D2>())
    step_warp_kernel(const __grid_constant__ MC<T, D1, D2, DY> mc,
                     const __grid_constant__ StepArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[WARPS_PER_CTA];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (lane == 0) {
    mbar_init(&bars[wib], 1);
    mbar_fence_init();
  }
  __syncwarp();
  uint32_t phase = 0;
  warp_run<T, D1, D2, DY, XZ, PPL, MF>(mc, a, (long long)blockIdx.x * WARPS_PER_CTA + wib, a.N,
                                   (long long)gridDim.x * WARPS_PER_CTA,
                                   smem_raw + (size_t)wib * a.stage_bytes, &bars[wib], phase);
}

// Many filters of one (precision, d1, d2, dy, PPL) class in one persistent
// launch: the class's groups are numbered filter after filter (fstart[f] is the
// first item of filter f) and each warp steps a contiguous chunk of them.
// With SHARED every filter of the launch has the same model constants, passed
// by value (read through the constant cache); otherwise they come from mcs[f].
template <typename T, int D1, int D2, int DY, bool XZ, int PPL, bool SHARED, int MF>
__global__ void __launch_bounds__(WARPS_PER_CTA * 32, warp_min_blocks<PPL, D2>())
    step_warp_batch_kernel(const __grid_constant__ MC<T, D1, D2, DY> mc1,
                           const MC<T, D1, D2, DY>* __restrict__ mcs,
                           const StepArgs<T>* __restrict__ descs, const long long* __restrict__ fstart,
                           int F, long long chunk, uint32_t region) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[WARPS_PER_CTA];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (lane == 0) {
    mbar_init(&bars[wib], 1);
    mbar_fence_init();
  }
  __syncwarp();
  const long long total = fstart[F];
  uint32_t phase = 0;
  unsigned char* ws = smem_raw + (size_t)wib * region;
  // The CTA takes WARPS_PER_CTA chunks in a row and walks them filter by filter. Each
  // filter's launch arguments (and its model constants, unless the launch shares one
  // set as a parameter) are staged once in shared memory after the warps' regions, so
  // the step reads them from there instead of holding global-memory copies in
  // registers; the filter's groups are dealt to the four warps in turn.
  using Const = MC<T, D1, D2, DY>;
  constexpr size_t kArgs = (sizeof(StepArgs<T>) + 15) / 16 * 16;
  StepArgs<T>* sa = reinterpret_cast<StepArgs<T>*>(smem_raw + (size_t)WARPS_PER_CTA * region);
  Const* smc = reinterpret_cast<Const*>(smem_raw + (size_t)WARPS_PER_CTA * region + kArgs);
  long long item = (long long)blockIdx.x * WARPS_PER_CTA * chunk;
  const long long cend = item + WARPS_PER_CTA * chunk;
  const long long iend = cend < total ? cend : total;
  int lo = 0, hi = F;  // the filter holding `item`: last f with fstart[f] <= item
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (fstart[mid] <= item) lo = mid; else hi = mid;
  }
  int f = lo;
  while (item < iend) {
    while (fstart[f + 1] <= item) ++f;
    const long long seg_end = iend < fstart[f + 1] ? iend : fstart[f + 1];
    __syncthreads();  // the previous filter's arguments and constants are no longer read
    {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(descs + f);
      uint32_t* dst = reinterpret_cast<uint32_t*>(sa);
      for (int e = threadIdx.x; e < (int)(sizeof(StepArgs<T>) / 4); e += WARPS_PER_CTA * 32) dst[e] = src[e];
    }
    if (!SHARED) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(mcs + f);
      uint32_t* dst = reinterpret_cast<uint32_t*>(smc);
      for (int e = threadIdx.x; e < (int)(sizeof(Const) / 4); e += WARPS_PER_CTA * 32) dst[e] = src[e];
    }
    __syncthreads();
    warp_run<T, D1, D2, DY, XZ, PPL, MF>(SHARED ? mc1 : *smc, *sa, item - fstart[f] + wib,
                                         seg_end - fstart[f], WARPS_PER_CTA, ws, &bars[wib], phase);
    item = seg_end;
  }
}

}  // namespace dpf
