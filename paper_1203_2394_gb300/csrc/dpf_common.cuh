// Device building blocks of the GB300 LA-DPF: counter-based random numbers,
// warp/block reductions and scans, and the exact integer systematic-resampling
// rules. Everything here is __device__ code for sm_103a.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dpf.h"

namespace dpf {

constexpr unsigned FULL = 0xffffffffu;

// Purposes of random draws: the counter's third word carries purpose << 24.
enum Purpose : uint32_t {
  P_INIT_X = 1, P_INIT_Z = 2, P_LA_J = 3, P_LA_X = 4, P_LA_Z = 5,
  P_OUTER = 6, P_SEL = 7, P_INNER = 8, P_PROP = 9,
  P_LCOMP = 10,  // mixture-component draw of the learned inner proposal
  P_PF_X = 12, P_PF_Z = 13  // the bootstrap particle filter's x and z transition noise
};

// Device error word bits (latched with atomicOr, read by the host after a sync).
enum ErrBit : int { ERR_NUMERIC = 1, ERR_TIMEOUT = 2, ERR_BOUNDS = 4 };

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products whose high halves are xor-ed with the other counter
// words and the round key; the key advances by the Weyl constants each round.
// ---------------------------------------------------------------------------
struct Key {
  uint32_t k0, k1;
};

__device__ __forceinline__ uint4 philox(uint4 c, Key key) {
  uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Counter of draw (t, i, purpose, sub, block).
__device__ __forceinline__ uint4 ctr(uint32_t t, uint32_t i, uint32_t purpose, uint32_t sub,
                                     uint32_t block) {
  return make_uint4(t, i, (purpose << 24) | (sub & 0xFFFFFFu), block);
}

__device__ __forceinline__ uint32_t rand_word(Key k, uint32_t t, uint32_t i, uint32_t purpose,
                                              uint32_t sub) {
  return philox(ctr(t, i, purpose, sub, 0), k).x;
}

// Uniform on (0,1): ((w >> 9) + 1/2) 2^-23, exact in binary32 and binary64.
__device__ __forceinline__ float u01(uint32_t w, float) {
  return fmaf((float)(w >> 9), 0x1p-23f, 0x1p-24f);
}
__device__ __forceinline__ double u01(uint32_t w, double) {
  return fma((double)(w >> 9), 0x1p-23, 0x1p-24);
}

// Hardware approximations (PTX .approx instructions) used by the FP32 path.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sin_approx(float x) {
  float y;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cos_approx(float x) {
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Box-Muller: two words -> two independent standard normals,
//   n0 = r cos(2 pi u_b), n1 = r sin(2 pi u_b),  r = sqrt(-2 ln u_a).
// FP32: the radius uses the hardware log2 except for u_a > 1 - 2^-10 (the top
// 2^13 of the 2^23 values), where the hardware log2's absolute error would be
// large relative to the small radius; there -ln u_a = -ln(1 - v) with v = 1 - u_a
// (exact) is summed as its Taylor series v + v^2/2 + v^3/3 + v^4/4 (truncation
// below 2^-41 relative). Below that band the hardware path's radius is within
// 1.2e-6 of the exact one. The branch is taken by a warp of 32 independent draws
// about 3% of the time. The angle uses the identity cos(2 pi u) = -cos(2 pi (u - 1/2))
// (and likewise sin) so the hardware sine and cosine see arguments in (-pi, pi).
// The accuracy is verified exhaustively over all 2^23 values of each uniform.
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float& n0, float& n1) {
  const uint32_t ka = wa >> 9;
  float r2;
  if (__builtin_expect(ka >= (1u << 23) - (1u << 13), 0)) {
    const float v = fmaf((float)((1u << 23) - 1u - ka), 0x1p-23f, 0x1p-24f);
    float s = fmaf(v, 0.25f, 0.333333333f);
    s = fmaf(v, s, 0.5f);
    s = fmaf(v, s, 1.0f);
    r2 = 2.0f * v * s;
  } else {
    // u_a = (ka + 1/2) 2^-23 = (1 + ka 2^-23) - (1 - 2^-24): the first term is ka placed in
    // the mantissa of 1.0, and the difference is exact (Sterbenz); no integer conversion
    const float ua = __int_as_float(0x3F800000u | ka) - 0x1.fffffep-1f;
    r2 = -1.38629436f * lg2_approx(ua);  // -2 ln 2 log2 u
  }
  const float r = sqrt_approx(r2);
  // the angle 2 pi (u_b - 1/2) with u_b - 1/2 = ((1 + kb 2^-23) - 3/2) + 2^-24: the
  // difference is exact, and the fused multiply-add rounds 2 pi times the exact sum once
  // (2 pi 2^-24 is the single-precision 2 pi scaled by a power of two, also exact)
  const float th = fmaf(__int_as_float(0x3F800000u | (wb >> 9)) - 1.5f, 6.28318531f,
                        0x1p-24f * 6.28318531f);
  n0 = -r * cos_approx(th);
  n1 = -r * sin_approx(th);
}
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, double& n0, double& n1) {
  const double ua = u01(wa, 0.0), ub = u01(wb, 0.0);
  const double r = sqrt(-2.0 * log(ua));
  double s, c;
  sincospi(2.0 * ub, &s, &c);
  n0 = r * c;
  n1 = r * s;
}

// N standard normals of draw (t, i, purpose, sub): pair p uses words
// 2(p mod 2), 2(p mod 2)+1 of block p/2.
template <int N, typename T>
__device__ __forceinline__ void normals(Key k, uint32_t t, uint32_t i, uint32_t purpose,
                                        uint32_t sub, T (&out)[N]) {
#pragma unroll
  for (int b = 0; b < (N + 3) / 4; ++b) {
    const uint4 w = philox(ctr(t, i, purpose, sub, (uint32_t)b), k);
    T a0, a1, a2, a3;
    box_muller(w.x, w.y, a0, a1);
    if (4 * b + 0 < N) out[4 * b + 0] = a0;
    if (4 * b + 1 < N) out[4 * b + 1] = a1;
    if (4 * b + 2 < N) {
      box_muller(w.z, w.w, a2, a3);
      out[4 * b + 2] = a2;
      if (4 * b + 3 < N) out[4 * b + 3] = a3;
    }
  }
}

// Philox4x32-10 with the round keys precomputed (they are kernel-uniform).
struct RoundKeys {
  uint32_t k0[10], k1[10];
};
__device__ __forceinline__ RoundKeys round_keys(Key key) {
  RoundKeys r;
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    r.k0[q] = key.k0 + (uint32_t)q * 0x9E3779B9u;
    r.k1[q] = key.k1 + (uint32_t)q * 0xBB67AE85u;
  }
  return r;
}
__device__ __forceinline__ uint4 philox_rk(uint4 c, const RoundKeys& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk.k0[r], (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ rk.k1[r], (uint32_t)p0);
  }
  return c;
}
// Normals 4b .. 4b+n-1 (n <= 4) of the draw (t, i, purpose, sub): one Philox
// block, Box-Muller on its first pair and, when needed, its second.
template <typename T>
__device__ __forceinline__ void normal_block_rk(const RoundKeys& rk, uint32_t t, uint32_t i,
                                                uint32_t purpose, uint32_t sub, int b, int n, T (&out)[4]) {
  const uint4 w = philox_rk(ctr(t, i, purpose, sub, (uint32_t)b), rk);
  box_muller(w.x, w.y, out[0], out[1]);
  if (n > 2) box_muller(w.z, w.w, out[2], out[3]);
}
template <int N, typename T>
__device__ __forceinline__ void normals_rk(const RoundKeys& rk, uint32_t t, uint32_t i,
                                           uint32_t purpose, uint32_t sub, T (&out)[N]) {
#pragma unroll
  for (int b = 0; b < (N + 3) / 4; ++b) {
    T e[4];
    normal_block_rk(rk, t, i, purpose, sub, b, N - 4 * b, e);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (4 * b + j < N) out[4 * b + j] = e[j];
  }
}

// The dy normals of the look-ahead's common inner draw of inner particle k (purpose
// LA_Z). For dy <= 2 two inner particles share one Philox block: particle k takes the
// Box-Muller pair of words 2(k mod 2), 2(k mod 2)+1 of block (t, i, LA_Z, k / 2); for
// dy > 2 they are the normals of draw (t, i, LA_Z, k).
template <int DY, typename T>
__device__ __forceinline__ void la_z_normals(Key key, uint32_t t, uint32_t i, uint32_t k, T (&out)[DY]) {
  if constexpr (DY <= 2) {
    const uint4 w = philox(ctr(t, i, P_LA_Z, k >> 1, 0u), key);
    T a0, a1;
    box_muller((k & 1u) ? w.z : w.x, (k & 1u) ? w.w : w.y, a0, a1);
    out[0] = a0;
    if constexpr (DY > 1) out[1] = a1;
  } else {
    normals<DY>(key, t, i, P_LA_Z, k, out);
  }
}

// ---------------------------------------------------------------------------
// Reductions and scans.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T neg_inf();
template <>
__device__ __forceinline__ float neg_inf<float>() { return -__int_as_float(0x7f800000); }
template <>
__device__ __forceinline__ double neg_inf<double>() {
  return -__longlong_as_double(0x7ff0000000000000ll);
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Block-wide max / sum over NT threads. `red` holds >= NT/32 elements of
// shared memory; the result is returned to every thread.
template <int NT, typename T>
__device__ __forceinline__ T block_max(T v, T* red) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  T r = red[0];
#pragma unroll
  for (int q = 1; q < NT / 32; ++q) r = fmax(r, red[q]);
  return r;
}
template <int NT, typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  T r = red[0];
#pragma unroll
  for (int q = 1; q < NT / 32; ++q) r += red[q];
  return r;
}

// Inclusive block scan of one uint32 per thread; `red` holds >= NT/32 words.
template <int NT>
__device__ __forceinline__ uint32_t block_incl_scan_u32(uint32_t v, uint32_t* red) {
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
#pragma unroll
  for (int q = 0; q < NT / 32; ++q)
    if (q < w) add += red[q];
  return v + add;
}

// ---------------------------------------------------------------------------
// Exact systematic resampling, local rule (segments of n <= 1024 weights):
//   S = 31 - ceil(log2 n), c_i = floor(W_i 2^(S-e)), C = sum c_i < 2^32,
//   out[k] = min{ i : cum_i * n_out * 2^b > (k 2^b + u_b) C },
// with b = 16, u_b = u >> 16 for n_out > 1 and b = 32, u_b = u for one draw.
// ---------------------------------------------------------------------------
// Segment of item b under the prefix table start[0..F] (start[0] = 0, start[F] =
// total): the largest f with start[f] <= b, which skips empty segments.
__device__ __forceinline__ int find_segment(const int* __restrict__ start, int F, int b) {
  int lo = 0, hi = F - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__host__ __device__ __forceinline__ int ceil_log2_i(long long n) {
  int b = 0;
  while ((1ll << b) < n) ++b;
  return b;
}

// c = floor(W 2^shift): an exact power-of-two scaling, then a floor.
__device__ __forceinline__ uint32_t quantize_u32(float W, int shift) {
  return (uint32_t)floorf(ldexpf(W, shift));
}
__device__ __forceinline__ uint32_t quantize_u32(double W, int shift) {
  return (uint32_t)floor(ldexp(W, shift));
}

// min i in [0, n) with cum[i] * scale > rhs; cum is non-decreasing and
// cum[n-1] * scale > rhs is guaranteed by the callers.
__device__ __forceinline__ int search_cum(const uint32_t* cum, int n, uint64_t scale,
                                          uint64_t rhs) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((uint64_t)cum[mid] * scale > rhs)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

// k-th output of the local rule with n_out outputs.
__device__ __forceinline__ int sys_local_pick(const uint32_t* cum, int n, uint32_t C, int n_out,
                                              int k, uint32_t u) {
  if (n_out == 1) return search_cum(cum, n, 1ull << 32, (uint64_t)u * C);
  const uint64_t rhs = (((uint64_t)k << 16) + (u >> 16)) * (uint64_t)C;
  return search_cum(cum, n, (uint64_t)n_out << 16, rhs);
}

// ---- shared-memory addresses, mbarriers and bulk copies ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(b))
      : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}


}  // namespace dpf
