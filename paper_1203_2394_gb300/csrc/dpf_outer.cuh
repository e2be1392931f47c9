// The outer stage of one step: the evidence increment, the ESS and the filtered
// mean (eq. weightsopt), and the global systematic resampling of the N outer
// particles (Fig. 4 step 3).
//
// A single filter runs it in one cooperative launch (every CTA resident at
// once) with one grid-wide barrier:
//   A. each CTA sums W_i = exp(lw_i - max lw), W_i^2, W_i times the particle's
//      x and z means, and the quantised counts c_i = floor(W_i 2^S), over its
//      contiguous range of items;
//   B. the CTAs publish their count totals and wait for one another (a bounded
//      wait); each then reads the totals of the CTAs before it (its exclusive
//      prefix) and of all of them (the quantised total C);
//   C. each CTA scans its items' counts chunk by chunk, turns each cumulative
//      count into the number of systematic points below it, and writes the
//      ancestor of every point that falls in the chunk;
//   D. one CTA combines the partial sums into the statistics (an extra CTA with no
//      items where the grid has room for it, so that this serial double-precision
//      work overlaps the others' scatter), and the last CTA to finish resets the
//      counters for the next step.
// Many filters run the same phases in two ordinary launches (A, then B-D), the
// launch boundary standing in for the barrier, with each filter's partition
// unchanged, so their results are bit-identical to the single launch's.
// The integer rule is the one dpf_resample's global scan applies (S = 62 -
// ceil(log2 N); output k takes the first item with cum * N 2^32 > (k 2^32 + u) C),
// so the ancestors are the ones it would return for the same weights and word.
#pragma once

#include <cuda/atomic>

#include "dpf_common.cuh"
#include "dpf_internal.h"
#include "dpf_resample.cuh"
#include "dpf_step.cuh"

namespace dpf {

template <typename T>
struct FusedOuterArgs {
  OuterArgs<T> o;               // weights, means, statistics, counters
  T* w_out;                     // the W_i fed to the rule (may be null)
  int32_t* anc;                 // the N ancestors
  unsigned long long* ctot;     // one count total a CTA
  unsigned int* arrive;         // barrier arrivals, reset by the last CTA (null: no barrier)
  int nwork;                    // CTAs that own items; one more, if launched, only computes statistics
  int shift;                    // S = 62 - ceil(log2 N)
  double logN;                  // log N
  Key key;                      // u = rand_word(key, t, 0, P_OUTER, 0)
  uint32_t t;
  int withhold;                 // a CTA that never arrives (a check of the bounded wait); -1: none
  double* host_stats;           // a pinned host mirror of stats[0 .. 4 + d) and the error word, or null
};

template <typename T>
__device__ __forceinline__ T pow2_t(int e);
template <>
__device__ __forceinline__ float pow2_t<float>(int e) { return __int_as_float((127 + e) << 23); }
template <>
__device__ __forceinline__ double pow2_t<double>(int e) {
  return __longlong_as_double((long long)(1023 + e) << 52);
}

// K(c) = #{ k in [0, n) : (k 2^32 + u) C < c n 2^32 }, the number of systematic
// points below the cumulative count c (the quantity points_below computes). The
// condition falls as k grows, so K is the first k where it fails: an estimate
// c n / C - u 2^-32 (single precision up to n = 2^24, whose error is a few units;
// double beyond) is settled by exact 128-bit comparisons.
__device__ __forceinline__ int points_below_est(unsigned long long c, long long n, uint32_t u,
                                                unsigned long long C) {
  if (c == 0) return 0;
  const u128 X = ((u128)c * (u128)(unsigned long long)n) << 32;
  long long k;
  if (n <= (1ll << 24)) {
    const float e = __fdividef((float)c, (float)C) * (float)n - (float)u * 0x1p-32f;
    k = e > 0.f ? (long long)ceilf(e) : 0;
  } else {
    const double e = (double)c / (double)C * (double)n - (double)u * 0x1p-32;
    k = e > 0.0 ? (long long)ceil(e) : 0;
  }
  if (k > n) k = n;
  while (k > 0 && !((u128)((unsigned long long)(k - 1) << 32 | u) * C < X)) --k;
  while (k < n && (u128)((unsigned long long)k << 32 | u) * C < X) ++k;
  return (int)k;
}

// ---- A: the partial sums and the count total of CTA `bid` of the `nb` CTAs of one filter ----
template <typename T, int D1, int D2>
__device__ __forceinline__ void outer_sums(const FusedOuterArgs<T>& a, int bid, int nb, T lwmax) {
  constexpr int NV = 2 + D1 + D2, NW = OF_NT / 32;
  __shared__ T sv[NV][NW];
  __shared__ unsigned long long su[NW];
  const OuterArgs<T>& o = a.o;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long N = o.N;
  const T sS = pow2_t<T>(a.shift);
  const long long nch = (N + OF_CHUNK - 1) / OF_CHUNK;
  const long long i0 = nch * bid / nb * OF_CHUNK, i1 = nch * (bid + 1) / nb * OF_CHUNK;
  const long long iend = i1 < N ? i1 : N;
  T v[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = T(0);
  unsigned long long cc = 0;
  for (long long i = i0 + tid; i < iend; i += OF_NT) {
    const T W = exp_t<T>(o.lw[i] - lwmax);
    cc += (unsigned long long)floor(W * sS);  // exact: a power-of-two scaling, then a floor
    v[0] += W;
    v[1] += W * W;
#pragma unroll
    for (int c = 0; c < D1; ++c) v[2 + c] += W * o.xm[(long long)c * N + i];
#pragma unroll
    for (int c = 0; c < D2; ++c) v[2 + D1 + c] += W * o.zm[(long long)c * N + i];
  }
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
  cc = warp_sum(cc);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sv[q][w] = v[q];
    su[w] = cc;
  }
  __syncthreads();
  if (tid == 0) {  // one thread publishes the CTA's row (so that one fence covers it)
    for (int q = 0; q < NV; ++q) {
      T s = T(0);
#pragma unroll
      for (int r = 0; r < NW; ++r) s += sv[q][r];
      o.partials[(long long)bid * NV + q] = (double)s;
    }
    unsigned long long s = 0;
#pragma unroll
    for (int r = 0; r < NW; ++r) s += su[r];
    a.ctot[bid] = s;
  }
}

// ---- B: the exclusive prefix of CTA `bid`'s count total and the total C, once every
// CTA's total is in place (block-wide: every thread receives both) ----
__device__ __forceinline__ void count_prefix(const unsigned long long* ctot, int bid, int nb,
                                             unsigned long long& pre, unsigned long long& C) {
  constexpr int NW = OF_NT / 32;
  __shared__ unsigned long long su[2][NW];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  unsigned long long p = 0, t = 0;
  for (int b = tid; b < nb; b += OF_NT) {
    const unsigned long long c = __ldcg(ctot + b);
    t += c;
    if (b < bid) p += c;
  }
  p = warp_sum(p);
  t = warp_sum(t);
  __syncthreads();
  if (lane == 0) {
    su[0][w] = p;
    su[1][w] = t;
  }
  __syncthreads();
  pre = 0;
  C = 0;
#pragma unroll
  for (int r = 0; r < NW; ++r) {
    pre += su[0][r];
    C += su[1][r];
  }
}

// ---- C: the chunks' cumulative counts, the points below them, the ancestors (C > 0) ----
template <typename T>
__device__ __forceinline__ void outer_scatter(const FusedOuterArgs<T>& a, int bid, int nb, T lwmax,
                                              unsigned long long pre, unsigned long long C) {
  constexpr int NW = OF_NT / 32;
  __shared__ unsigned long long su[NW];
  __shared__ int ks[OF_CHUNK + 1];
  const OuterArgs<T>& o = a.o;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long N = o.N;
  const T sS = pow2_t<T>(a.shift);
  const long long nch = (N + OF_CHUNK - 1) / OF_CHUNK;
  const long long ch0 = nch * bid / nb, ch1 = nch * (bid + 1) / nb;
  const uint32_t u = rand_word(a.key, a.t, 0, P_OUTER, 0);
  unsigned long long run = pre;
  for (long long ch = ch0; ch < ch1; ++ch) {
    const long long base = ch * OF_CHUNK;
    unsigned long long c[OF_IPT], ts = 0;
#pragma unroll
    for (int q = 0; q < OF_IPT; ++q) {
      const long long i = base + tid * OF_IPT + q;
      unsigned long long ci = 0;
      if (i < N) {
        const T W = exp_t<T>(o.lw[i] - lwmax);
        if (a.w_out) a.w_out[i] = W;
        ci = (unsigned long long)floor(W * sS);
      }
      c[q] = ci;
      ts += ci;
    }
    // exclusive block scan of the per-thread sums
    unsigned long long incl = ts;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
      const unsigned long long n = __shfl_up_sync(FULL, incl, s);
      if (lane >= s) incl += n;
    }
    if (lane == 31) su[w] = incl;
    __syncthreads();
    unsigned long long wpre = 0, agg = 0;
#pragma unroll
    for (int r = 0; r < NW; ++r) {
      if (r < w) wpre += su[r];
      agg += su[r];
    }
    unsigned long long cum = run + wpre + incl - ts;
    if (tid == 0) ks[0] = points_below_est(run, N, u, C);
#pragma unroll
    for (int q = 0; q < OF_IPT; ++q) {
      cum += c[q];
      ks[tid * OF_IPT + q + 1] = points_below_est(cum, N, u, C);
    }
    __syncthreads();
    // output k lies in item j's range ks[j] <= k < ks[j + 1] (an empty range is never
    // hit, so j is never an item past N, whose count is zero)
    const int khi = ks[OF_CHUNK];
    for (int k = ks[0] + tid; k < khi; k += OF_NT) {
      int lo = 0, hi = OF_CHUNK;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (ks[mid] <= k)
          lo = mid;
        else
          hi = mid;
      }
      a.anc[k] = (int32_t)(base + lo);
    }
    run += agg;
    __syncthreads();  // ks and su are reused by the next chunk
  }
}

// ---- D: the statistics from the `nb` CTAs' partial sums, by one CTA once they are
// all in place ----
template <typename T>
__device__ __forceinline__ void outer_stats(const FusedOuterArgs<T>& a, int nb, T lwmax,
                                            unsigned long long C) {
  constexpr int NW = OF_NT / 32;
  __shared__ double sd[OF_MAX_NV];
  const OuterArgs<T>& o = a.o;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int D = o.d1 + o.d2, NV = 2 + D;
  for (int q = w; q < NV; q += NW) {
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += __ldcg(o.partials + (long long)b * NV + q);
    s = warp_sum(s);
    if (lane == 0) sd[q] = s;
  }
  __syncthreads();
  const double t1 = sd[0];
  for (int c = tid; c < D; c += OF_NT) {
    const double m = sd[2 + c] / t1;
    const int p = o.perm[c];
    o.stats[4 + p] = m;
    if (o.mean_out) o.mean_out[p] = m;
  }
  if (tid == 0) {
    const bool bad = !(lwmax > neg_inf<T>()) || lwmax != lwmax || !(t1 > 0) || C == 0;
    if (bad) atomicOr(o.err, ERR_NUMERIC);
    const double lz = (double)lwmax + log(t1) - a.logN;
    o.stats[0] += lz;
    o.stats[1] = lz;
    o.stats[2] = t1 * t1 / sd[1];
    o.stats[3] = t1;
    if (o.logz_out) *o.logz_out = o.stats[0];
    *o.lwmax_t = lwmax;
    *o.Csum = C;
  }
  if (a.host_stats) {  // the mirror: the statistics as written above, then the error word
    __syncthreads();
    for (int q = tid; q < 4 + D; q += OF_NT) a.host_stats[q] = o.stats[q];
    if (tid == 0) a.host_stats[4 + D] = (double)*(volatile int*)o.err;
  }
}

// The last of the `nb` CTAs to get here resets the counters for the next step: by
// then every CTA has read the largest log-weight's key and passed the barrier.
template <typename T>
__device__ __forceinline__ void outer_done(const FusedOuterArgs<T>& a, int nb) {
  __syncthreads();
  if (threadIdx.x == 0 && atomicAdd(a.o.done, 1u) == (unsigned)nb - 1u) {
    *a.o.lwmax_key = 0ull;
    *a.o.done = 0u;
    if (a.arrive) *a.arrive = 0u;
  }
}

// One filter's outer stage in one cooperative launch (every CTA resident at once).
template <typename T, int D1, int D2>
__global__ void __launch_bounds__(OF_NT) fused_outer_kernel(const __grid_constant__ FusedOuterArgs<T> a) {
  __shared__ int s_ok;
  const int tid = threadIdx.x, bid = blockIdx.x, nb = gridDim.x, nw = a.nwork;
  T lwmax;
  order_decode(*a.o.lwmax_key, lwmax);
  if (bid < nw) outer_sums<T, D1, D2>(a, bid, nw, lwmax);
  __syncthreads();
  // grid-wide barrier: every CTA is resident, and the wait is bounded all the same
  if (tid == 0) {
    __threadfence();  // the CTA's partial row and count total, written by this thread
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> arr(*a.arrive);
    if (bid != a.withhold) arr.fetch_add(1u, cuda::memory_order_release);
    bool ok = arr.load(cuda::memory_order_acquire) >= (unsigned)nb;
    int spins = 0;
    while (!ok && spins < SPIN_LIMIT) {
      __nanosleep(64);
      ok = arr.load(cuda::memory_order_acquire) >= (unsigned)nb;
      ++spins;
    }
    s_ok = ok;
    if (!ok) atomicOr(a.o.err, ERR_TIMEOUT);
  }
  __syncthreads();
  unsigned long long pre, C;
  count_prefix(a.ctot, bid < nw ? bid : nw, nw, pre, C);
  if (bid == (nb > nw ? nw : nw - 1)) outer_stats<T>(a, nw, lwmax, C);
  if (bid < nw && s_ok && C > 0) outer_scatter<T>(a, bid, nw, lwmax, pre, C);  // else the ancestors stay
  outer_done<T>(a, nb);
}

// The same stage for many filters in two launches, CTAs cstart[f] .. cstart[f+1]-1
// serving filter f with the partition and arithmetic of its single launch: the
// sums, then (after the launch boundary) the prefix, the scatter and the statistics.
template <typename T, int D1, int D2>
__global__ void __launch_bounds__(OF_NT)
    outer_sums_batch_kernel(const FusedOuterArgs<T>* __restrict__ args, const int* __restrict__ cstart, int F) {
  __shared__ int s_f;
  if (threadIdx.x == 0) s_f = find_segment(cstart, F, (int)blockIdx.x);
  __syncthreads();
  const int f = s_f;
  const FusedOuterArgs<T>& a = args[f];
  T lwmax;
  order_decode(*a.o.lwmax_key, lwmax);
  outer_sums<T, D1, D2>(a, (int)blockIdx.x - cstart[f], cstart[f + 1] - cstart[f], lwmax);
}

template <typename T>
__global__ void __launch_bounds__(OF_NT)
    outer_scatter_batch_kernel(const FusedOuterArgs<T>* __restrict__ args, const int* __restrict__ cstart, int F) {
  __shared__ int s_f;
  if (threadIdx.x == 0) s_f = find_segment(cstart, F, (int)blockIdx.x);
  __syncthreads();
  const int f = s_f;
  const FusedOuterArgs<T>& a = args[f];
  const int bid = (int)blockIdx.x - cstart[f], nb = cstart[f + 1] - cstart[f];
  T lwmax;
  order_decode(*a.o.lwmax_key, lwmax);
  unsigned long long pre, C;
  count_prefix(a.ctot, bid, nb, pre, C);
  if (C > 0) outer_scatter<T>(a, bid, nb, lwmax, pre, C);
  if (bid == nb - 1) outer_stats<T>(a, nb, lwmax, C);
  outer_done<T>(a, nb);
}

// CTAs resident on the device at once for the single-filter launch.
template <typename T, int D1, int D2>
int fused_outer_cap() {
  static const int cap = [] {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fused_outer_kernel<T, D1, D2>, OF_NT, 0);
    const int c = occ * sms;
    return c < 2 ? 2 : c;
  }();
  return cap;
}

// CTAs that own items in a filter's outer stage over N items: one a chunk, at most
// OF_MAX_CTAS and one fewer than the resident capacity (the same in the single and
// batched forms, so that their partitions agree).
template <typename T, int D1, int D2>
int fused_outer_grid(long long N) {
  const long long cap = fused_outer_cap<T, D1, D2>() - 1;
  const long long lim = cap < OF_MAX_CTAS ? cap : OF_MAX_CTAS;
  const long long nch = (N + OF_CHUNK - 1) / OF_CHUNK;
  return (int)(nch < lim ? nch : lim);
}

// The single-filter launch: a.nwork CTAs with items and one for the statistics.
template <typename T, int D1, int D2>
cudaError_t fused_outer_launch(const FusedOuterArgs<T>& a, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)a.nwork + 1u);
  cfg.blockDim = dim3(OF_NT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fused_outer_kernel<T, D1, D2>, a);
}

}  // namespace dpf
