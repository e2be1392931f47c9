// Global systematic resampling on the GPU: a reduction for the quantised total
// C, then one pass that scans the quantised counts with a decoupled look-back
// (Merrill & Garland, "Single-pass Parallel Prefix Scan with Decoupled
// Look-back", 2016) and scatters each tile's share of the ancestor indices.
#pragma once

#include <cuda/atomic>

#include "dpf_common.cuh"
#include "dpf_internal.h"

namespace dpf {

constexpr int SPIN_LIMIT = 1 << 22;  // bounded look-back wait (~0.3 s with the back-off)

typedef unsigned __int128 u128;

// K(c) = #{ k in [0, n) : (k 2^32 + u) C < c n 2^32 }: the number of systematic
// points below the cumulative count c (global rule).
__device__ __forceinline__ long long points_below(unsigned long long c, long long n, uint32_t u,
                                                  unsigned long long C) {
  if (c == 0) return 0;
  const u128 X = ((u128)c * (u128)(unsigned long long)n) << 32;
  const u128 uC = (u128)u * (u128)C;
  if (X <= uC) return 0;
  // K = ceil((X - uC) / (C 2^32)) = floor(Y / C) + 1 with Y = (X - uC - 1) >> 32 < 2^94:
  // a double estimate of the quotient (<= n < 2^31), corrected exactly in 128 bits
  const u128 Y = (X - uC - 1) >> 32;
  const double yd = (double)(unsigned long long)(Y >> 64) * 18446744073709551616.0 +
                    (double)(unsigned long long)Y;
  long long q = (long long)(yd / (double)C);
  if (q < 0) q = 0;
  while (q > 0 && (u128)(unsigned long long)q * C > Y) --q;
  while ((u128)(unsigned long long)(q + 1) * C <= Y) ++q;
  const long long k = q + 1;
  return k >= n ? n : k;
}

// Inputs of the scan-and-scatter pass: the weights W_i, with e = floor(log2 max W)
// given through the shift S - e.
template <typename T>
struct GlobalArgs {
  const T* w;              // n weights
  long long n;
  int shift;               // S - e
  const int* shift_dev;    // if non-null, read S - e from here instead
  const unsigned long long* C;  // device scalar: the quantised total
  const uint32_t* u_ptr;   // device scalar uniform word, or null
  Key key;                 // else u = rand_word(key, t, 0, P_OUTER, 0)
  uint32_t t;
  int32_t* out;
  ScanState st;
  unsigned long long ticket_base;
  uint32_t epoch;
  int* err;
  long long withhold;  // a tile that publishes nothing (a check of the bounded waits); -1: none
};

template <typename T>
__device__ __forceinline__ T exp_t(T v);
template <>
__device__ __forceinline__ float exp_t<float>(float v) { return expf(v); }
template <>
__device__ __forceinline__ double exp_t<double>(double v) { return exp(v); }

// c = floor(W 2^shift) as a 64-bit count (exact: power-of-two scaling, floor).
__device__ __forceinline__ unsigned long long quantize_u64(float W, int shift) {
  return (unsigned long long)floorf(ldexpf(W, shift));
}
__device__ __forceinline__ unsigned long long quantize_u64(double W, int shift) {
  return (unsigned long long)floor(ldexp(W, shift));
}

// One tile of the `ntiles` tiles of one resampling, the tile taken by ticket.
template <typename T>
__device__ __forceinline__ void global_scan_scatter_body(const GlobalArgs<T>& a, long long ntiles) {
  __shared__ unsigned long long cum[SCAN_TILE];
  __shared__ unsigned long long wsum[SCAN_NT / 32];
  __shared__ unsigned long long s_prefix;
  __shared__ long long s_tile;
  __shared__ long long s_klo, s_khi;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  if (tid == 0) {
    const unsigned long long tk = atomicAdd(a.st.ticket, 1ull) - a.ticket_base;
    s_tile = tk < (unsigned long long)ntiles ? (long long)tk : -1;
    if (s_tile < 0) atomicOr(a.err, ERR_BOUNDS);
  }
  __syncthreads();
  const long long tile = s_tile;
  if (tile < 0) return;
  const long long base = tile * SCAN_TILE;
  const unsigned long long C = *a.C;
  const int shift = a.shift_dev ? *a.shift_dev : a.shift;
  const uint32_t u = a.u_ptr ? *a.u_ptr : rand_word(a.key, a.t, 0, P_OUTER, 0);

  // quantise this thread's items (blocked arrangement) and sum them
  unsigned long long c[SCAN_IPT];
  unsigned long long tsum = 0;
#pragma unroll
  for (int q = 0; q < SCAN_IPT; ++q) {
    const long long i = base + (long long)tid * SCAN_IPT + q;
    unsigned long long ci = 0;
    if (i < a.n) {
      ci = quantize_u64(a.w[i], shift);
    }
    c[q] = ci;
    tsum += ci;
  }
  // block exclusive scan of the per-thread sums
  unsigned long long v = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long nb = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += nb;
  }
  if (lane == 31) wsum[wid] = v;
  __syncthreads();
  unsigned long long wpre = 0, agg = 0;
#pragma unroll
  for (int q = 0; q < SCAN_NT / 32; ++q) {
    if (q < wid) wpre += wsum[q];
    agg += wsum[q];
  }
  const unsigned long long texcl = v - tsum + wpre;

  // decoupled look-back for the tile's exclusive prefix: warp 0 publishes the
  // tile's aggregate, then reads its predecessors' flags 32 at a time until it
  // meets an inclusive prefix (every wait is bounded)
  if (wid == 0) {
    const uint32_t ep = a.epoch & 0x3FFFFFFFu;
    unsigned long long prefix = 0;
    if (tile == a.withhold) {
      // publishes nothing: its successors' waits must run out and report
    } else if (tile == 0) {
      if (lane == 0) {
        a.st.incl[0] = agg;
        cuda::atomic_ref<uint32_t, cuda::thread_scope_device>(a.st.flags[0])
            .store((ep << 2) | 2u, cuda::memory_order_release);
      }
    } else {
      if (lane == 0) {
        a.st.agg[tile] = agg;
        cuda::atomic_ref<uint32_t, cuda::thread_scope_device>(a.st.flags[tile])
            .store((ep << 2) | 1u, cuda::memory_order_release);
      }
      long long hi = tile - 1;
      while (true) {
        const long long j = hi - lane;
        uint32_t fv = 0;
        bool ready = true;
        if (j >= 0) {
          cuda::atomic_ref<uint32_t, cuda::thread_scope_device> f(a.st.flags[j]);
          fv = f.load(cuda::memory_order_acquire);
          ready = (fv >> 2) == ep && (fv & 3u) != 0u;
          int spins = 0;
          while (!ready && spins < SPIN_LIMIT) {
            __nanosleep(64);
            fv = f.load(cuda::memory_order_acquire);
            ready = (fv >> 2) == ep && (fv & 3u) != 0u;
            ++spins;
          }
        }
        if (!__all_sync(FULL, ready)) {
          if (lane == 0) atomicOr(a.err, ERR_TIMEOUT);
          break;
        }
        const unsigned inc = __ballot_sync(FULL, j >= 0 && (fv & 3u) == 2u);
        const int first = inc ? __ffs(inc) - 1 : 32;
        unsigned long long val = 0;
        if (j >= 0 && lane <= first) val = lane == first ? a.st.incl[j] : a.st.agg[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(FULL, val, o);
        prefix += val;
        if (inc || hi < 32) break;
        hi -= 32;
      }
      if (lane == 0) {
        a.st.incl[tile] = prefix + agg;
        cuda::atomic_ref<uint32_t, cuda::thread_scope_device>(a.st.flags[tile])
            .store((ep << 2) | 2u, cuda::memory_order_release);
      }
    }
    if (lane == 0) {
      s_prefix = prefix;
      s_klo = points_below(prefix, a.n, u, C);
      s_khi = points_below(prefix + agg, a.n, u, C);
    }
  }
  __syncthreads();
  // global inclusive cumulative counts of this tile into shared memory
  unsigned long long run = s_prefix + texcl;
#pragma unroll
  for (int q = 0; q < SCAN_IPT; ++q) {
    run += c[q];
    cum[tid * SCAN_IPT + q] = run;
  }
  __syncthreads();
  // scatter: output k takes the first item of this tile with cum * n 2^32 > (k 2^32 + u) C
  const long long len = (a.n - base) < SCAN_TILE ? (a.n - base) : SCAN_TILE;
  const u128 scale = (u128)(unsigned long long)a.n << 32;
  for (long long k = s_klo + tid; k < s_khi; k += SCAN_NT) {
    const u128 rhs = ((u128)(unsigned long long)k << 32 | u) * (u128)C;
    int lo = 0, hi = (int)len - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((u128)cum[mid] * scale > rhs)
        hi = mid;
      else
        lo = mid + 1;
    }
    a.out[k] = (int32_t)(base + lo);
  }
}

template <typename T>
__global__ void __launch_bounds__(SCAN_NT) global_scan_scatter(GlobalArgs<T> a) {
  global_scan_scatter_body<T>(a, gridDim.x);
}

}  // namespace dpf
