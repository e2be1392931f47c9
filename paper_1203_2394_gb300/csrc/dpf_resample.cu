// dpf_resample: the standalone systematic-resampling entry point (global rule
// over one segment, or the local rule over many short segments).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "dpf_internal.h"
#include "dpf_resample.cuh"

namespace dpf {

// Largest weight as an order-preserving 64-bit key (weights are >= 0, so the
// IEEE bit pattern orders like the value); flags negative, NaN and inf.
template <typename T>
__global__ void wmax_kernel(const T* w, long long n, unsigned long long* maxkey, int* err) {
  unsigned long long best = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const T W = w[i];
    if (!(W >= T(0)) || isinf(W)) atomicOr(err, ERR_NUMERIC);
    const unsigned long long k = sizeof(T) == 8 ? (unsigned long long)__double_as_longlong((double)W)
                                                : (unsigned long long)__float_as_uint((float)W);
    best = k > best ? k : best;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(FULL, best, o);
    best = v > best ? v : best;
  }
  if ((threadIdx.x & 31) == 0 && best) atomicMax(maxkey, best);
}

// C = sum floor(W_i 2^(S - e)) with e from the largest weight; also publishes S - e.
template <typename T>
__global__ void sumc_kernel(const T* w, long long n, int S, const unsigned long long* maxkey,
                            unsigned long long* C, int* shift_out, int* err) {
  const unsigned long long k = *maxkey;
  if (k == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, ERR_NUMERIC);
    return;
  }
  const int e = sizeof(T) == 8 ? ilogb(__longlong_as_double((long long)k))
                               : ilogbf(__uint_as_float((uint32_t)k));
  const int shift = S - e;
  if (blockIdx.x == 0 && threadIdx.x == 0) *shift_out = shift;
  unsigned long long s = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    s += quantize_u64(w[i], shift);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(C, s);
}

// Local rule: one block per segment of n <= NT weights.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) local_resample_kernel(const T* w, int n, const uint32_t* u,
                                                            int32_t* out, int* err) {
  __shared__ uint32_t cum[NT];
  __shared__ T redT[NT / 32];
  __shared__ uint32_t redU[NT / 32];
  const long long seg = blockIdx.x;
  const int j = threadIdx.x;
  T W = T(0);
  if (j < n) W = w[seg * n + j];
  const int bad = __syncthreads_or(j < n && (!(W >= T(0)) || isinf(W)));
  if (bad) {
    if (j == 0) atomicOr(err, ERR_NUMERIC);
    return;
  }
  const T mx = block_max<NT>(W, redT);
  if (!(mx > T(0))) {
    if (j == 0) atomicOr(err, ERR_NUMERIC);
    return;
  }
  const int e = sizeof(T) == 8 ? ilogb((double)mx) : ilogbf((float)mx);
  const int shift = (31 - ceil_log2_i(n)) - e;
  const uint32_t c = j < n ? quantize_u32(W, shift) : 0u;
  const uint32_t incl = block_incl_scan_u32<NT>(c, redU);
  cum[j] = incl;
  __syncthreads();
  const uint32_t C = cum[n - 1];
  if (j < n) out[seg * n + j] = sys_local_pick(cum, n, C, n, j, u[seg]);
}

template <typename T>
static dpf_status launch_local(const T* w, int n, long long nseg, const uint32_t* u, int32_t* out,
                               int* err, cudaStream_t s) {
#define DPF_LOCAL_CASE(NTV)                                                      \
  if (n <= NTV) {                                                                \
    local_resample_kernel<T, NTV><<<(unsigned)nseg, NTV, 0, s>>>(w, n, u, out, err); \
    return DPF_OK;                                                               \
  }
  DPF_LOCAL_CASE(32)
  DPF_LOCAL_CASE(64)
  DPF_LOCAL_CASE(128)
  DPF_LOCAL_CASE(256)
  DPF_LOCAL_CASE(512)
  DPF_LOCAL_CASE(1024)
#undef DPF_LOCAL_CASE
  return set_error(DPF_E_INVALID, "dpf_resample: local segments hold at most 1024 weights");
}

template <typename T>
static void launch_global(const T* w, long long n, const uint32_t* u, int32_t* out, Scratch& sc,
                          cudaStream_t s, long long withhold = -1) {
  const int S = 62 - ceil_log2_i(n);
  const int grid = (int)std::min<long long>((n + 1023) / 1024, 4 * 152);
  wmax_kernel<T><<<grid, 256, 0, s>>>(w, n, sc.maxkey, sc.err);
  sumc_kernel<T><<<grid, 256, 0, s>>>(w, n, S, sc.maxkey, sc.C, sc.shift, sc.err);
  GlobalArgs<T> a{};
  a.w = w;
  a.n = n;
  a.shift_dev = sc.shift;
  a.C = sc.C;
  a.u_ptr = u;
  a.out = out;
  a.st = sc.scan;
  a.ticket_base = 0;
  a.epoch = 1;
  a.err = sc.err;
  a.withhold = withhold;
  const long long tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  global_scan_scatter<T><<<(unsigned)tiles, SCAN_NT, 0, s>>>(a);
}

// Launch the global-rule pipeline on scratch the caller has laid out (and zeroed).
void launch_global_on(const void* w, int32_t dtype, long long n, const uint32_t* u, int32_t* out,
                      Scratch& sc, cudaStream_t s) {
  if (dtype == DPF_F32)
    launch_global<float>((const float*)w, n, u, out, sc, s);
  else
    launch_global<double>((const double*)w, n, u, out, sc, s);
}

template <typename T>
__global__ void box_muller_kernel(const uint32_t* words, long long n_pairs, T* out) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n_pairs;
       p += (long long)gridDim.x * blockDim.x) {
    T a, b;
    box_muller(words[2 * p], words[2 * p + 1], a, b);
    out[2 * p] = a;
    out[2 * p + 1] = b;
  }
}

}  // namespace dpf

using namespace dpf;

extern "C" dpf_status dpf_box_muller(const uint32_t* words, int64_t n_pairs, int32_t dtype,
                                     void* out, void* stream) {
  clear_error();
  if (n_pairs < 0 || (n_pairs > 0 && (!words || !out)))
    return set_error(DPF_E_INVALID, "dpf_box_muller: bad arguments");
  if (dtype != DPF_F32 && dtype != DPF_F64) return set_error(DPF_E_INVALID, "dpf_box_muller: dtype");
  if (n_pairs == 0) return DPF_OK;
  const int grid = (int)std::min<long long>((n_pairs + 255) / 256, 152 * 8);
  if (dtype == DPF_F32)
    box_muller_kernel<float><<<grid, 256, 0, (cudaStream_t)stream>>>(words, n_pairs, (float*)out);
  else
    box_muller_kernel<double><<<grid, 256, 0, (cudaStream_t)stream>>>(words, n_pairs, (double*)out);
  return cuda_error(cudaGetLastError(), "dpf_box_muller");
}

__global__ void fill_ones_kernel(float* w, long long n) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < n) w[e] = 1.f;
}

extern "C" dpf_status dpf_check_bounded_wait(void* stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = 3 * SCAN_TILE;
  float* w = nullptr;
  int32_t* out = nullptr;
  uint32_t* u = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&w, sizeof(float) * n, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&out, sizeof(int32_t) * n, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&u, sizeof(uint32_t), s);
  if (e != cudaSuccess) return cuda_error(e, "dpf_check_bounded_wait: allocation");
  fill_ones_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w, n);
  cudaMemsetAsync(u, 0, sizeof(uint32_t), s);
  Scratch sc;
  dpf_status st = scratch_alloc(sc, 3, s);
  if (!st) {
    launch_global<float>(w, n, u, out, sc, s, 0);  // tile 0 withholds its prefix
    st = scratch_finish(sc, s, "dpf_check_bounded_wait");
  }
  cudaFreeAsync(w, s);
  cudaFreeAsync(out, s);
  cudaFreeAsync(u, s);
  if (st != DPF_E_TIMEOUT)
    return st ? st : set_error(DPF_E_CUDA, "dpf_check_bounded_wait: the scan's wait did not run out");
  // the same for the grid barrier of a step's outer stage (CTA 0 never arrives)
  st = check_outer_barrier(s);
  if (st != DPF_E_TIMEOUT)
    return st ? st : set_error(DPF_E_CUDA, "dpf_check_bounded_wait: the outer stage's barrier wait did not run out");
  return st;
}

extern "C" dpf_status dpf_resample(const void* w, int32_t dtype, int64_t n_total, int64_t n_seg,
                                   int32_t rule, const uint32_t* u, int32_t* out_idx,
                                   void* stream) {
  clear_error();
  if (n_total < 0 || n_seg < 1) return set_error(DPF_E_INVALID, "dpf_resample: bad sizes");
  if (n_total == 0) return DPF_OK;
  if (!w || !u || !out_idx) return set_error(DPF_E_INVALID, "dpf_resample: null pointer");
  if (dtype != DPF_F32 && dtype != DPF_F64) return set_error(DPF_E_INVALID, "dpf_resample: dtype");
  if (n_total % n_seg) return set_error(DPF_E_INVALID, "dpf_resample: n_seg must divide n_total");
  if (n_total >= (1ll << 31)) return set_error(DPF_E_INVALID, "dpf_resample: n_total >= 2^31");
  cudaStream_t s = (cudaStream_t)stream;
  const long long seglen = n_total / n_seg;
  if (rule == DPF_SYS_GLOBAL) {
    if (n_seg != 1) return set_error(DPF_E_INVALID, "dpf_resample: global rule needs n_seg == 1");
    const long long tiles = (n_total + SCAN_TILE - 1) / SCAN_TILE;
    Scratch sc;
    dpf_status st = scratch_alloc(sc, tiles, s);
    if (st) return st;
    if (dtype == DPF_F32)
      launch_global<float>((const float*)w, n_total, u, out_idx, sc, s);
    else
      launch_global<double>((const double*)w, n_total, u, out_idx, sc, s);
    return scratch_finish(sc, s, "dpf_resample");
  }
  if (rule != DPF_SYS_LOCAL) return set_error(DPF_E_INVALID, "dpf_resample: unknown rule");
  if (seglen > 1024) return set_error(DPF_E_INVALID, "dpf_resample: local segments hold <= 1024");
  Scratch sc;
  dpf_status st = scratch_alloc(sc, 0, s);
  if (st) return st;
  st = dtype == DPF_F32
           ? launch_local<float>((const float*)w, (int)seglen, n_seg, u, out_idx, sc.err, s)
           : launch_local<double>((const double*)w, (int)seglen, n_seg, u, out_idx, sc.err, s);
  if (st) {
    scratch_free(sc, s);
    return st;
  }
  return scratch_finish(sc, s, "dpf_resample");
}
