// A check of the outer stage's bounded barrier wait (part of
// dpf_check_bounded_wait): no GPU fault, only a wait that runs out.
#include <cuda_runtime.h>

#include <cmath>

#include "dpf_internal.h"
#include "dpf_outer.cuh"

namespace dpf {

// The cooperative outer stage over 3 chunks of zero log-weights (d1 = d2 = 1; 3 CTAs
// with items and one for the statistics) with CTA 0 never arriving at the grid
// barrier: the waits of all four CTAs run out, the error word reports the timeout,
// the scatter is skipped, and the last CTA still resets the counters. Returns the
// status the error word maps to.
dpf_status check_outer_barrier(cudaStream_t s) {
  const long long n = 3 * OF_CHUNK;
  const size_t fb = sizeof(float) * n;
  const size_t bytes = 4 * fb + sizeof(int32_t) * n + 256;
  unsigned char* b = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&b, bytes, s);
  if (e != cudaSuccess) return cuda_error(e, "dpf_check_bounded_wait: allocation");
  e = cudaMemsetAsync(b, 0, bytes, s);
  unsigned char* tail = b + 4 * fb + sizeof(int32_t) * n;  // 256 bytes of scalars, 8-aligned
  FusedOuterArgs<float> a{};
  OuterArgs<float>& o = a.o;
  o.lw = (const float*)b;
  o.xm = (const float*)(b + fb);
  o.zm = (const float*)(b + 2 * fb);
  a.w_out = (float*)(b + 3 * fb);
  a.anc = (int32_t*)(b + 4 * fb);
  o.N = n;
  o.d1 = 1;
  o.d2 = 1;
  o.partials = (double*)(tail + 0);                    // 3 rows of 4
  a.ctot = (unsigned long long*)(tail + 96);           // 3
  o.lwmax_key = (unsigned long long*)(tail + 120);
  o.Csum = (unsigned long long*)(tail + 128);
  o.done = (unsigned int*)(tail + 136);                // done, then the barrier's arrivals
  a.arrive = o.done + 1;
  o.err = (int*)(tail + 144);
  o.lwmax_t = (float*)(tail + 148);
  o.stats = (double*)(tail + 152);                     // 4 + 2
  o.perm = (const int*)(tail + 200);                   // {0, 1}
  const unsigned long long key0 = 0x80000000ull;       // the order key of 0.0f
  const int perm[2] = {0, 1};
  if (e == cudaSuccess) e = cudaMemcpyAsync(tail + 120, &key0, 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tail + 200, perm, sizeof(perm), cudaMemcpyHostToDevice, s);
  a.shift = 62 - ceil_log2_i(n);
  a.logN = std::log((double)n);
  a.key = Key{1u, 0u};
  a.t = 1;
  a.withhold = 0;
  a.nwork = 3;
  if (e == cudaSuccess) e = fused_outer_launch<float, 1, 1>(a, s);
  int w = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&w, o.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(b, s);
  if (e != cudaSuccess) return cuda_error(e, "dpf_check_bounded_wait: outer stage");
  return err_word_status(w, "dpf_check_bounded_wait: outer stage");
}

}  // namespace dpf
