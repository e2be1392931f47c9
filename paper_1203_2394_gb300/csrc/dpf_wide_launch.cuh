// The step launch of a wide variant (see dpf_variant_wide.cuh): the block kernel
// with the model constants in device memory, one inner particle a thread.
#pragma once

#include "dpf_variant_wide.cuh"

namespace dpf {

// The model constants of the (float, 8, 56, 8) variant, in this translation unit's
// constant bank (52 KB of the 64 KB): uniform reads become constant-bank operands. They
// are copied from the context's device copy before every launch, in stream order, so
// filters of this variant on one stream may hold different models; filters stepped
// concurrently on different streams must share one model.
static __constant__ MC<float, 8, 56, 8> c_wide_mc;

template <bool TC>
__global__ void __launch_bounds__(256)
    step_kernel_wide(const __grid_constant__ StepArgs<float> a) {
  step_body<float, 8, 56, 8, false, 1, false, TC>(c_wide_mc, a);
}

template <typename T, int D1, int D2, int DY, bool TC>
dpf_status wide_launch(Ctx& x, StepArgs<T>& a, cudaStream_t s) {
  static_assert(sizeof(T) == 4 && D1 == 8 && D2 == 56 && DY == 8, "the compiled wide variant");
  constexpr int MAX_M = WideVariantImpl<T, D1, D2, DY>::MAX_M;
  static_assert(MAX_M == 256, "launch bounds of step_kernel_wide");
  auto k = step_kernel_wide<TC>;
  const int nt = threads_for(x.M);
  const size_t sm = step_geometry<T, D1, D2, DY, false>(x.M, x.L, nt, &a, a.first != 0, 1, TC);
  static size_t attr = 0;  // the largest dynamic shared memory requested so far
  if (sm > attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
    attr = sm;
  }
  if (x.grid_step == 0) {  // persistent grid: as many CTAs as fit on the device at once
    int nb = 0, dev = 0, nsm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, nt, sm);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_error(e, "step kernel occupancy");
    x.grid_step = (nb > 0 ? nb : 1) * nsm;
  }
  cudaError_t e = cudaMemcpyToSymbolAsync(c_wide_mc, x.d_mconst, sizeof(MC<float, 8, 56, 8>), 0,
                                          cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_error(e, "model constants to the constant bank");
  const long long grid = std::min<long long>(x.N, x.grid_step);
  k<<<(unsigned)grid, nt, sm, s>>>(a);
  return cuda_error(cudaGetLastError(), "step kernel launch");
}

}  // namespace dpf
