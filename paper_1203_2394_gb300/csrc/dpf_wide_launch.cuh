// The step launch of a wide variant (see dpf_variant_wide.cuh): the block kernel
// with the model constants in device memory, one inner particle a thread.
#pragma once

#include "dpf_variant_wide.cuh"

namespace dpf {

template <typename T, int D1, int D2, int DY, bool TC>
dpf_status wide_launch(Ctx& x, StepArgs<T>& a) {
  constexpr int MAX_M = WideVariantImpl<T, D1, D2, DY>::MAX_M;
  auto k = step_kernel_g<T, D1, D2, DY, false, 1, MAX_M, false, TC>;
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
  const long long grid = std::min<long long>(x.N, x.grid_step);
  k<<<(unsigned)grid, nt, sm, x.stream>>>((const MC<T, D1, D2, DY>*)x.d_mconst, a);
  return cuda_error(cudaGetLastError(), "step kernel launch");
}

}  // namespace dpf
