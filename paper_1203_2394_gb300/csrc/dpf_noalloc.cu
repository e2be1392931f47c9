// dpf_resample_noalloc: the global systematic resampler with its scratch in a
// fixed, statically allocated device array instead of memory allocated per call.
//
// Some callers cannot allocate device memory when they resample: a control
// loop that must not allocate after start-up (an allocation can block on the
// driver or fail under memory pressure), or an application whose framework
// allocator has reserved the whole device so that cudaMalloc would fail. This
// entry point serves them: it makes no cudaMalloc, cudaFree or other
// allocating call. The price is a fixed limit on the number of weights, and
// one scratch array per device shared by every call.
#include <cuda_runtime.h>

#include <mutex>

#include "dpf_internal.h"

namespace dpf {

constexpr long long kNoAllocMaxN = 1ll << 22;  // at most 4,194,304 weights per call
constexpr long long kNoAllocTiles = (kNoAllocMaxN + 2047) / 2048;
constexpr size_t kNoAllocBytes = 64 + (size_t)kNoAllocTiles * (8 + 8 + 4) + 16;  // 41,040 bytes

// The scratch itself (every device that loads the library holds one copy
// until the process exits). Host code must not pass this name to a kernel:
// on the host it is only a stand-in; its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch, looked up once per device.
static void* scratch_address(int dev, cudaError_t* err) {
  static std::mutex mu;
  static void* addr[64] = {nullptr};
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0 || dev >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  if (!addr[dev]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (*err != cudaSuccess) return nullptr;
    addr[dev] = p;
  }
  *err = cudaSuccess;
  return addr[dev];
}

}  // namespace dpf

using namespace dpf;

extern "C" dpf_status dpf_resample_noalloc(const void* w, int32_t dtype, int64_t n,
                                           const uint32_t* u, int32_t* out_idx, void* stream) {
  clear_error();
  if (n < 0) return set_error(DPF_E_INVALID, "dpf_resample_noalloc: n < 0");
  if (n == 0) return DPF_OK;
  if (!w || !u || !out_idx) return set_error(DPF_E_INVALID, "dpf_resample_noalloc: null pointer");
  if (dtype != DPF_F32 && dtype != DPF_F64)
    return set_error(DPF_E_INVALID, "dpf_resample_noalloc: dtype");
  if (n > kNoAllocMaxN)
    return set_error(DPF_E_INVALID,
                     "dpf_resample_noalloc: n exceeds its fixed scratch (at most 4194304 weights); "
                     "use dpf_resample");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "dpf_resample_noalloc: cudaGetDevice");
  unsigned char* b = (unsigned char*)scratch_address(dev, &e);
  if (!b) return cuda_error(e, "dpf_resample_noalloc: cudaGetSymbolAddress");
  cudaStream_t s = (cudaStream_t)stream;
  const long long tiles = (n + 2047) / 2048;
  const size_t used = 64 + (size_t)tiles * (8 + 8 + 4);
  // the scratch keeps the previous call's contents: clear the part this call uses
  e = cudaMemsetAsync(b, 0, used, s);
  if (e != cudaSuccess) return cuda_error(e, "dpf_resample_noalloc: clearing the scratch");
  Scratch sc;
  sc.block = b;
  sc.maxkey = (unsigned long long*)(b + 0);
  sc.C = (unsigned long long*)(b + 8);
  sc.scan.ticket = (unsigned long long*)(b + 16);
  sc.shift = (int*)(b + 24);
  sc.err = (int*)(b + 28);
  sc.scan.agg = (unsigned long long*)(b + 64);
  sc.scan.incl = sc.scan.agg + tiles;
  sc.scan.flags = (uint32_t*)(sc.scan.incl + tiles);
  launch_global_on(w, dtype, n, u, out_idx, sc, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "dpf_resample_noalloc: launch");
  int werr = 0;
  e = cudaMemcpyAsync(&werr, sc.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_error(e, "dpf_resample_noalloc");
  if (werr & 2) return set_error(DPF_E_TIMEOUT, "dpf_resample_noalloc: a device wait timed out");
  if (werr & 1) return set_error(DPF_E_NUMERIC, "dpf_resample_noalloc: no positive or a NaN weight");
  if (werr) return set_error(DPF_E_CUDA, "dpf_resample_noalloc: device bounds check failed");
  return DPF_OK;
}
