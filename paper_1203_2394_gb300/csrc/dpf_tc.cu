// dpf_tc_matmul: the tensor-core product the step and proposal kernels build on,
// run alone so that the descriptors, the operand layout, the TF32 split and the
// TMEM read-back can be checked against a plain product.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dpf_internal.h"
#include "dpf_tc.cuh"

namespace dpf {

constexpr int TCM_NT = 128;            // one thread per row of the 128-row tile
constexpr int TCM_SPIN = 1 << 20;      // bounded wait for the MMAs

// One CTA per 128-row tile of D = A B^T. MODE 0: TF32 once; 1: 3xTF32
// (A_hi B_hi + A_hi B_lo + A_lo B_hi); 2: BF16 operands.
template <int MODE>
__global__ void __launch_bounds__(TCM_NT)
    tc_matmul_kernel(const void* __restrict__ A, const void* __restrict__ B, float* __restrict__ D,
                     int N, int K, uint32_t ncols, int* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_taddr;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  constexpr int ES = MODE == 2 ? 2 : 4;  // element bytes
  const int kc16 = K * ES / 16;
  const uint32_t a_bytes = 128u * K * ES, b_bytes = (uint32_t)N * K * ES;
  unsigned char* a_hi = sm;
  unsigned char* a_lo = sm + a_bytes;
  unsigned char* b_hi = sm + 2 * a_bytes;
  unsigned char* b_lo = b_hi + b_bytes;
  const long long row0 = (long long)blockIdx.x * 128;

  if (w == 0) {
    tc::tmem_alloc(&s_taddr, ncols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  // operands into the K-major layout
  if (MODE == 2) {
    const __nv_bfloat16* a = (const __nv_bfloat16*)A + (row0 + tid) * K;
    for (int k = 0; k < K; ++k) *(__nv_bfloat16*)(a_hi + tc::kmajor_offset(tid, 2 * k, kc16)) = a[k];
    for (int n = tid; n < N; n += TCM_NT) {
      const __nv_bfloat16* b = (const __nv_bfloat16*)B + (long long)n * K;
      for (int k = 0; k < K; ++k) *(__nv_bfloat16*)(b_hi + tc::kmajor_offset(n, 2 * k, kc16)) = b[k];
    }
  } else {
    const float* a = (const float*)A + (row0 + tid) * K;
    for (int k = 0; k < K; ++k) {
      float hi, lo;
      tc::split_tf32(a[k], hi, lo);
      *(float*)(a_hi + tc::kmajor_offset(tid, 4 * k, kc16)) = hi;
      *(float*)(a_lo + tc::kmajor_offset(tid, 4 * k, kc16)) = lo;
    }
    for (int n = tid; n < N; n += TCM_NT) {
      const float* b = (const float*)B + (long long)n * K;
      for (int k = 0; k < K; ++k) {
        float hi, lo;
        tc::split_tf32(b[k], hi, lo);
        *(float*)(b_hi + tc::kmajor_offset(n, 4 * k, kc16)) = hi;
        *(float*)(b_lo + tc::kmajor_offset(n, 4 * k, kc16)) = lo;
      }
    }
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = s_taddr;
  if (tid == 0) {
    const uint32_t idesc = tc::instr_desc(MODE == 2 ? tc::FMT_BF16 : tc::FMT_TF32, 128, N);
    const uint32_t sa_hi = smem_addr(a_hi), sa_lo = smem_addr(a_lo);
    const uint32_t sb_hi = smem_addr(b_hi), sb_lo = smem_addr(b_lo);
    const int ksteps = K * ES / 32;
    for (int ks = 0; ks < ksteps; ++ks) {
      const uint32_t off = (uint32_t)ks * 256;
      if (MODE == 2) {
        tc::mma_f16(taddr, tc::smem_desc(sa_hi + off, kc16), tc::smem_desc(sb_hi + off, kc16), idesc,
                    ks > 0);
      } else if (MODE == 0) {
        tc::mma_tf32(taddr, tc::smem_desc(sa_hi + off, kc16), tc::smem_desc(sb_hi + off, kc16), idesc,
                     ks > 0);
      } else {
        // small terms first, then the leading one
        tc::mma_tf32(taddr, tc::smem_desc(sa_lo + off, kc16), tc::smem_desc(sb_hi + off, kc16), idesc,
                     ks > 0);
        tc::mma_tf32(taddr, tc::smem_desc(sa_hi + off, kc16), tc::smem_desc(sb_lo + off, kc16), idesc, 1);
        tc::mma_tf32(taddr, tc::smem_desc(sa_hi + off, kc16), tc::smem_desc(sb_hi + off, kc16), idesc, 1);
      }
    }
    tc::commit(&bar);
  }
  const bool ok = tc::bar_wait(&bar, 0, TCM_SPIN);
  if (!ok && lane == 0) atomicOr(err, ERR_TIMEOUT);
  tc::fence_after();
  if (ok) {
    float* d = D + (row0 + tid) * N;
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::ld16(taddr + ((uint32_t)(32 * w) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) d[c0 + j] = v[j];
    }
  }
  tc::fence_before();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(taddr, ncols);
}

}  // namespace dpf

using namespace dpf;

extern "C" dpf_status dpf_tc_matmul(const void* A, const void* B, float* D, int32_t M, int32_t N,
                                    int32_t K, int32_t mode, void* stream) {
  clear_error();
  if (!A || !B || !D) return set_error(DPF_E_INVALID, "dpf_tc_matmul: null pointer");
  const int kstep = mode == DPF_TC_BF16 ? 16 : 8;
  const int kmax = mode == DPF_TC_BF16 ? 128 : 64;
  if (mode < DPF_TC_TF32 || mode > DPF_TC_BF16 || M < 128 || M % 128 || N < 16 || N > 128 || N % 16 ||
      K < kstep || K > kmax || K % kstep)
    return set_error(DPF_E_INVALID,
                     "dpf_tc_matmul: M a multiple of 128, N a multiple of 16 in [16, 128], K a multiple of "
                     "8 up to 64 (TF32) or of 16 up to 128 (BF16)");
  cudaStream_t s = (cudaStream_t)stream;
  const int es = mode == DPF_TC_BF16 ? 2 : 4;
  const size_t smem = (size_t)2 * 128 * K * es + (size_t)2 * N * K * es;
  uint32_t ncols = 32;
  while ((int)ncols < N) ncols <<= 1;
  int* err = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&err, sizeof(int), s);
  if (e != cudaSuccess) return cuda_error(e, "dpf_tc_matmul: allocation");
  cudaMemsetAsync(err, 0, sizeof(int), s);
  auto launch = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<M / 128, TCM_NT, smem, s>>>(A, B, D, N, K, ncols, err);
  };
  if (mode == DPF_TC_TF32) launch(tc_matmul_kernel<0>);
  else if (mode == DPF_TC_TF32X3) launch(tc_matmul_kernel<1>);
  else launch(tc_matmul_kernel<2>);
  e = cudaGetLastError();
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(err, s);
  if (e != cudaSuccess) return cuda_error(e, "dpf_tc_matmul");
  if (h) return set_error(DPF_E_TIMEOUT, "dpf_tc_matmul: the MMAs did not complete in time");
  return DPF_OK;
}
