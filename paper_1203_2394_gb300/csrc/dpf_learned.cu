// The learned inner proposal: an MLP (3 hidden ReLU layers) with a Gaussian-mixture
// head, its training on the GPU (forward, backward and Adam kernels written here) and
// the packing of its weights for the tensor-core forward pass of the filter step.
//
// Parameters, one FP32 buffer in this order (row-major, W_l is out x in):
//   W1 (H x din), b1 (H), W2 (H x H), b2, W3 (H x H), b3, W4 (dout x H), b4 (dout),
// with dout = C (1 + 2 d2): logits, then the C x d2 means, then the C x d2 raw log
// standard deviations (clamped to [-7, 5] where used).
//
// Training minimises the weighted negative log-likelihood of the recorded
// (features, z) rows, sum_b w_b (-log q(z_b | f_b)) / sum_b w_b, per minibatch, with
// Adam (Kingma and Ba 2015). With bf16 on, the forward pass rounds the inputs, the
// weights and every hidden activation to bfloat16 as the tensor-core pass does
// (gradients pass the rounding straight through); off, it is plain FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dpf_learned.h"
#include "dpf_tc.cuh"

namespace dpf {

// ---- the training products: C[M x N] = op(A) op(B) with an epilogue ----
// A(m, k) = TA ? A[k lda + m] : A[m lda + k];  B(k, n) = TB ? B[n ldb + k] : B[k ldb + n].
// EPI: 0 store; 1 bias, ReLU and optional bfloat16 rounding; 2 bias; 3 multiply by
// (mask(m, n) > 0), mask with leading dimension ldc.
__device__ __forceinline__ float round_bf16(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// On the tensor cores (tcgen05):
// One CTA of 128 threads per 128-row x npad-column tile of C (npad <= 64 columns of a
// TMEM accumulator in FP32; blockIdx.y picks the column tile) and one slice of K
// (blockIdx.z; the slices of a long K add their partial products into C, which the
// caller has zeroed, with atomic adds: the plain-store epilogue only). K is taken in
// chunks of 128 bytes a row (64 BF16 or 32 TF32 values): the threads load op(A) and
// op(B)^T from global memory, round them to the operand format and write them in the
// K-major layout without swizzle; one thread issues the MMAs (four 32-byte K steps a
// chunk) and commits them to an mbarrier that every thread waits on (bounded; the CTA
// agrees on the outcome before it reuses the tiles); thread r then reads row r of the
// accumulator for the epilogue.
// PREC 0: BF16 operands (kind::f16), the forward pass's own rounding; PREC 1: 3xTF32
// (A_hi B_hi + A_hi B_lo + A_lo B_hi, kind::tf32), about FP32 accuracy.
constexpr int TG_NT = 128;
constexpr int TG_ROWB = 128;        // bytes of one K chunk of a row
constexpr int TG_KC16 = TG_ROWB / 16;
constexpr int TG_SPIN = 1 << 22;

template <int PREC>
__device__ __forceinline__ void tg_put(unsigned char* hi, unsigned char* lo, int r, int c, float v) {
  if (PREC == 0) {
    *(__nv_bfloat16*)(hi + tc::kmajor_offset(r, 2 * c, TG_KC16)) = __float2bfloat16_rn(v);
  } else {
    float h, l;
    tc::split_tf32(v, h, l);
    *(float*)(hi + tc::kmajor_offset(r, 4 * c, TG_KC16)) = h;
    *(float*)(lo + tc::kmajor_offset(r, 4 * c, TG_KC16)) = l;
  }
}

template <bool TA, bool TB, int EPI, int PREC>
__global__ void __launch_bounds__(TG_NT)
    tgemm_kernel(int M, int N, int K, const float* __restrict__ A, int lda, const float* __restrict__ B, int ldb,
                 float* __restrict__ C, int ldc, const float* __restrict__ bias, const float* __restrict__ mask,
                 int round, int npad, uint32_t ncols, int kslice, int* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_taddr;
  constexpr int KC = PREC == 0 ? TG_ROWB / 2 : TG_ROWB / 4;  // K values a chunk
  const int tid = threadIdx.x, w = tid >> 5;
  const uint32_t a_bytes = 128u * TG_ROWB, b_bytes = (uint32_t)npad * TG_ROWB;
  unsigned char* a_hi = sm;
  unsigned char* b_hi = sm + a_bytes;
  unsigned char* a_lo = sm + a_bytes + b_bytes;  // 3xTF32 only
  unsigned char* b_lo = a_lo + a_bytes;
  const long long m0 = (long long)blockIdx.x * 128;
  const int n0 = blockIdx.y * npad;                      // this CTA's first column
  const int kbeg = blockIdx.z * kslice;                  // and its slice of K
  const int kend = kbeg + kslice < K ? kbeg + kslice : K;
  const bool split = gridDim.z > 1;
  if (w == 0) {
    tc::tmem_alloc(&s_taddr, ncols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = s_taddr;
  const uint32_t idesc = tc::instr_desc(PREC == 0 ? tc::FMT_BF16 : tc::FMT_TF32, 128, npad);
  int ok = 1;
  uint32_t phase = 0;
  for (int k0 = kbeg; k0 < kend && ok; k0 += KC) {
    // op(A) rows m0 .. m0 + 127 and op(B)^T rows 0 .. npad - 1, K columns k0 .. k0 + KC - 1;
    // the index runs fastest along the operand's contiguous dimension
    for (int e = tid; e < 128 * KC; e += TG_NT) {
      const int r = TA ? e % 128 : e / KC, c = TA ? e / 128 : e % KC;
      const long long m = m0 + r;
      const int k = k0 + c;
      float v = 0.f;
      if (m < M && k < kend) v = TA ? A[(long long)k * lda + m] : A[m * lda + k];
      tg_put<PREC>(a_hi, a_lo, r, c, v);
    }
    for (int e = tid; e < npad * KC; e += TG_NT) {
      const int nl = TB ? e / KC : e % npad, c = TB ? e % KC : e / npad;
      const int n = n0 + nl, k = k0 + c;
      float v = 0.f;
      if (n < N && k < kend) v = TB ? B[(long long)n * ldb + k] : B[(long long)k * ldb + n];
      tg_put<PREC>(b_hi, b_lo, nl, c, v);
    }
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
      const uint32_t sah = smem_addr(a_hi), sbh = smem_addr(b_hi), sal = smem_addr(a_lo), sbl = smem_addr(b_lo);
#pragma unroll
      for (int ks = 0; ks < TG_ROWB / 32; ++ks) {
        const uint32_t off = (uint32_t)ks * 256;
        const uint32_t acc = (k0 > kbeg || ks > 0) ? 1u : 0u;
        if (PREC == 0) {
          tc::mma_f16(taddr, tc::smem_desc(sah + off, TG_KC16), tc::smem_desc(sbh + off, TG_KC16), idesc, acc);
        } else {  // small terms first, then the leading one
          tc::mma_tf32(taddr, tc::smem_desc(sal + off, TG_KC16), tc::smem_desc(sbh + off, TG_KC16), idesc, acc);
          tc::mma_tf32(taddr, tc::smem_desc(sah + off, TG_KC16), tc::smem_desc(sbl + off, TG_KC16), idesc, 1);
          tc::mma_tf32(taddr, tc::smem_desc(sah + off, TG_KC16), tc::smem_desc(sbh + off, TG_KC16), idesc, 1);
        }
      }
      tc::commit(&bar);
    }
    const bool done = tc::bar_wait(&bar, phase, TG_SPIN);
    phase ^= 1u;
    tc::fence_after();
    ok = __syncthreads_and(done ? 1 : 0);  // every thread saw the MMAs finish before the tiles change
  }
  if (!ok) {
    if (tid == 0) atomicOr(err, ERR_TIMEOUT);
    tc::bar_wait(&bar, phase ^ 1u, TG_SPIN);  // give MMAs still in flight a second bound
  } else {
    const long long m = m0 + tid;
    for (int c0 = 0; c0 < npad; c0 += 16) {
      float v[16];
      tc::ld16(taddr + ((uint32_t)(32 * w) << 16) + (uint32_t)c0, v);
      if (m < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c0 + j;
          if (n >= N) break;
          float x = v[j];
          if (EPI == 1) {
            x = fmaxf(x + bias[n], 0.f);
            if (round) x = round_bf16(x);
          } else if (EPI == 2) {
            x += bias[n];
          } else if (EPI == 3) {
            x = mask[m * ldc + n] > 0.f ? x : 0.f;
          }
          if (split)
            atomicAdd(C + m * ldc + n, x);
          else
            C[m * ldc + n] = x;
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(taddr, ncols);
}

// C = op(A) op(B) with the epilogue EPI on the tensor cores: BF16 operands when the
// proposal trains in its BF16 form, 3xTF32 otherwise. Column tiles of up to 64; a long
// K (the batch dimension of a weight gradient) is split over CTAs that accumulate into C.
template <bool TA, bool TB, int EPI>
static void tgemm(cudaStream_t s, int prec_bf16, int* err, int M, int N, int K, const float* A, int lda,
                  const float* B, int ldb, float* C, int ldc, const float* bias = nullptr,
                  const float* mask = nullptr, int round = 0) {
  const int npad = std::min(64, (N + 15) / 16 * 16);
  const uint32_t ncols = npad <= 32 ? 32u : 64u;
  const int mt = (M + 127) / 128, nt = (N + npad - 1) / npad;
  const int kc = prec_bf16 ? TG_ROWB / 2 : TG_ROWB / 4;
  // slices of at least 4 chunks, enough of them for about 152 CTAs (plain-store products)
  int ks = 1;
  if (EPI == 0)
    while (ks < 16 && (long long)mt * nt * ks * 2 <= 152 && K / (2 * ks) >= 4 * kc) ks *= 2;
  const int kslice = (K + ks - 1) / ks / kc * kc + ((K + ks - 1) / ks % kc ? kc : 0);
  ks = (K + kslice - 1) / kslice;  // every slice holds part of K
  if (ks > 1) cudaMemsetAsync(C, 0, sizeof(float) * (size_t)M * ldc, s);
  const dim3 grid((unsigned)mt, (unsigned)nt, (unsigned)ks);
  // at most 512 / ncols CTAs can hold TMEM on an SM at once: a CTA asks for enough shared
  // memory that no more become resident (they would wait inside the allocation)
  const size_t floor_smem = ncols >= 64 ? 29 * 1024 : 0;
  if (prec_bf16) {
    const size_t smem = std::max((size_t)(128 + npad) * TG_ROWB, floor_smem);
    auto k = tgemm_kernel<TA, TB, EPI, 0>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<grid, TG_NT, smem, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, mask, round, npad, ncols, kslice, err);
  } else {
    const size_t smem = std::max((size_t)2 * (128 + npad) * TG_ROWB, floor_smem);
    auto k = tgemm_kernel<TA, TB, EPI, 1>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<grid, TG_NT, smem, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, mask, round, npad, ncols, kslice, err);
  }
}

// ---- the mixture head: loss and d(loss)/d(out) per row ----
struct HeadArgs {
  const float* out;  // n x dout
  const float* Z;    // n x d2
  const float* w;    // n
  const double* wsum;
  float* dout;       // n x dout
  double* loss;      // accumulated: sum_b w_b (-log q_b) / wsum
  int n, d2, C, dout_n;
};

__global__ void head_loss_kernel(HeadArgs a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.n) return;
  const int C = a.C, d2 = a.d2, D = a.dout_n;
  const float* o = a.out + (long long)b * D;
  const float* z = a.Z + (long long)b * d2;
  float* g = a.dout + (long long)b * D;
  // log softmax of the logits
  float lmax = -INFINITY;
  for (int c = 0; c < C; ++c) lmax = fmaxf(lmax, o[c]);
  float se = 0.f;
  for (int c = 0; c < C; ++c) se += expf(o[c] - lmax);
  const float lse_a = lmax + logf(se);
  float lc[kMaxComponents];
  float cmax = -INFINITY;
  const float HL2PI = 0.91893853320467274f;
  for (int c = 0; c < C; ++c) {
    float s = o[c] - lse_a;
    for (int d = 0; d < d2; ++d) {
      const float mu = o[C + c * d2 + d];
      const float ls = fminf(fmaxf(o[C + C * d2 + c * d2 + d], kLogSigMin), kLogSigMax);
      const float u = (z[d] - mu) * expf(-ls);
      s += -0.5f * u * u - ls - HL2PI;
    }
    lc[c] = s;
    cmax = fmaxf(cmax, s);
  }
  float sc = 0.f;
  for (int c = 0; c < C; ++c) sc += expf(lc[c] - cmax);
  const float lq = cmax + logf(sc);
  const float wn = (float)((double)a.w[b] / *a.wsum);
  atomicAdd(a.loss, -(double)wn * (double)lq);
  for (int c = 0; c < C; ++c) {
    const float gam = expf(lc[c] - lq);
    const float pi = expf(o[c] - lse_a);
    g[c] = wn * (pi - gam);
    for (int d = 0; d < d2; ++d) {
      const float mu = o[C + c * d2 + d];
      const float raw = o[C + C * d2 + c * d2 + d];
      const float ls = fminf(fmaxf(raw, kLogSigMin), kLogSigMax);
      const float is = expf(-ls);
      const float u = (z[d] - mu) * is;
      g[C + c * d2 + d] = -wn * gam * u * is;
      const bool inside = raw > kLogSigMin && raw < kLogSigMax;
      g[C + C * d2 + c * d2 + d] = inside ? -wn * gam * (u * u - 1.f) : 0.f;
    }
  }
}

// Affine (outer-amortised) head: out = (raw log s, c); Z row = (z, mu, m) (3 d2);
// zhat = m + (z - m - c) / s; -log q = 1/2 (zhat - mu)^T Q^-1 (zhat - mu) + sum log s + const.
struct AffineArgs {
  const float* out;
  const float* Z;
  const float* w;
  const double* wsum;
  float* dout;
  double* loss;
  int n, d2;
  const float* qinv;  // d2 x d2, row-major (device)
  float half_logdet;
};

__global__ void head_affine_kernel(AffineArgs a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.n) return;
  const int d2 = a.d2;
  const float* o = a.out + (long long)b * 2 * d2;
  const float* zr = a.Z + (long long)b * 3 * d2;
  float* g = a.dout + (long long)b * 2 * d2;
  float r[kMaxD2Amortised], u[kMaxD2Amortised], ls[kMaxD2Amortised];
  float sum_ls = 0.f;
  for (int d = 0; d < d2; ++d) {
    ls[d] = fminf(fmaxf(o[d], kLogSigMin), kLogSigMax);
    u[d] = zr[d] - zr[2 * d2 + d] - o[d2 + d];  // z - m - c
    const float zhat = zr[2 * d2 + d] + u[d] * expf(-ls[d]);
    r[d] = zhat - zr[d2 + d];
    sum_ls += ls[d];
  }
  float quad = 0.f;
  float gz[kMaxD2Amortised];
  for (int d = 0; d < d2; ++d) {
    float v = 0.f;
    for (int e = 0; e < d2; ++e) v += a.qinv[d * d2 + e] * r[e];
    gz[d] = v;
    quad += r[d] * v;
  }
  const float wn = (float)((double)a.w[b] / *a.wsum);
  atomicAdd(a.loss, (double)wn * (0.5 * (double)quad + (double)sum_ls + (double)a.half_logdet));
  for (int d = 0; d < d2; ++d) {
    const float is = expf(-ls[d]);
    const bool inside = o[d] > kLogSigMin && o[d] < kLogSigMax;
    g[d] = inside ? wn * (-gz[d] * u[d] * is + 1.f) : 0.f;
    g[d2 + d] = -wn * gz[d] * is;
  }
}

__global__ void wsum_kernel(const float* w, int n, double* out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < n; b += 256) s += (double)w[b];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// db[n] = sum_b d[b][n] (rows in order)
__global__ void colsum_kernel(const float* d, int rows, int cols, float* db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= cols) return;
  float s = 0.f;
  for (int b = 0; b < rows; ++b) s += d[(long long)b * cols + n];
  db[n] = s;
}

__global__ void round_rows_kernel(const float* src, float* dst, long long n, int round) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < n) dst[e] = round ? round_bf16(src[e]) : src[e];
}

// minibatch gather: rows perm[b] of F, Z, w
__global__ void gather_rows_kernel(const float* F, const float* Z, const float* w, const int64_t* perm,
                                   int nb, int din, int d2, float* Fb, float* Zb, float* wb, int round) {
  const int b = blockIdx.x;
  if (b >= nb) return;
  const long long r = perm[b];
  for (int c = threadIdx.x; c < din; c += blockDim.x) {
    const float v = F[r * din + c];
    Fb[(long long)b * din + c] = round ? round_bf16(v) : v;
  }
  for (int c = threadIdx.x; c < d2; c += blockDim.x) Zb[(long long)b * d2 + c] = Z[r * d2 + c];  // d2: row width
  if (threadIdx.x == 0) wb[b] = w[r];
}

struct AdamArgs {
  float* W;
  float* Wq;  // the weights the forward pass uses (bfloat16-rounded weight matrices)
  float* m;
  float* v;
  const float* g;
  long long n;
  long long wend[kLayers];  // [wbeg[l], wend[l]) is weight matrix l
  long long wbeg[kLayers];
  float lr, b1, b2, eps, c1, c2;  // c1 = 1 - b1^t, c2 = 1 - b2^t
  int round;
};

__global__ void adam_kernel(AdamArgs a) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= a.n) return;
  const float g = a.g[e];
  const float m = a.b1 * a.m[e] + (1.f - a.b1) * g;
  const float v = a.b2 * a.v[e] + (1.f - a.b2) * g * g;
  a.m[e] = m;
  a.v[e] = v;
  const float mh = m / a.c1, vh = v / a.c2;
  const float w = a.W[e] - a.lr * mh / (sqrtf(vh) + a.eps);
  a.W[e] = w;
  bool is_w = false;
  for (int l = 0; l < kLayers; ++l) is_w |= (e >= a.wbeg[l] && e < a.wend[l]);
  a.Wq[e] = (is_w && a.round) ? round_bf16(w) : w;
}

__global__ void quantize_params_kernel(const float* W, float* Wq, long long n, AdamArgs seg) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  bool is_w = false;
  for (int l = 0; l < kLayers; ++l) is_w |= (e >= seg.wbeg[l] && e < seg.wend[l]);
  Wq[e] = (is_w && seg.round) ? round_bf16(W[e]) : W[e];
}

// ---- host side ----
static dpf_status palloc(dpf_proposal& p, void** ptr, size_t bytes) {
  cudaError_t e = device_malloc(ptr, bytes < 16 ? 16 : bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return set_error(DPF_E_NOMEM, "proposal: device allocation failed");
  }
  p.allocs.push_back(*ptr);
  return DPF_OK;
}

int dpf_proposal_dout(const dpf_proposal* p) { return p->dout; }
int dpf_proposal_kind(const dpf_proposal* p) { return p->kind; }

static AdamArgs segments(const dpf_proposal& p) {
  AdamArgs a{};
  for (int l = 0; l < kLayers; ++l) {
    a.wbeg[l] = p.offW[l];
    a.wend[l] = p.offW[l] + (long long)p.rows[l] * p.cols[l];
  }
  a.round = p.bf16 ? 1 : 0;
  return a;
}

dpf_status proposal_requantize(dpf_proposal& p) {
  AdamArgs seg = segments(p);
  quantize_params_kernel<<<(unsigned)((p.nparams + 255) / 256), 256, 0, p.stream>>>(p.W, p.Wq, p.nparams, seg);
  p.packed_valid = false;
  return cuda_error(cudaGetLastError(), "proposal quantize");
}

// Ensure the per-minibatch workspace holds nb rows.
static dpf_status workspace(dpf_proposal& p, int nb) {
  if (nb <= p.ws_rows) return DPF_OK;
  const size_t H = p.hidden;
  auto take = [&](float** q, size_t n) { return palloc(p, (void**)q, sizeof(float) * n); };
  if (take(&p.Fb, (size_t)nb * p.din) || take(&p.Zb, (size_t)nb * p.zw) || take(&p.wb, nb) ||
      take(&p.h1, nb * H) || take(&p.h2, nb * H) || take(&p.h3, nb * H) || take(&p.ob, (size_t)nb * p.dout) ||
      take(&p.dA, nb * H) || take(&p.dB, nb * H) || take(&p.dO, (size_t)nb * p.dout) ||
      palloc(p, (void**)&p.perm_d, sizeof(int64_t) * nb))
    return DPF_E_NOMEM;
  p.ws_rows = nb;
  return DPF_OK;
}

// Forward and backward over the nb rows already in Fb/Zb/wb: loss into *loss_dev
// (accumulated), gradients into grad (nparams floats).
static dpf_status fwd_bwd(dpf_proposal& p, int nb, double* loss_dev, float* grad) {
  cudaStream_t s = p.stream;
  const int H = p.hidden, din = p.din, dO = p.dout;
  const float* Wq = p.Wq;
  const int rd = p.bf16 ? 1 : 0;
  const float *W1 = Wq + p.offW[0], *W2 = Wq + p.offW[1], *W3 = Wq + p.offW[2], *W4 = Wq + p.offW[3];
  const float *b1 = Wq + p.offB[0], *b2 = Wq + p.offB[1], *b3 = Wq + p.offB[2], *b4 = Wq + p.offB[3];
  // forward: h_l = round(relu(h_{l-1} W_l^T + b_l)), out = h3 W4^T + b4
  tgemm<false, true, 1>(s, p.bf16 ? 1 : 0, p.err_d, nb, H, din, p.Fb, din, W1, din, p.h1, H, b1, nullptr, rd);
  tgemm<false, true, 1>(s, p.bf16 ? 1 : 0, p.err_d, nb, H, H, p.h1, H, W2, H, p.h2, H, b2, nullptr, rd);
  tgemm<false, true, 1>(s, p.bf16 ? 1 : 0, p.err_d, nb, H, H, p.h2, H, W3, H, p.h3, H, b3, nullptr, rd);
  tgemm<false, true, 2>(s, p.bf16 ? 1 : 0, p.err_d, nb, dO, H, p.h3, H, W4, H, p.ob, dO, b4);
  wsum_kernel<<<1, 256, 0, s>>>(p.wb, nb, p.wsum_d);
  if (p.kind == 0) {
    HeadArgs ha{p.ob, p.Zb, p.wb, p.wsum_d, p.dO, loss_dev, nb, p.d2, p.C, dO};
    head_loss_kernel<<<(nb + 127) / 128, 128, 0, s>>>(ha);
  } else {
    AffineArgs aa{};
    aa.out = p.ob; aa.Z = p.Zb; aa.w = p.wb; aa.wsum = p.wsum_d; aa.dout = p.dO; aa.loss = loss_dev;
    aa.n = nb; aa.d2 = p.d2;
    aa.qinv = p.qinv_d;
    aa.half_logdet = p.half_logdet;
    head_affine_kernel<<<(nb + 127) / 128, 128, 0, s>>>(aa);
  }
  if (!grad) return cuda_error(cudaGetLastError(), "proposal forward");
  float *gW1 = grad + p.offW[0], *gW2 = grad + p.offW[1], *gW3 = grad + p.offW[2], *gW4 = grad + p.offW[3];
  float *gb1 = grad + p.offB[0], *gb2 = grad + p.offB[1], *gb3 = grad + p.offB[2], *gb4 = grad + p.offB[3];
  // layer 4: dW4 = dO^T h3, db4 = colsum dO, d3 = (dO W4) * (h3 > 0)
  tgemm<true, false, 0>(s, p.bf16 ? 1 : 0, p.err_d, dO, H, nb, p.dO, dO, p.h3, H, gW4, H);
  colsum_kernel<<<(dO + 127) / 128, 128, 0, s>>>(p.dO, nb, dO, gb4);
  tgemm<false, false, 3>(s, p.bf16 ? 1 : 0, p.err_d, nb, H, dO, p.dO, dO, W4, H, p.dA, H, nullptr, p.h3);
  // layer 3
  tgemm<true, false, 0>(s, p.bf16 ? 1 : 0, p.err_d, H, H, nb, p.dA, H, p.h2, H, gW3, H);
  colsum_kernel<<<(H + 127) / 128, 128, 0, s>>>(p.dA, nb, H, gb3);
  tgemm<false, false, 3>(s, p.bf16 ? 1 : 0, p.err_d, nb, H, H, p.dA, H, W3, H, p.dB, H, nullptr, p.h2);
  // layer 2
  tgemm<true, false, 0>(s, p.bf16 ? 1 : 0, p.err_d, H, H, nb, p.dB, H, p.h1, H, gW2, H);
  colsum_kernel<<<(H + 127) / 128, 128, 0, s>>>(p.dB, nb, H, gb2);
  tgemm<false, false, 3>(s, p.bf16 ? 1 : 0, p.err_d, nb, H, H, p.dB, H, W2, H, p.dA, H, nullptr, p.h1);
  // layer 1
  tgemm<true, false, 0>(s, p.bf16 ? 1 : 0, p.err_d, H, din, nb, p.dA, H, p.Fb, din, gW1, din);
  colsum_kernel<<<(H + 127) / 128, 128, 0, s>>>(p.dA, nb, H, gb1);
  return cuda_error(cudaGetLastError(), "proposal backward");
}

dpf_status proposal_forward_rows(dpf_proposal& p, const float* F, long long n, float* hidden, float* out, int* err,
                                 cudaStream_t s) {
  if (n < 1) return DPF_OK;
  if (n > (1LL << 30)) return set_error(DPF_E_INVALID, "proposal forward: too many rows");
  const int H = p.hidden, din = p.din, dO = p.dout, m = (int)n;
  const int pb = p.bf16 ? 1 : 0;
  const float* Wq = p.Wq;
  float* ha = hidden;
  float* hb = hidden + (size_t)n * H;
  tgemm<false, true, 1>(s, pb, err, m, H, din, F, din, Wq + p.offW[0], din, ha, H, Wq + p.offB[0], nullptr, pb);
  tgemm<false, true, 1>(s, pb, err, m, H, H, ha, H, Wq + p.offW[1], H, hb, H, Wq + p.offB[1], nullptr, pb);
  tgemm<false, true, 1>(s, pb, err, m, H, H, hb, H, Wq + p.offW[2], H, ha, H, Wq + p.offB[2], nullptr, pb);
  tgemm<false, true, 2>(s, pb, err, m, dO, H, ha, H, Wq + p.offW[3], H, out, dO, Wq + p.offB[3]);
  return cuda_error(cudaGetLastError(), "proposal forward");
}

static dpf_status adam(dpf_proposal& p, const float* grad, float lr) {
  p.adam_t += 1;
  AdamArgs a = segments(p);
  a.W = p.W;
  a.Wq = p.Wq;
  a.m = p.am;
  a.v = p.av;
  a.g = grad;
  a.n = p.nparams;
  a.lr = lr;
  a.b1 = 0.9f;
  a.b2 = 0.999f;
  a.eps = 1e-8f;
  a.c1 = (float)(1.0 - std::pow(0.9, (double)p.adam_t));
  a.c2 = (float)(1.0 - std::pow(0.999, (double)p.adam_t));
  adam_kernel<<<(unsigned)((p.nparams + 255) / 256), 256, 0, p.stream>>>(a);
  p.packed_valid = false;
  return cuda_error(cudaGetLastError(), "adam");
}

// splitmix64 (Steele, Lea and Flood 2014): the minibatch order of training.
static uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static dpf_status proposal_make(int kind, int32_t d1, int32_t d2, int32_t dy, int32_t hidden, int32_t components,
                                int din, int dout, int zw, void* stream, dpf_proposal** out) {
  const int max_din = kind == 1 ? kMaxDinAmortised : kMaxDin;
  const int max_d2 = kind == 1 ? kMaxD2Amortised : kMaxD2;
  if (d1 < 1 || d2 < 1 || dy < 1 || din > max_din || d2 > max_d2 || hidden < 16 || hidden > kMaxHidden ||
      hidden % 16 || components < 1 || components > kMaxComponents || dout > kMaxDout)
    return set_error(DPF_E_INVALID, "dpf_proposal_create: unsupported sizes (mixture: din <= 16, d2 <= 8; "
                                    "amortised: din <= 160, d2 <= 64; hidden a multiple of 16 up to 256, "
                                    "components 1..8, head <= 128)");
  dpf_proposal* p = new dpf_proposal();
  p->kind = kind;
  p->d1 = d1;
  p->d2 = d2;
  p->dy = dy;
  p->din = din;
  p->hidden = hidden;
  p->C = components;
  p->dout = dout;
  p->zw = zw;
  p->stream = (cudaStream_t)stream;
  const int H = hidden;
  p->rows[0] = H; p->cols[0] = din;
  p->rows[1] = H; p->cols[1] = H;
  p->rows[2] = H; p->cols[2] = H;
  p->rows[3] = p->dout; p->cols[3] = H;
  long long o = 0;
  for (int l = 0; l < kLayers; ++l) {
    p->offW[l] = o;
    o += (long long)p->rows[l] * p->cols[l];
    p->offB[l] = o;
    o += p->rows[l];
  }
  p->nparams = o;
  const size_t bytes = sizeof(float) * (size_t)o;
  if (palloc(*p, (void**)&p->W, bytes) || palloc(*p, (void**)&p->Wq, bytes) ||
      palloc(*p, (void**)&p->am, bytes) || palloc(*p, (void**)&p->av, bytes) ||
      palloc(*p, (void**)&p->grad, bytes) || palloc(*p, (void**)&p->loss_d, sizeof(double)) ||
      palloc(*p, (void**)&p->wsum_d, sizeof(double)) || palloc(*p, (void**)&p->err_d, sizeof(int))) {
    dpf_proposal_destroy(p);
    return DPF_E_NOMEM;
  }
  cudaMemsetAsync(p->err_d, 0, sizeof(int), p->stream);
  cudaMemsetAsync(p->W, 0, bytes, p->stream);
  cudaMemsetAsync(p->Wq, 0, bytes, p->stream);
  cudaMemsetAsync(p->am, 0, bytes, p->stream);
  cudaMemsetAsync(p->av, 0, bytes, p->stream);
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) {
    dpf_proposal_destroy(p);
    return cuda_error(e, "dpf_proposal_create");
  }
  *out = p;
  return DPF_OK;
}

}  // namespace dpf

using namespace dpf;

extern "C" {

dpf_status dpf_proposal_create(int32_t d1, int32_t d2, int32_t dy, int32_t hidden, int32_t components,
                               void* stream, dpf_proposal** out) {
  clear_error();
  if (!out) return set_error(DPF_E_INVALID, "dpf_proposal_create: null output");
  *out = nullptr;
  return dpf::proposal_make(0, d1, d2, dy, hidden, components, 2 * d1 + d2 + dy, components * (1 + 2 * d2), d2,
                            stream, out);
}

dpf_status dpf_proposal_create_amortised(int32_t d1, int32_t d2, int32_t dy, int32_t hidden, const double* Qz,
                                         void* stream, dpf_proposal** out) {
  clear_error();
  if (!out || !Qz) return set_error(DPF_E_INVALID, "dpf_proposal_create_amortised: null argument");
  *out = nullptr;
  if (d2 < 1 || d2 > kMaxD2Amortised)
    return set_error(DPF_E_INVALID, "dpf_proposal_create_amortised: d2 in 1..64");
  // Q_z^-1 and log det(2 pi Q_z) by a Cholesky factorisation on the host
  std::vector<double> Lc(d2 * d2, 0.0), inv(d2 * d2, 0.0);
  for (int r = 0; r < d2; ++r)
    for (int c = 0; c <= r; ++c) {
      double v = Qz[r * d2 + c];
      for (int k = 0; k < c; ++k) v -= Lc[r * d2 + k] * Lc[c * d2 + k];
      if (r == c) {
        if (!(v > 0)) return set_error(DPF_E_INVALID, "dpf_proposal_create_amortised: Q_z not positive definite");
        Lc[r * d2 + r] = std::sqrt(v);
      } else {
        Lc[r * d2 + c] = v / Lc[c * d2 + c];
      }
    }
  double logdet = 0.0;
  for (int r = 0; r < d2; ++r) logdet += 2.0 * std::log(Lc[r * d2 + r]);
  for (int col = 0; col < d2; ++col) {  // solve Q x = e_col
    std::vector<double> yv(d2), xv(d2);
    for (int r = 0; r < d2; ++r) {
      double v = (r == col) ? 1.0 : 0.0;
      for (int k = 0; k < r; ++k) v -= Lc[r * d2 + k] * yv[k];
      yv[r] = v / Lc[r * d2 + r];
    }
    for (int r = d2 - 1; r >= 0; --r) {
      double v = yv[r];
      for (int k = r + 1; k < d2; ++k) v -= Lc[k * d2 + r] * xv[k];
      xv[r] = v / Lc[r * d2 + r];
    }
    for (int r = 0; r < d2; ++r) inv[r * d2 + col] = xv[r];
  }
  dpf_status st = dpf::proposal_make(1, d1, d2, dy, hidden, 1, 2 * d1 + dy + 2 * d2, 2 * d2, 3 * d2, stream, out);
  if (st) return st;
  for (int q = 0; q < d2 * d2; ++q) (*out)->qinv[q] = (float)inv[q];
  dpf_proposal* p = *out;
  cudaError_t e = cudaErrorMemoryAllocation;
  if (palloc(*p, (void**)&p->qinv_d, sizeof(float) * (size_t)d2 * d2) == DPF_OK)
    e = cudaMemcpyAsync(p->qinv_d, p->qinv, sizeof(float) * (size_t)d2 * d2, cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) {
    dpf_proposal_destroy(p);
    *out = nullptr;
    return e == cudaErrorMemoryAllocation ? DPF_E_NOMEM : cuda_error(e, "dpf_proposal_create_amortised");
  }
  (*out)->half_logdet = (float)(0.5 * (logdet + d2 * std::log(2.0 * M_PI)));
  return DPF_OK;
}

dpf_status dpf_proposal_set_centre(dpf_proposal* p, int32_t per_particle) {
  clear_error();
  if (!p || p->kind != 1 || (per_particle != 0 && per_particle != 1))
    return set_error(DPF_E_INVALID, "dpf_proposal_set_centre: an outer-amortised proposal and 0 or 1");
  p->centre = per_particle;
  return DPF_OK;
}

dpf_status dpf_proposal_num_params(const dpf_proposal* p, int64_t* n) {
  clear_error();
  if (!p || !n) return set_error(DPF_E_INVALID, "dpf_proposal_num_params: null argument");
  *n = p->nparams;
  return DPF_OK;
}

dpf_status dpf_proposal_set_bf16(dpf_proposal* p, int32_t enable) {
  clear_error();
  if (!p) return set_error(DPF_E_INVALID, "dpf_proposal_set_bf16: null proposal");
  p->bf16 = enable != 0;
  dpf_status st = proposal_requantize(*p);
  if (st) return st;
  return cuda_error(cudaStreamSynchronize(p->stream), "dpf_proposal_set_bf16");
}

dpf_status dpf_proposal_set_weights(dpf_proposal* p, const float* params, int64_t n) {
  clear_error();
  if (!p || !params || n != p->nparams)
    return set_error(DPF_E_INVALID, "dpf_proposal_set_weights: need exactly num_params floats");
  cudaError_t e = cudaMemcpyAsync(p->W, params, sizeof(float) * n, cudaMemcpyHostToDevice, p->stream);
  if (e != cudaSuccess) return cuda_error(e, "dpf_proposal_set_weights");
  cudaMemsetAsync(p->am, 0, sizeof(float) * n, p->stream);
  cudaMemsetAsync(p->av, 0, sizeof(float) * n, p->stream);
  p->adam_t = 0;
  dpf_status st = proposal_requantize(*p);
  if (st) return st;
  return cuda_error(cudaStreamSynchronize(p->stream), "dpf_proposal_set_weights");
}

dpf_status dpf_proposal_get_weights(const dpf_proposal* p, float* params, int64_t n) {
  clear_error();
  if (!p || !params || n != p->nparams)
    return set_error(DPF_E_INVALID, "dpf_proposal_get_weights: need exactly num_params floats");
  cudaError_t e = cudaMemcpyAsync(params, p->W, sizeof(float) * n, cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  return cuda_error(e, "dpf_proposal_get_weights");
}

// The training products' error word: DPF_E_TIMEOUT (and cleared) if a wait gave up.
static dpf_status training_err(dpf_proposal& p, const char* what) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, p.err_d, sizeof(int), cudaMemcpyDeviceToHost, p.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p.stream);
  if (e != cudaSuccess) return cuda_error(e, what);
  if (h) {
    cudaMemsetAsync(p.err_d, 0, sizeof(int), p.stream);
    return set_error(DPF_E_TIMEOUT, std::string(what) + ": a tensor-core product did not complete in time");
  }
  return DPF_OK;
}

dpf_status dpf_proposal_loss_grad(dpf_proposal* p, const float* F, const float* Z, const float* w, int64_t n,
                                  double* loss, float* grad_dev) {
  clear_error();
  if (!p || !F || !Z || !w || n < 1 || n > (1 << 24))
    return set_error(DPF_E_INVALID, "dpf_proposal_loss_grad: bad arguments");
  dpf_status st = workspace(*p, (int)n);
  if (st) return st;
  cudaStream_t s = p->stream;
  const int rd = p->bf16 ? 1 : 0;
  round_rows_kernel<<<(unsigned)((n * p->din + 255) / 256), 256, 0, s>>>(F, p->Fb, n * p->din, rd);
  cudaMemcpyAsync(p->Zb, Z, sizeof(float) * n * p->zw, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(p->wb, w, sizeof(float) * n, cudaMemcpyDeviceToDevice, s);
  cudaMemsetAsync(p->loss_d, 0, sizeof(double), s);
  st = fwd_bwd(*p, (int)n, p->loss_d, grad_dev);
  if (st) return st;
  double h = 0.0;
  cudaError_t e = cudaMemcpyAsync(&h, p->loss_d, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_error(e, "dpf_proposal_loss_grad");
  st = training_err(*p, "dpf_proposal_loss_grad");
  if (st) return st;
  if (loss) *loss = h;
  return DPF_OK;
}

dpf_status dpf_proposal_adam_step(dpf_proposal* p, const float* grad_dev, float lr) {
  clear_error();
  if (!p || !grad_dev || !(lr > 0.f)) return set_error(DPF_E_INVALID, "dpf_proposal_adam_step: bad arguments");
  dpf_status st = adam(*p, grad_dev, lr);
  if (st) return st;
  return cuda_error(cudaStreamSynchronize(p->stream), "dpf_proposal_adam_step");
}

dpf_status dpf_proposal_train(dpf_proposal* p, const float* F, const float* Z, const float* w, int64_t n,
                              int32_t batch, int32_t epochs, float lr, uint64_t seed, double* losses) {
  clear_error();
  if (!p || !F || !Z || !w || n < 1 || batch < 1 || batch > (1 << 16) || epochs < 1 || !(lr > 0.f))
    return set_error(DPF_E_INVALID, "dpf_proposal_train: bad arguments");
  const int nb_max = (int)std::min<int64_t>(batch, n);
  dpf_status st = workspace(*p, nb_max);
  if (st) return st;
  cudaStream_t s = p->stream;
  const int rd = p->bf16 ? 1 : 0;
  std::vector<int64_t> perm(n);
  for (int64_t i = 0; i < n; ++i) perm[i] = i;
  uint64_t rs = seed;
  int64_t* perm_dev = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&perm_dev, sizeof(int64_t) * n, s);
  if (e != cudaSuccess) return cuda_error(e, "dpf_proposal_train: allocation");
  std::vector<double> ep_loss(epochs, 0.0);
  double* eloss_d = nullptr;
  e = cudaMallocAsync((void**)&eloss_d, sizeof(double) * epochs, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(perm_dev, s);
    return cuda_error(e, "dpf_proposal_train: allocation");
  }
  cudaMemsetAsync(eloss_d, 0, sizeof(double) * epochs, s);
  const int64_t nbatches = (n + nb_max - 1) / nb_max;
  for (int ep = 0; ep < epochs && !st; ++ep) {
    for (int64_t i = n - 1; i > 0; --i) {  // Fisher-Yates with splitmix64
      const int64_t j = (int64_t)(splitmix64(rs) % (uint64_t)(i + 1));
      std::swap(perm[i], perm[j]);
    }
    e = cudaMemcpyAsync(perm_dev, perm.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // perm is rewritten next epoch
    if (e != cudaSuccess) {
      st = cuda_error(e, "dpf_proposal_train: permutation");
      break;
    }
    for (int64_t bi = 0; bi < nbatches && !st; ++bi) {
      const int64_t b0 = bi * nb_max;
      const int nb = (int)std::min<int64_t>(nb_max, n - b0);
      gather_rows_kernel<<<nb, 32, 0, s>>>(F, Z, w, perm_dev + b0, nb, p->din, p->zw, p->Fb, p->Zb, p->wb, rd);
      st = fwd_bwd(*p, nb, eloss_d + ep, p->grad);
      if (!st) st = adam(*p, p->grad, lr);
    }
  }
  if (!st) {
    e = cudaMemcpyAsync(ep_loss.data(), eloss_d, sizeof(double) * epochs, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_error(e, "dpf_proposal_train");
  }
  cudaFreeAsync(perm_dev, s);
  cudaFreeAsync(eloss_d, s);
  if (!st) st = training_err(*p, "dpf_proposal_train");
  if (!st && losses)
    for (int ep = 0; ep < epochs; ++ep) losses[ep] = ep_loss[ep] / (double)nbatches;
  return st;
}

void dpf_proposal_destroy(dpf_proposal* p) {
  if (!p) return;
  if (p->stream) cudaStreamSynchronize(p->stream);
  for (void* q : p->allocs) cudaFree(q);
  delete p;
}

}  // extern "C"
