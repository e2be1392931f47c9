// The learned proposal on the tensor cores: the MLP forward pass of 128-row tiles
// (tcgen05 kind::f16 with BF16 operands, FP32 accumulators in TMEM), used alone
// (dpf_proposal_forward) and as the inner update of the filter step (selection,
// local resampling and feature rows before it; the mixture draw and the importance
// weights after it), plus the recording of training rows.
//
// Per tile, one thread per row: layer 1 (K = 16 padded inputs) and the head
// (N = 32 padded outputs) have their weights resident in shared memory; the two
// 256 x 256 layers stream their weights through a three-stage ring of 16 KB
// chunks (32 K-columns each) copied by cp.async.bulk from a packed copy in global
// memory, so the copy of the next chunks overlaps the MMAs of the current ones.
// Every hidden layer's accumulator (128 x 256 FP32, TMEM columns 0..255) is read
// back row by row, biased, passed through ReLU, rounded to BF16 and written as
// the next layer's A operand (K-major, no swizzle). All waits are bounded.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "dpf_learned.h"
#include "dpf_tc.cuh"
#include "dpf_variant.cuh"

namespace dpf {

constexpr int LH = 256;                // hidden width of the tensor-core pass
constexpr int LDIN = 16;               // inputs padded to one K step
constexpr int LNP = 32;                // head outputs padded to an MMA N
constexpr int LKCH = 32;               // K columns per streamed chunk
constexpr int LNCH = LH / LKCH;        // chunks per hidden layer
constexpr int LSTAGES = 3;
constexpr uint32_t LCHUNK = LH * LKCH * 2;  // bytes of one chunk
constexpr int L_SPIN = 1 << 22;
constexpr uint32_t LTMEM_COLS = 512;
constexpr int kFilterComponents = 4;  // mixture components of the filter's compiled pass

// packed global layout (bytes)
constexpr size_t PK_W1 = 0;
constexpr size_t PK_W2 = PK_W1 + (size_t)LH * LDIN * 2;
constexpr size_t PK_W3 = PK_W2 + (size_t)LNCH * LCHUNK;
constexpr size_t PK_W4 = PK_W3 + (size_t)LNCH * LCHUNK;
constexpr size_t PK_B = PK_W4 + (size_t)LNP * LH * 2;
constexpr size_t PK_BYTES = PK_B + sizeof(float) * (3 * LH + LNP);

// One iteration of the kernel takes 2 x 128 rows (tiles A and B, TMEM columns 0..255 and
// 256..511); 8 compute warps hold one row a thread, a ninth warp feeds the weight ring.
constexpr int LROWS = 256;
constexpr int LCOMPUTE = 256;                               // compute threads
constexpr int LTHREADS = LCOMPUTE + 32;                     // + the producer warp
// shared-memory layout (bytes)
constexpr uint32_t SM_ACT = 0;                              // 2 x (128 x 256 bf16), kc16 = 32
constexpr uint32_t SM_IN = SM_ACT + 2 * 128 * LH * 2;       // 2 x (128 x 16 bf16), kc16 = 2
constexpr uint32_t SM_W1 = SM_IN + 2 * 128 * LDIN * 2;      // 256 x 16, kc16 = 2
constexpr uint32_t SM_W4 = SM_W1 + LH * LDIN * 2;           // 32 x 256, kc16 = 32
constexpr uint32_t SM_RING = SM_W4 + LNP * LH * 2;          // 3 x (256 x 32), kc16 = 4
constexpr uint32_t SM_BIAS = SM_RING + LSTAGES * LCHUNK;    // b1 b2 b3 (256 each), b4 (32)
constexpr uint32_t SM_CUM = SM_BIAS + sizeof(float) * (3 * LH + LNP);  // 256 uint32
constexpr uint32_t SM_RED = SM_CUM + LROWS * 4;             // 8 floats, 8 words
constexpr uint32_t SM_BYTES = SM_RED + 64;
static_assert(SM_BYTES <= 227 * 1024, "shared memory of the learned kernel");

// Barrier of the 256 compute threads only (the producer warp runs its own loop).
__device__ __forceinline__ void compute_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Pack one FP32 matrix (rows x cols, row-major) into BF16 K-major chunks of kch
// columns, rows padded to rows_pad and columns to a multiple of kch with zeros.
__global__ void pack_matrix_kernel(const float* __restrict__ W, int rows, int cols, int rows_pad, int kch,
                                   int nchunks, unsigned char* __restrict__ dst) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)rows_pad * kch * nchunks;
  if (e >= total) return;
  const int n = (int)(e / ((long long)kch * nchunks));
  const int k = (int)(e % ((long long)kch * nchunks));
  const int ch = k / kch, kl = k % kch;
  const float v = (n < rows && k < cols) ? W[(long long)n * cols + k] : 0.f;
  const size_t off = (size_t)ch * rows_pad * kch * 2 + tc::kmajor_offset(n, 2 * kl, kch * 2 / 16);
  *(__nv_bfloat16*)(dst + off) = __float2bfloat16_rn(v);
}

__global__ void pack_bias_kernel(const float* __restrict__ b1, const float* __restrict__ b2,
                                 const float* __restrict__ b3, const float* __restrict__ b4, int dout,
                                 float* __restrict__ dst) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < 3 * LH) dst[e] = e < LH ? b1[e] : e < 2 * LH ? b2[e - LH] : b3[e - 2 * LH];
  else if (e < 3 * LH + LNP) dst[e] = (e - 3 * LH) < dout ? b4[e - 3 * LH] : 0.f;
}

static dpf_status pack(dpf_proposal& p) {
  if (p.packed_valid) return DPF_OK;
  if (!p.packed) {
    cudaError_t e = cudaMalloc(&p.packed, PK_BYTES);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p.packed = nullptr;
      return set_error(DPF_E_NOMEM, "proposal: packed weights");
    }
    p.allocs.push_back(p.packed);
    p.packed_bytes = PK_BYTES;
  }
  cudaStream_t s = p.stream;
  unsigned char* d = (unsigned char*)p.packed;
  const float* Wq = p.Wq;
  auto launch = [&](const float* W, int rows, int cols, int rows_pad, int kch, int nch, size_t off) {
    const long long total = (long long)rows_pad * kch * nch;
    pack_matrix_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(W, rows, cols, rows_pad, kch, nch, d + off);
  };
  launch(Wq + p.offW[0], LH, p.din, LH, LDIN, 1, PK_W1);
  launch(Wq + p.offW[1], LH, LH, LH, LKCH, LNCH, PK_W2);
  launch(Wq + p.offW[2], LH, LH, LH, LKCH, LNCH, PK_W3);
  launch(Wq + p.offW[3], p.dout, LH, LNP, LH, 1, PK_W4);
  pack_bias_kernel<<<(3 * LH + LNP + 255) / 256, 256, 0, s>>>(Wq + p.offB[0], Wq + p.offB[1], Wq + p.offB[2],
                                                               Wq + p.offB[3], p.dout, (float*)(d + PK_B));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "proposal pack");
  p.packed_valid = true;
  return DPF_OK;
}

struct LearnArgs {
  const unsigned char* wp;  // packed weights (PK_* layout)
  int din, dout, C;
  // forward-only mode
  const float* F;
  float* out;
  long long nrows;
  // filter mode
  float* dbg_head;  // N M x dout head outputs, or null
  uint32_t scaleC;  // 2^(31 - ceil log2 C)
  int* err;
};

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(a));
  const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(b));
  return lo | (hi << 16);
}

// Read one hidden accumulator row (256 FP32 columns of TMEM, 64 per load), add the
// bias, ReLU, round to BF16 and store it as row r of the activation tile.
__device__ __forceinline__ void hidden_epilogue(uint32_t taddr_row, const float* bias, unsigned char* act, int r) {
#pragma unroll 1
  for (int c0 = 0; c0 < LH; c0 += 64) {
    float v[64];
    tc::ld64(taddr_row + (uint32_t)c0, v);
#pragma unroll
    for (int h = 0; h < 64; h += 8) {
      uint4 q;
      q.x = pack_bf16x2(fmaxf(v[h + 0] + bias[c0 + h + 0], 0.f), fmaxf(v[h + 1] + bias[c0 + h + 1], 0.f));
      q.y = pack_bf16x2(fmaxf(v[h + 2] + bias[c0 + h + 2], 0.f), fmaxf(v[h + 3] + bias[c0 + h + 3], 0.f));
      q.z = pack_bf16x2(fmaxf(v[h + 4] + bias[c0 + h + 4], 0.f), fmaxf(v[h + 5] + bias[c0 + h + 5], 0.f));
      q.w = pack_bf16x2(fmaxf(v[h + 6] + bias[c0 + h + 6], 0.f), fmaxf(v[h + 7] + bias[c0 + h + 7], 0.f));
      *(uint4*)(act + tc::kmajor_offset(r, 2 * (c0 + h), 32)) = q;
    }
  }
}

// Group reductions over the M consecutive rows of a tile (M in {32, 64, 128}).
__device__ __forceinline__ float group_max(float v, int M, float* red) {
  v = warp_max(v);
  if (M <= 32) return v;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  compute_sync();
  if (lane == 0) red[w] = v;
  compute_sync();
  const int g0 = (w * 32 / M) * (M / 32);
  float m = red[g0];
  for (int q = 1; q < M / 32; ++q) m = fmaxf(m, red[g0 + q]);
  return m;
}
__device__ __forceinline__ float group_sum(float v, int M, float* red) {
  v = warp_sum(v);
  if (M <= 32) return v;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  compute_sync();
  if (lane == 0) red[w] = v;
  compute_sync();
  const int g0 = (w * 32 / M) * (M / 32);
  float s = 0.f;
  for (int q = 0; q < M / 32; ++q) s += red[g0 + q];
  return s;
}

// MODE 0: head outputs of feature rows; MODE 1: the filter's inner update with NC
// mixture components (compile-time, so that the head's arrays stay in registers).
template <int MODE, int D1, int D2, int DY, bool XZ, int NC>
__global__ void __launch_bounds__(LTHREADS, 1)
    learned_kernel(const __grid_constant__ MC<float, D1, D2, DY> mc, const __grid_constant__ StepArgs<float> a,
                   const __grid_constant__ LearnArgs la) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t full[LSTAGES], empty[LSTAGES], mbar;
  __shared__ uint32_t s_taddr;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int half = tid >> 7;  // tile A (0) or B (1) of this thread's row
  const int r128 = tid & 127;
  unsigned char* act = sm + SM_ACT + half * (128 * LH * 2);
  unsigned char* in = sm + SM_IN + half * (128 * LDIN * 2);
  float* bias = (float*)(sm + SM_BIAS);
  uint32_t* cum = (uint32_t*)(sm + SM_CUM);
  float* red = (float*)(sm + SM_RED);
  const float NEG = -INFINITY;

  const int M = MODE == 1 ? a.M : 128;
  const long long rows_total = MODE == 1 ? a.N * (long long)a.M : la.nrows;
  const long long niters = (rows_total + LROWS - 1) / LROWS;
  const long long my_iters = niters > blockIdx.x ? (niters - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long total_chunks = my_iters * 2 * LNCH;

  // ---- set-up: barriers, TMEM, resident weights and biases ----
  if (tid == 0) {
    for (int s = 0; s < LSTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&mbar, 1);
    mbar_fence_init();
  }
  if (w == 0) {
    tc::tmem_alloc(&s_taddr, LTMEM_COLS);
    tc::tmem_relinquish();
  }
  for (int e = tid; e < (int)(LH * LDIN * 2 / 16); e += LTHREADS)
    ((uint4*)(sm + SM_W1))[e] = ((const uint4*)(la.wp + PK_W1))[e];
  for (int e = tid; e < (int)(LNP * LH * 2 / 16); e += LTHREADS)
    ((uint4*)(sm + SM_W4))[e] = ((const uint4*)(la.wp + PK_W4))[e];
  for (int e = tid; e < 3 * LH + LNP; e += LTHREADS) bias[e] = ((const float*)(la.wp + PK_B))[e];
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = s_taddr;
  // this thread's accumulator row: lanes 32 (w % 4) .., columns 256 half ..
  const uint32_t trow = taddr + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(half * LH);
  bool ok = true;

  if (w == LCOMPUTE / 32) {
    // ---- producer warp: refill each ring stage as soon as its MMAs are done ----
    if (lane == 0) {
      for (long long c = 0; c < total_chunks; ++c) {
        const int s = (int)(c % LSTAGES);
        if (c >= LSTAGES && !tc::bar_wait(&empty[s], (uint32_t)(((c / LSTAGES) - 1) & 1), L_SPIN)) {
          ok = false;
          break;
        }
        const int q = (int)(c % (2 * LNCH));
        const unsigned char* src =
            la.wp + (q < LNCH ? PK_W2 + (size_t)q * LCHUNK : PK_W3 + (size_t)(q - LNCH) * LCHUNK);
        mbar_arrive_tx(&full[s], LCHUNK);
        bulk_load(sm + SM_RING + s * LCHUNK, src, LCHUNK, &full[s]);
      }
      // wait until the last chunks' MMAs have released their stages, so that no
      // copy is in flight when the kernel ends
      for (long long c = std::max<long long>(0, total_chunks - LSTAGES); c < total_chunks && ok; ++c)
        if (!tc::bar_wait(&empty[c % LSTAGES], (uint32_t)((c / LSTAGES) & 1), L_SPIN)) ok = false;
    }
  } else {
  long long c_use = 0;      // next chunk to consume (thread 0)
  uint32_t mph = 0;         // phase of mbar (compute threads)

  const uint32_t id_h = tc::instr_desc(tc::FMT_BF16, 128, LH);
  const uint32_t id_o = tc::instr_desc(tc::FMT_BF16, 128, LNP);

  for (long long it = blockIdx.x; it < niters; it += gridDim.x) {
    const long long row = it * LROWS + tid;
    const bool live = row < rows_total;
    // ---- prologue: this row's input features ----
    float feat[LDIN];
#pragma unroll
    for (int k = 0; k < LDIN; ++k) feat[k] = 0.f;
    // filter-mode registers
    long long g = 0;
    int j = 0, anc_g = 0;
    float xa[D1], xt[D1], zb[D2];
    if (MODE == 0) {
#pragma unroll
      for (int k = 0; k < LDIN; ++k)
        if (live && k < la.din) feat[k] = la.F[row * la.din + k];
    } else {
      g = row / M;
      j = (int)(row % M);
      const long long gg = live ? g : 0;
      anc_g = a.anc[gg];
      const long long NM = a.N * (long long)M;
      // selection of x_{t-1} among the ancestor's look-ahead draws (one SIR draw)
      const int L = a.L;
      int msel = 0;
      {
        const float l0 = lane < L ? a.lwh_old[(long long)anc_g * L + lane] : NEG;
        const float l1 = lane + 32 < L ? a.lwh_old[(long long)anc_g * L + lane + 32] : NEG;
        // every lane of a warp holds one group (M >= 32): the warp's lanes read that group
        const float mx = warp_max(fmaxf(l0, l1));
        const uint32_t c0 = lane < L ? (uint32_t)floorf(exp2f((l0 - mx) * 1.4426950408889634f) * a.scaleL) : 0u;
        const uint32_t c1 = lane + 32 < L ? (uint32_t)floorf(exp2f((l1 - mx) * 1.4426950408889634f) * a.scaleL) : 0u;
        uint32_t s0 = c0, s1 = c1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t n0 = __shfl_up_sync(FULL, s0, o), n1 = __shfl_up_sync(FULL, s1, o);
          if (lane >= o) {
            s0 += n0;
            s1 += n1;
          }
        }
        const uint32_t tot0 = __shfl_sync(FULL, s0, 31), tot1 = __shfl_sync(FULL, s1, 31);
        const uint64_t Cs = (uint64_t)tot0 + tot1;
        const uint32_t usel = philox(ctr(a.t - 1, (uint32_t)gg, P_SEL, 0u, 0u), a.key).x;
        const uint64_t rhs = (uint64_t)usel * Cs;
        const unsigned b0 = __ballot_sync(FULL, ((uint64_t)s0 << 32) > rhs);
        const unsigned b1 = __ballot_sync(FULL, ((uint64_t)(s1 + tot0) << 32) > rhs);
        msel = b0 ? __ffs(b0) - 1 : (b1 ? 32 + __ffs(b1) - 1 : L - 1);
        if ((Cs == 0 || msel >= L) && live && j == 0) atomicOr(a.err, ERR_NUMERIC);
        if (msel >= L) msel = L - 1;
      }
#pragma unroll
      for (int c = 0; c < D1; ++c) {
        xt[c] = a.xbb_old[((long long)anc_g * L + msel) * D1 + c];
        xa[c] = a.x_old[(long long)anc_g * a.xp + c];
      }
      if (live && j == 0) {
        a.sel[g] = msel;
        for (int c = 0; c < a.xp; ++c) a.x_new[g * a.xp + c] = c < D1 ? xt[c < D1 ? c : 0] : 0.f;
      }
      // local resampling of the ancestor's inner set by alpha = lq + log p(x_t | x_a, z)
      float al = a.lq_old[(long long)anc_g * M + j];
      if (XZ) {
        float mxa[D1], wres[D1];
        mu_x(mc, xa, a.gcos_prev, mxa);
#pragma unroll
        for (int r = 0; r < D1; ++r) {
          float v = 0.f;
#pragma unroll
          for (int c = 0; c <= r; ++c) v += mc.LqxInv[r][c] * (xt[c] - mxa[c]);
          wres[r] = v;
        }
        float q = 0.f;
#pragma unroll
        for (int r = 0; r < D1; ++r) {
          float v = wres[r];
#pragma unroll
          for (int c = 0; c < D2; ++c) v -= mc.WAxz[r][c] * a.z_old[c * NM + (long long)anc_g * M + j];
          q += v * v;
        }
        al -= 0.5f * q;
      }
      const float amax = group_max(al, M, red);
      const uint32_t cq = (uint32_t)floorf(exp2f((al - amax) * 1.4426950408889634f) * a.scaleM);
      uint32_t inc = cq;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t n = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += n;
      }
      compute_sync();
      if (lane == 31) ((uint32_t*)red)[8 + w] = inc;  // warp totals after the float slots
      compute_sync();
      const int gw0 = (w * 32 / M) * (M / 32);  // first warp of this group
      for (int q = gw0; q < w; ++q) inc += ((uint32_t*)red)[8 + q];
      cum[tid] = inc;
      compute_sync();
      const int gbase = (tid / M) * M;
      const uint32_t Cg = cum[gbase + M - 1];
      if (Cg == 0 && live && j == 0) atomicOr(a.err, ERR_NUMERIC);
      const uint32_t uin = philox(ctr(a.t - 1, (uint32_t)gg, P_INNER, 0u, 0u), a.key).x;
      const int b = sys_local_pick(cum + gbase, M, Cg, M, j, uin);
      if (a.dbg_b && live) a.dbg_b[g * M + j] = b;
#pragma unroll
      for (int c = 0; c < D2; ++c) zb[c] = a.z_old[c * NM + (long long)anc_g * M + b];
      if (live) {
#pragma unroll
        for (int c = 0; c < D1; ++c) {
          feat[c] = xa[c];
          feat[D1 + c] = xt[c];
        }
#pragma unroll
        for (int c = 0; c < D2; ++c) feat[2 * D1 + c] = zb[c];
#pragma unroll
        for (int q = 0; q < DY; ++q) feat[2 * D1 + D2 + q] = a.y_prev[q];
      }
    }
    {
      uint4 q0, q1;
      q0.x = pack_bf16x2(feat[0], feat[1]);
      q0.y = pack_bf16x2(feat[2], feat[3]);
      q0.z = pack_bf16x2(feat[4], feat[5]);
      q0.w = pack_bf16x2(feat[6], feat[7]);
      q1.x = pack_bf16x2(feat[8], feat[9]);
      q1.y = pack_bf16x2(feat[10], feat[11]);
      q1.z = pack_bf16x2(feat[12], feat[13]);
      q1.w = pack_bf16x2(feat[14], feat[15]);
      *(uint4*)(in + tc::kmajor_offset(r128, 0, 2)) = q0;
      *(uint4*)(in + tc::kmajor_offset(r128, 16, 2)) = q1;
    }
    tc::fence_proxy_async();
    tc::fence_before();
    compute_sync();

    const uint32_t s_act0 = smem_addr(sm + SM_ACT), s_in0 = smem_addr(sm + SM_IN);
    // ---- layer 1 (both tiles) ----
    if (tid == 0) {
      tc::fence_after();
      for (int h = 0; h < 2; ++h)
        tc::mma_f16(taddr + h * LH, tc::smem_desc(s_in0 + h * (128 * LDIN * 2), 2),
                    tc::smem_desc(smem_addr(sm + SM_W1), 2), id_h, 0u);
      tc::commit(&mbar);
    }
    ok &= tc::bar_wait(&mbar, mph, L_SPIN);
    mph ^= 1u;
    tc::fence_after();
    hidden_epilogue(trow, bias, act, r128);
    tc::fence_proxy_async();
    tc::fence_before();
    compute_sync();

    // ---- layers 2 and 3 (streamed weights) ----
#pragma unroll 1
    for (int layer = 0; layer < 2; ++layer) {
      if (tid == 0) {
        tc::fence_after();
        for (int k = 0; k < LNCH; ++k) {
          const long long c = c_use++;
          const int s = (int)(c % LSTAGES);
          if (!tc::bar_wait(&full[s], (uint32_t)((c / LSTAGES) & 1), L_SPIN)) ok = false;
          const uint32_t sb = smem_addr(sm + SM_RING + s * LCHUNK);
#pragma unroll
          for (int ks = 0; ks < LKCH / 16; ++ks)
#pragma unroll
            for (int h = 0; h < 2; ++h)
              tc::mma_f16(taddr + h * LH,
                          tc::smem_desc(s_act0 + h * (128 * LH * 2) + (uint32_t)(k * (LKCH / 8) + ks * 2) * 128u, 32),
                          tc::smem_desc(sb + (uint32_t)ks * 256u, LKCH / 8), id_h, (k > 0 || ks > 0) ? 1u : 0u);
          tc::commit(&empty[s]);  // the producer refills the stage once these MMAs are done
        }
        tc::commit(&mbar);
      }
      ok &= tc::bar_wait(&mbar, mph, L_SPIN);
      mph ^= 1u;
      tc::fence_after();
      hidden_epilogue(trow, bias + (layer + 1) * LH, act, r128);
      tc::fence_proxy_async();
      tc::fence_before();
      compute_sync();
    }

    // ---- head ----
    if (tid == 0) {
      tc::fence_after();
      const uint32_t sb = smem_addr(sm + SM_W4);
      // the head of tile h goes to its own columns 0..31 (read by its last hidden epilogue)
#pragma unroll
      for (int ks = 0; ks < LH / 16; ++ks)
#pragma unroll
        for (int h = 0; h < 2; ++h)
          tc::mma_f16(taddr + h * LH, tc::smem_desc(s_act0 + h * (128 * LH * 2) + (uint32_t)ks * 256u, 32),
                      tc::smem_desc(sb + (uint32_t)ks * 256u, 32), id_o, ks > 0 ? 1u : 0u);
      tc::commit(&mbar);
    }
    ok &= tc::bar_wait(&mbar, mph, L_SPIN);
    mph ^= 1u;
    tc::fence_after();
    float o[LNP];
    {
      float v[16];
      tc::ld16(trow, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) o[q] = v[q] + bias[3 * LH + q];
      tc::ld16(trow + 16, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) o[16 + q] = v[q] + bias[3 * LH + 16 + q];
    }
    tc::fence_before();

    if (MODE == 0) {
#pragma unroll
      for (int q = 0; q < LNP; ++q)
        if (live && q < la.dout) la.out[row * la.dout + q] = o[q];
    } else {
      // ---- the mixture draw and the importance weight ----
      constexpr int C = NC;
      constexpr int DO = NC * (1 + 2 * D2);
      if (la.dbg_head && live) {
#pragma unroll
        for (int q = 0; q < DO; ++q) la.dbg_head[row * DO + q] = o[q];
      }
      float lmax = NEG;
#pragma unroll
      for (int c = 0; c < C; ++c) lmax = fmaxf(lmax, o[c]);
      float se = 0.f;
#pragma unroll
      for (int c = 0; c < C; ++c) se += expf(o[c] - lmax);
      const float lse_a = lmax + logf(se);
      // component: one-draw systematic pick over exp(logit - max), quantised
      uint32_t cumc[C];
      uint32_t run = 0;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        run += (uint32_t)floorf(exp2f((o[c] - lmax) * 1.4426950408889634f) * (float)la.scaleC);
        cumc[c] = run;
      }
      const uint32_t uc = philox(ctr(a.t - 1, (uint32_t)g, P_LCOMP, (uint32_t)j, 0u), a.key).x;
      const uint64_t rhs = (uint64_t)uc * run;
      // the first component whose cumulative count passes the draw (unrolled select)
      int comp = C - 1;
#pragma unroll
      for (int c = C - 1; c >= 0; --c)
        if (((uint64_t)cumc[c] << 32) > rhs) comp = c;
      float eps[D2];
      normals<D2>(a.key, a.t - 1, (uint32_t)g, P_PROP, (uint32_t)j, eps);
      float z[D2];
#pragma unroll
      for (int d = 0; d < D2; ++d) {
        float mu = 0.f, lsr = 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c)
          if (c == comp) {
            mu = o[C + c * D2 + d];
            lsr = o[C + C * D2 + c * D2 + d];
          }
        const float ls = fminf(fmaxf(lsr, kLogSigMin), kLogSigMax);
        z[d] = mu + expf(ls) * eps[d];
      }
      // log q(z): LSE over components (the -d2/2 log 2 pi constant cancels in lq)
      float lc[C];
      float cmax = NEG;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        float s = o[c] - lse_a;
#pragma unroll
        for (int d = 0; d < D2; ++d) {
          const float mu = o[C + c * D2 + d];
          const float ls = fminf(fmaxf(o[C + C * D2 + c * D2 + d], kLogSigMin), kLogSigMax);
          const float u = (z[d] - mu) * expf(-ls);
          s += -0.5f * u * u - ls;
        }
        lc[c] = s;
        cmax = fmaxf(cmax, s);
      }
      float sc = 0.f;
#pragma unroll
      for (int c = 0; c < C; ++c) sc += expf(lc[c] - cmax);
      const float lqz = cmax + logf(sc);
      // log N(z; A_zx x_a + A_zz z_b, Q_z) up to its constant
      float rp[D2];
#pragma unroll
      for (int r = 0; r < D2; ++r) {
        float m = 0.f;
#pragma unroll
        for (int c = 0; c < D1; ++c) m += mc.Azx[r][c] * xa[c];
#pragma unroll
        for (int c = 0; c < D2; ++c) m += mc.Azz[r][c] * zb[c];
        float v = z[r] - m;
#pragma unroll
        for (int c = 0; c < r; ++c) v -= mc.Lqz[r][c] * rp[c];
        rp[r] = v / mc.Lqz[r][r];
      }
      float lpz = 0.f;
#pragma unroll
      for (int r = 0; r < D2; ++r) lpz -= 0.5f * rp[r] * rp[r];
      // log p(y | x_t, z) up to its constant
      float hx[DY];
      h_x(mc, xt, hx);
      float res[DY];
#pragma unroll
      for (int q = 0; q < DY; ++q) {
        float v = a.y_prev[q] - hx[q];
#pragma unroll
        for (int c = 0; c < D2; ++c) v -= mc.Hz[q][c] * z[c];
        res[q] = v;
      }
      float lpy = 0.f;
#pragma unroll
      for (int q = 0; q < DY; ++q) {
        float v = 0.f;
#pragma unroll
        for (int c = 0; c <= q; ++c) v += mc.LrInv[q][c] * res[c];
        lpy -= 0.5f * v * v;
      }
      float lr = lpz - lqz + lpy;
      if (!live) lr = NEG;
      const float gm = group_max(lr, M, red);
      const float gs = group_sum(live ? expf(lr - gm) : 0.f, M, red);
      const float lqn = lr - gm - logf(gs);
      if (live) {
        const long long NM = a.N * (long long)M;
#pragma unroll
        for (int d = 0; d < D2; ++d) a.z_new[d * NM + row] = z[d];
        a.lq_new[row] = lqn;
        if (!(lqn == lqn)) atomicOr(a.err, ERR_NUMERIC);
      }
    }
    compute_sync();  // TMEM and the tiles are free for the next iteration
  }
  }  // compute warps
  if (!ok && lane == 0) atomicOr(MODE == 1 ? a.err : la.err, ERR_TIMEOUT);
  tc::fence_before();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(taddr, LTMEM_COLS);
}

template <int MODE, int D1, int D2, int DY, bool XZ, int NC>
static dpf_status launch_learned(const MC<float, D1, D2, DY>& mc, const StepArgs<float>& a, const LearnArgs& la,
                                 long long rows, cudaStream_t s) {
  auto k = learned_kernel<MODE, D1, D2, DY, XZ, NC>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_BYTES);
    if (e != cudaSuccess) return cuda_error(e, "learned kernel attribute");
    attr = true;
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long iters = (rows + LROWS - 1) / LROWS;
  const int grid = (int)std::max<long long>(1, std::min<long long>(iters, nsm));
  k<<<grid, LTHREADS, SM_BYTES, s>>>(mc, a, la);
  return cuda_error(cudaGetLastError(), "learned kernel launch");
}

static uint32_t scale_for(int n) {
  return 1u << (31 - ceil_log2_i(n));
}

// ---- the outer-amortised proposal: one network row per outer particle ----
// Group features (x_{t-1} of the ancestor, x_t, y_t, m, v) with mu_ij = A_zx x_{t-1} +
// A_zz z_{t-1}^(a, b_ij), m and v their mean and variance over j; the head gives the
// group's (raw log s, c); the particle draws zhat = mu + L_qz eps (PROP noise) and
// takes z = k + c + s (zhat - k) about the centre k (m, or the particle's own mu), weighted by log N(z; mu, Q_z) - log N(zhat; mu, Q_z)
// + sum log s + log p(y_t | x_t, z).

// Selection, local resampling and the group features; one warp per outer particle,
// PP = M / 32 consecutive inner particles a lane.
template <int D1, int D2, int DY, bool XZ, int PP>
__global__ void __launch_bounds__(128)
    oa_prepare_kernel(const __grid_constant__ MC<float, D1, D2, DY> mc, const __grid_constant__ StepArgs<float> a,
                      int32_t* __restrict__ bidx_out, float* __restrict__ feat, int din) {
  constexpr int M = 32 * PP;
  __shared__ uint32_t cum_s[4][M];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long g = blockIdx.x * 4LL + w;
  if (g >= a.N) return;  // whole warps only
  uint32_t* cum = cum_s[w];
  const float NEG = -INFINITY;
  const long long NM = a.N * (long long)M;
  const int anc_g = a.anc[g];
  const int L = a.L;
  int msel;
  {
    const float l0 = lane < L ? a.lwh_old[(long long)anc_g * L + lane] : NEG;
    const float l1 = lane + 32 < L ? a.lwh_old[(long long)anc_g * L + lane + 32] : NEG;
    const float mx = warp_max(fmaxf(l0, l1));
    const uint32_t c0 = lane < L ? (uint32_t)floorf(exp2f((l0 - mx) * 1.4426950408889634f) * a.scaleL) : 0u;
    const uint32_t c1 = lane + 32 < L ? (uint32_t)floorf(exp2f((l1 - mx) * 1.4426950408889634f) * a.scaleL) : 0u;
    uint32_t s0 = c0, s1 = c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t n0 = __shfl_up_sync(FULL, s0, o), n1 = __shfl_up_sync(FULL, s1, o);
      if (lane >= o) {
        s0 += n0;
        s1 += n1;
      }
    }
    const uint32_t tot0 = __shfl_sync(FULL, s0, 31), tot1 = __shfl_sync(FULL, s1, 31);
    const uint64_t Cs = (uint64_t)tot0 + tot1;
    const uint32_t usel = philox(ctr(a.t - 1, (uint32_t)g, P_SEL, 0u, 0u), a.key).x;
    const uint64_t rhs = (uint64_t)usel * Cs;
    const unsigned b0 = __ballot_sync(FULL, ((uint64_t)s0 << 32) > rhs);
    const unsigned b1 = __ballot_sync(FULL, ((uint64_t)(s1 + tot0) << 32) > rhs);
    msel = b0 ? __ffs(b0) - 1 : (b1 ? 32 + __ffs(b1) - 1 : L - 1);
    if ((Cs == 0 || msel >= L) && lane == 0) atomicOr(a.err, ERR_NUMERIC);
    if (msel >= L) msel = L - 1;
  }
  float xt[D1], xa[D1];
#pragma unroll
  for (int c = 0; c < D1; ++c) {
    xt[c] = a.xbb_old[((long long)anc_g * L + msel) * D1 + c];
    xa[c] = a.x_old[(long long)anc_g * a.xp + c];
  }
  if (lane == 0) {
    a.sel[g] = msel;
    for (int c = 0; c < a.xp; ++c) a.x_new[g * a.xp + c] = c < D1 ? xt[c < D1 ? c : 0] : 0.f;
  }
  float wres[D1];
  if (XZ) {
    float mxa[D1];
    mu_x(mc, xa, a.gcos_prev, mxa);
#pragma unroll
    for (int r = 0; r < D1; ++r) {
      float v = 0.f;
#pragma unroll
      for (int c = 0; c <= r; ++c) v += mc.LqxInv[r][c] * (xt[c] - mxa[c]);
      wres[r] = v;
    }
  }
  float al[PP];
  float amax = NEG;
#pragma unroll
  for (int p = 0; p < PP; ++p) {
    const int k = lane * PP + p;
    float v0 = a.lq_old[(long long)anc_g * M + k];
    if (XZ) {
      float q = 0.f;
#pragma unroll
      for (int r = 0; r < D1; ++r) {
        float v = wres[r];
#pragma unroll
        for (int c = 0; c < D2; ++c) v -= mc.WAxz[r][c] * a.z_old[c * NM + (long long)anc_g * M + k];
        q += v * v;
      }
      v0 -= 0.5f * q;
    }
    al[p] = v0;
    amax = fmaxf(amax, v0);
  }
  amax = warp_max(amax);
  uint32_t loc[PP];
  uint32_t run = 0;
#pragma unroll
  for (int p = 0; p < PP; ++p) {
    run += (uint32_t)floorf(exp2f((al[p] - amax) * 1.4426950408889634f) * a.scaleM);
    loc[p] = run;
  }
  uint32_t inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t n = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += n;
  }
#pragma unroll
  for (int p = 0; p < PP; ++p) cum[lane * PP + p] = loc[p] + inc - run;
  __syncwarp();
  const uint32_t C = cum[M - 1];
  if (C == 0 && lane == 0) atomicOr(a.err, ERR_NUMERIC);
  const uint32_t uin = philox(ctr(a.t - 1, (uint32_t)g, P_INNER, 0u, 0u), a.key).x;
  float mu[PP][D2];
  float msum[D2];
#pragma unroll
  for (int d = 0; d < D2; ++d) msum[d] = 0.f;
#pragma unroll
  for (int p = 0; p < PP; ++p) {
    const int k = lane * PP + p;
    const int b = sys_local_pick(cum, M, C, M, k, uin);
    bidx_out[g * M + k] = b;
    if (a.dbg_b) a.dbg_b[g * M + k] = b;
    float zb[D2];
#pragma unroll
    for (int c = 0; c < D2; ++c) zb[c] = a.z_old[c * NM + (long long)anc_g * M + b];
#pragma unroll
    for (int r = 0; r < D2; ++r) {
      float v = 0.f;
#pragma unroll
      for (int c = 0; c < D1; ++c) v += mc.Azx[r][c] * xa[c];
#pragma unroll
      for (int c = 0; c < D2; ++c) v += mc.Azz[r][c] * zb[c];
      mu[p][r] = v;
      msum[r] += v;
    }
  }
  float m[D2], vs[D2];
#pragma unroll
  for (int d = 0; d < D2; ++d) m[d] = warp_sum(msum[d]) / (float)M;
#pragma unroll
  for (int d = 0; d < D2; ++d) {
    float q = 0.f;
#pragma unroll
    for (int p = 0; p < PP; ++p) q += (mu[p][d] - m[d]) * (mu[p][d] - m[d]);
    vs[d] = warp_sum(q) / (float)M;
  }
  if (lane == 0) {
    float* f = feat + g * din;
    int k = 0;
#pragma unroll
    for (int c = 0; c < D1; ++c) f[k++] = xa[c];
#pragma unroll
    for (int c = 0; c < D1; ++c) f[k++] = xt[c];
#pragma unroll
    for (int q = 0; q < DY; ++q) f[k++] = a.y_prev[q];
#pragma unroll
    for (int d = 0; d < D2; ++d) f[k++] = m[d];
#pragma unroll
    for (int d = 0; d < D2; ++d) f[k++] = vs[d];
  }
}

// The draws and weights of the amortised proposal; one warp per outer particle.
template <int D1, int D2, int DY, int PP>
__global__ void __launch_bounds__(128)
    oa_update_kernel(const __grid_constant__ MC<float, D1, D2, DY> mc, const __grid_constant__ StepArgs<float> a,
                     const int32_t* __restrict__ bidx, const float* __restrict__ feat, const float* __restrict__ out,
                     int din, int dout, int centre) {
  constexpr int M = 32 * PP;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long g = blockIdx.x * 4LL + w;
  if (g >= a.N) return;
  const float NEG = -INFINITY;
  const long long NM = a.N * (long long)M;
  const int anc_g = a.anc[g];
  float xa[D1], xt[D1];
#pragma unroll
  for (int c = 0; c < D1; ++c) {
    xa[c] = a.x_old[(long long)anc_g * a.xp + c];
    xt[c] = a.x_new[g * a.xp + c];
  }
  float ls[D2], sc[D2], cc[D2], m[D2];
  float sum_ls = 0.f;
#pragma unroll
  for (int d = 0; d < D2; ++d) {
    ls[d] = fminf(fmaxf(out[g * dout + d], kLogSigMin), kLogSigMax);
    sc[d] = expf(ls[d]);
    cc[d] = out[g * dout + D2 + d];
    m[d] = feat[g * din + 2 * D1 + DY + d];
    sum_ls += ls[d];
  }
  float hx[DY];
  h_x(mc, xt, hx);
  float z[PP][D2], lr[PP];
  float lmax = NEG;
#pragma unroll
  for (int p = 0; p < PP; ++p) {
    const int k = lane * PP + p;
    const int b = bidx[g * M + k];
    float zb[D2], mu[D2];
#pragma unroll
    for (int c = 0; c < D2; ++c) zb[c] = a.z_old[c * NM + (long long)anc_g * M + b];
#pragma unroll
    for (int r = 0; r < D2; ++r) {
      float v = 0.f;
#pragma unroll
      for (int c = 0; c < D1; ++c) v += mc.Azx[r][c] * xa[c];
#pragma unroll
      for (int c = 0; c < D2; ++c) v += mc.Azz[r][c] * zb[c];
      mu[r] = v;
    }
    float eps[D2];
    normals<D2>(a.key, a.t - 1, (uint32_t)g, P_PROP, (uint32_t)k, eps);
    float e2 = 0.f;
#pragma unroll
    for (int r = 0; r < D2; ++r) {
      float zh = mu[r];
#pragma unroll
      for (int c = 0; c <= r; ++c) zh += mc.Lqz[r][c] * eps[c];
      const float k = centre ? mu[r] : m[r];
      z[p][r] = k + cc[r] + sc[r] * (zh - k);
      e2 += eps[r] * eps[r];
    }
    // log N(z; mu, Q_z) by forward substitution with L_qz
    float rp[D2];
    float lpz = 0.f;
#pragma unroll
    for (int r = 0; r < D2; ++r) {
      float v = z[p][r] - mu[r];
#pragma unroll
      for (int c = 0; c < r; ++c) v -= mc.Lqz[r][c] * rp[c];
      rp[r] = v / mc.Lqz[r][r];
      lpz -= 0.5f * rp[r] * rp[r];
    }
    float lpy = 0.f;
#pragma unroll
    for (int q = 0; q < DY; ++q) {
      float res[DY];
      (void)res;
      float v = 0.f;
#pragma unroll
      for (int c2 = 0; c2 <= q; ++c2) {
        float rr = a.y_prev[c2] - hx[c2];
#pragma unroll
        for (int c = 0; c < D2; ++c) rr -= mc.Hz[c2][c] * z[p][c];
        v += mc.LrInv[q][c2] * rr;
      }
      lpy -= 0.5f * v * v;
    }
    lr[p] = lpz - (-0.5f * e2 - sum_ls) + lpy;
    lmax = fmaxf(lmax, lr[p]);
  }
  lmax = warp_max(lmax);
  float se = 0.f;
#pragma unroll
  for (int p = 0; p < PP; ++p) se += expf(lr[p] - lmax);
  const float lse = lmax + logf(warp_sum(se));
#pragma unroll
  for (int p = 0; p < PP; ++p) {
    const int k = lane * PP + p;
#pragma unroll
    for (int d = 0; d < D2; ++d) a.z_new[d * NM + g * M + k] = z[p][d];
    const float lq = lr[p] - lse;
    a.lq_new[g * M + k] = lq;
    if (!(lq == lq)) atomicOr(a.err, ERR_NUMERIC);
  }
}

// Training rows of the amortised proposal from the last inner update: one warp per
// outer particle writes, for each of its inner particles, the group features and
// (z_t, mu, m), and w = exp(lq_t) / N.
template <int D1, int D2, int DY, int PP>
__global__ void __launch_bounds__(128)
    oa_record_kernel(const __grid_constant__ MC<float, D1, D2, DY> mc, const float* x_old, const float* x_new,
                     const float* z_old, const float* z_new, const float* lq_new, const float* y_prev,
                     const int32_t* anc_prev, const int32_t* bidx, long long N, int xp, long long i0,
                     long long n_outer, float* G, float* Zr, float* wr) {
  constexpr int M = 32 * PP;
  constexpr int DIN = 2 * D1 + DY + 2 * D2;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long q = blockIdx.x * 4LL + w;
  if (q >= n_outer) return;
  const long long g = i0 + q;
  const long long NM = N * (long long)M;
  const int a = anc_prev[g];
  float xa[D1], xt[D1];
#pragma unroll
  for (int c = 0; c < D1; ++c) {
    xa[c] = x_old[(long long)a * xp + c];
    xt[c] = x_new[g * xp + c];
  }
  float mu[PP][D2], msum[D2];
#pragma unroll
  for (int d = 0; d < D2; ++d) msum[d] = 0.f;
#pragma unroll
  for (int p = 0; p < PP; ++p) {
    const int k = lane * PP + p;
    const int b = bidx[g * M + k];
#pragma unroll
    for (int r = 0; r < D2; ++r) {
      float v = 0.f;
#pragma unroll
      for (int c = 0; c < D1; ++c) v += mc.Azx[r][c] * xa[c];
#pragma unroll
      for (int c = 0; c < D2; ++c) v += mc.Azz[r][c] * z_old[c * NM + (long long)a * M + b];
      mu[p][r] = v;
      msum[r] += v;
    }
  }
  float m[D2], vs[D2];
#pragma unroll
  for (int d = 0; d < D2; ++d) m[d] = warp_sum(msum[d]) / (float)M;
#pragma unroll
  for (int d = 0; d < D2; ++d) {
    float s2 = 0.f;
#pragma unroll
    for (int p = 0; p < PP; ++p) s2 += (mu[p][d] - m[d]) * (mu[p][d] - m[d]);
    vs[d] = warp_sum(s2) / (float)M;
  }
#pragma unroll
  for (int p = 0; p < PP; ++p) {
    const int k = lane * PP + p;
    const long long e = q * M + k;
    float* f = G + e * DIN;
    int o = 0;
#pragma unroll
    for (int c = 0; c < D1; ++c) f[o++] = xa[c];
#pragma unroll
    for (int c = 0; c < D1; ++c) f[o++] = xt[c];
#pragma unroll
    for (int c = 0; c < DY; ++c) f[o++] = y_prev[c];
#pragma unroll
    for (int d = 0; d < D2; ++d) f[o++] = m[d];
#pragma unroll
    for (int d = 0; d < D2; ++d) f[o++] = vs[d];
    float* zr = Zr + e * 3 * D2;
#pragma unroll
    for (int d = 0; d < D2; ++d) {
      zr[d] = z_new[d * NM + g * M + k];
      zr[D2 + d] = mu[p][d];
      zr[2 * D2 + d] = m[d];
    }
    wr[e] = expf(lq_new[g * M + k]) / (float)N;
  }
}

template <int PP>
static dpf_status oa_step_pp(Ctx& x, const MC<float, 2, 2, 2>& mc, StepArgs<float>& a, dpf_proposal& p) {
  const unsigned blocks = (unsigned)((x.N + 3) / 4);
  if (x.hm.xz)
    oa_prepare_kernel<2, 2, 2, true, PP><<<blocks, 128, 0, x.stream>>>(mc, a, (int32_t*)x.oa_bidx, (float*)x.oa_feat, p.din);
  else
    oa_prepare_kernel<2, 2, 2, false, PP><<<blocks, 128, 0, x.stream>>>(mc, a, (int32_t*)x.oa_bidx, (float*)x.oa_feat, p.din);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "amortised prepare launch");
  LearnArgs la{};
  la.wp = (const unsigned char*)p.packed;
  la.din = p.din;
  la.dout = p.dout;
  la.C = 1;
  la.F = (const float*)x.oa_feat;
  la.out = (float*)x.oa_out;
  la.nrows = x.N;
  la.err = x.err;
  MC<float, 2, 2, 2> mc0;
  memset(&mc0, 0, sizeof(mc0));
  StepArgs<float> a0{};
  a0.err = x.err;
  dpf_status st = launch_learned<0, 2, 2, 2, false, kFilterComponents>(mc0, a0, la, x.N, x.stream);
  if (st) return st;
  oa_update_kernel<2, 2, 2, PP><<<blocks, 128, 0, x.stream>>>(mc, a, (const int32_t*)x.oa_bidx,
                                                               (const float*)x.oa_feat, (const float*)x.oa_out,
                                                               p.din, p.dout, p.centre);
  return cuda_error(cudaGetLastError(), "amortised update launch");
}

// The per-group fallback: the inner effective sample size of each group's learned
// update, ESS = (sum_j W_j)^2 / sum_j W_j^2 with W = exp(lq), against thr = fb_frac M.
// Groups below it (or with no finite weight) are flagged and listed (in no particular
// order) for the plain inner update; one warp a group.
__global__ void fallback_lists_kernel(const float* __restrict__ lq, long long N, int M, float thr,
                                      int32_t* flag, int32_t* list, int32_t* count) {
  const long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= N) return;  // whole warps
  float s1 = 0.f, s2 = 0.f;
  for (int k = lane; k < M; k += 32) {
    const float w = expf(lq[i * M + k]);
    s1 += w;
    s2 += w * w;
  }
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  if (lane == 0) {
    const bool fb = !(s1 * s1 >= thr * s2);
    flag[i] = fb ? 1 : 0;
    if (fb) list[atomicAdd(count, 1)] = (int32_t)i;
  }
}

dpf_status learned_fallback_lists(Ctx& x) {
  const long long t = x.t + 1;
  if (x.fb_frac <= 0.0)  // no fallback: no group is flagged
    return cuda_error(cudaMemsetAsync(x.fb_flag, 0, sizeof(int32_t) * x.N, x.stream), "fallback flags");
  cudaError_t e = cudaMemsetAsync(x.fb_count, 0, sizeof(int32_t), x.stream);
  if (e != cudaSuccess) return cuda_error(e, "fallback counts");
  const unsigned blocks = (unsigned)((x.N + 3) / 4);
  fallback_lists_kernel<<<blocks, 128, 0, x.stream>>>((const float*)x.lq[(t + 1) % 2], x.N, x.M,
                                                      (float)(x.fb_frac * x.M), x.fb_flag, x.fb_list,
                                                      x.fb_count);
  return cuda_error(cudaGetLastError(), "fallback lists launch");
}

// The inner update of the coming step with the learned proposal (the variant
// (FP32, 2, 2, 2)); then the look-ahead runs alone from the materialised state.
dpf_status learned_inner_step(Ctx& x) {
  dpf_proposal& p = *x.proposal;
  if (p.kind == 1 && oa_wide_shape(x)) return oa_wide_step(x, p);
  dpf_status st = pack(p);
  if (st) return st;
  typedef VariantImpl<float, 2, 2, 2, 0> V;
  StepArgs<float> a{};
  V::fill_args(x, a);
  a.xp = x.xp;  // the padded x row (set by the step geometry for the other kernels)
  LearnArgs la{};
  la.wp = (const unsigned char*)p.packed;
  la.din = p.din;
  la.dout = p.dout;
  la.C = p.C;
  la.dbg_head = x.debug ? (float*)x.dbg_head : nullptr;
  la.scaleC = scale_for(p.C);
  la.err = x.err;
  const MC<float, 2, 2, 2>& mc = *reinterpret_cast<const MC<float, 2, 2, 2>*>(x.mconst.data());
  if (p.kind == 1) {
    switch (x.M) {
      case 32: return oa_step_pp<1>(x, mc, a, p);
      case 64: return oa_step_pp<2>(x, mc, a, p);
      case 128: return oa_step_pp<4>(x, mc, a, p);
      default: return oa_step_pp<8>(x, mc, a, p);
    }
  }
  const long long rows = x.N * (long long)x.M;
  return x.hm.xz ? launch_learned<1, 2, 2, 2, true, kFilterComponents>(mc, a, la, rows, x.stream)
                 : launch_learned<1, 2, 2, 2, false, kFilterComponents>(mc, a, la, rows, x.stream);
}

// ---- training rows from the last inner update ----
struct RecordArgs {
  const float *x_old, *x_new, *z_old, *z_new, *lq_new, *y_prev;
  const int32_t *anc_prev, *bidx;
  long long N, i0, n_outer;
  int M, d1, d2, dy, xp, din;
  float* F;
  float* Z;
  float* w;
};

__global__ void record_kernel(RecordArgs r) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= r.n_outer * r.M) return;
  const long long g = r.i0 + e / r.M;
  const int j = (int)(e % r.M);
  const long long NM = r.N * (long long)r.M;
  const long long a = r.anc_prev[g];
  const int b = r.bidx[g * r.M + j];
  float* f = r.F + e * r.din;
  int k = 0;
  for (int c = 0; c < r.d1; ++c) f[k++] = r.x_old[a * r.xp + c];
  for (int c = 0; c < r.d1; ++c) f[k++] = r.x_new[g * r.xp + c];
  for (int c = 0; c < r.d2; ++c) f[k++] = r.z_old[c * NM + a * r.M + b];
  for (int q = 0; q < r.dy; ++q) f[k++] = r.y_prev[q];
  for (int c = 0; c < r.d2; ++c) r.Z[e * r.d2 + c] = r.z_new[c * NM + g * r.M + j];
  r.w[e] = expf(r.lq_new[g * r.M + j]) / (float)r.N;
}

}  // namespace dpf

using namespace dpf;

extern "C" {

dpf_status dpf_proposal_forward(dpf_proposal* p, const float* F, int64_t n, float* out) {
  clear_error();
  if (!p || !F || !out || n < 1) return set_error(DPF_E_INVALID, "dpf_proposal_forward: bad arguments");
  if (p->hidden != LH || p->dout > LNP || p->din > LDIN)
    return set_error(DPF_E_UNSUPPORTED, "dpf_proposal_forward: the tensor-core pass needs hidden = 256, "
                                        "din <= 16 and dout <= 32");
  dpf_status st = pack(*p);
  if (st) return st;
  int* err = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&err, sizeof(int), p->stream);
  if (e != cudaSuccess) return cuda_error(e, "dpf_proposal_forward: allocation");
  cudaMemsetAsync(err, 0, sizeof(int), p->stream);
  LearnArgs la{};
  la.wp = (const unsigned char*)p->packed;
  la.din = p->din;
  la.dout = p->dout;
  la.C = p->C;
  la.F = F;
  la.out = out;
  la.nrows = n;
  la.err = err;
  MC<float, 2, 2, 2> mc;
  memset(&mc, 0, sizeof(mc));
  StepArgs<float> a{};
  st = launch_learned<0, 2, 2, 2, false, kFilterComponents>(mc, a, la, n, p->stream);
  int h = 0;
  e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  cudaFreeAsync(err, p->stream);
  if (st) return st;
  if (e != cudaSuccess) return cuda_error(e, "dpf_proposal_forward");
  if (h) return set_error(DPF_E_TIMEOUT, "dpf_proposal_forward: a bounded wait gave up");
  return DPF_OK;
}

dpf_status dpf_set_proposal(dpf_ctx* x, dpf_proposal* p) {
  clear_error();
  if (!x) return set_error(DPF_E_INVALID, "dpf_set_proposal: null context");
  if (!p) {
    x->proposal = nullptr;
    return DPF_OK;
  }
  if (x->pf || x->std_dpf)
    return set_error(DPF_E_INVALID, "dpf_set_proposal: the learned proposal serves the LA-DPF only");
  if (x->prec != DPF_F32 || p->d1 != x->d1 || p->d2 != x->d2 || p->dy != x->dy)
    return set_error(DPF_E_INVALID, "dpf_set_proposal: the proposal's (d1, d2, dy) and FP32 must match the filter");
  if (p->kind == 0 && (!(x->d1 == 2 && x->d2 == 2 && x->dy == 2) || p->hidden != LH || p->C != kFilterComponents ||
                       !(x->M == 32 || x->M == 64 || x->M == 128)))
    return set_error(DPF_E_UNSUPPORTED, "dpf_set_proposal: compiled for (d1, d2, dy) = (2, 2, 2), hidden 256, "
                                        "4 components and M in {32, 64, 128}");
  const bool wide = p->kind == 1 && oa_wide_shape(*x);
  if (p->kind == 1 && !wide &&
      (!(x->d1 == 2 && x->d2 == 2 && x->dy == 2) || p->hidden != LH ||
       !(x->M == 32 || x->M == 64 || x->M == 128 || x->M == 256)))
    return set_error(DPF_E_UNSUPPORTED, "dpf_set_proposal: the amortised pass is compiled for (d1, d2, dy) = "
                                        "(2, 2, 2), hidden 256 and M in {32, 64, 128, 256}, and for (8, 56, 8) "
                                        "with x free of z and M a multiple of 32 up to 256");
  auto grow = [&](void** q, size_t bytes) -> cudaError_t {
    if (*q) return cudaSuccess;
    cudaError_t e = device_malloc(q, bytes);
    if (e == cudaSuccess) x->allocs.push_back(*q);
    if (e == cudaSuccess) e = cudaMemsetAsync(*q, 0, bytes, x->stream);
    return e;
  };
  {  // the per-group fallback's flags, group lists and counts
    cudaError_t e = grow((void**)&x->fb_flag, sizeof(int32_t) * (size_t)x->N);
    if (e == cudaSuccess) e = grow((void**)&x->fb_list, sizeof(int32_t) * (size_t)x->N);
    if (e == cudaSuccess) e = grow((void**)&x->fb_count, sizeof(int32_t));
    if (e != cudaSuccess) return cuda_error(e, "dpf_set_proposal: fallback buffers");
  }
  if (p->kind == 1) {
    cudaError_t e = grow(&x->oa_bidx, sizeof(int32_t) * (size_t)x->N * x->M);
    if (e == cudaSuccess) e = grow(&x->oa_feat, sizeof(float) * (size_t)x->N * std::max(LDIN, p->din));
    if (e == cudaSuccess) e = grow(&x->oa_out, sizeof(float) * (size_t)x->N * std::max(LNP, p->dout));
    if (e == cudaSuccess && wide) e = grow(&x->oa_hidden, sizeof(float) * 2 * (size_t)x->N * p->hidden);
    if (e == cudaSuccess && wide) e = grow(&x->oa_mu, sizeof(float) * (size_t)x->d2 * x->N * x->M);
    if (e != cudaSuccess) return cuda_error(e, "dpf_set_proposal: amortised buffers");
  }
  x->proposal = p;
  return DPF_OK;
}

dpf_status dpf_set_fallback(dpf_ctx* x, double frac) {
  clear_error();
  if (!x || !(frac >= 0.0 && frac <= 1.0))
    return set_error(DPF_E_INVALID, "dpf_set_fallback: null context or frac outside [0, 1]");
  x->fb_frac = frac;
  return DPF_OK;
}

dpf_status dpf_record_tuples_amortised(dpf_ctx* x, int64_t i0, int64_t n_outer, float* G, float* Z, float* w) {
  clear_error();
  if (!x || !G || !Z || !w || i0 < 0 || n_outer < 1 || i0 + n_outer > x->N)
    return set_error(DPF_E_INVALID, "dpf_record_tuples_amortised: bad arguments");
  if (x->t < 2 || !x->dbg_b || !x->anc_prev || x->prec != DPF_F32)
    return set_error(DPF_E_INVALID, "dpf_record_tuples_amortised: needs an FP32 filter stepped at least twice "
                                    "with debug recording on");
  if (oa_wide_shape(*x)) {
    dpf_status st = oa_wide_record(*x, i0, n_outer, G, Z, w);
    if (st) return st;
    return cuda_error(cudaStreamSynchronize(x->stream), "dpf_record_tuples_amortised");
  }
  if (!(x->d1 == 2 && x->d2 == 2 && x->dy == 2) || x->M % 32 || x->M > 256)
    return set_error(DPF_E_UNSUPPORTED, "dpf_record_tuples_amortised: compiled for (2, 2, 2) and (8, 56, 8), "
                                        "M a multiple of 32 up to 256");
  const long long t = x->t;
  const MC<float, 2, 2, 2>& mc = *reinterpret_cast<const MC<float, 2, 2, 2>*>(x->mconst.data());
  const unsigned blocks = (unsigned)((n_outer + 3) / 4);
  auto go = [&](auto kern) {
    kern<<<blocks, 128, 0, x->stream>>>(mc, (const float*)x->x[t % 2], (const float*)x->x[(t + 1) % 2],
                                        (const float*)x->z[t % 2], (const float*)x->z[(t + 1) % 2],
                                        (const float*)x->lq[(t + 1) % 2],
                                        (const float*)x->yb + ((t + 1) % 2) * x->dy, x->anc_prev, x->dbg_b, x->N,
                                        x->xp, i0, n_outer, G, Z, w);
  };
  switch (x->M) {
    case 32: go(oa_record_kernel<2, 2, 2, 1>); break;
    case 64: go(oa_record_kernel<2, 2, 2, 2>); break;
    case 128: go(oa_record_kernel<2, 2, 2, 4>); break;
    default: go(oa_record_kernel<2, 2, 2, 8>); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  return cuda_error(e, "dpf_record_tuples_amortised");
}

dpf_status dpf_record_tuples(dpf_ctx* x, int64_t i0, int64_t n_outer, float* F, float* Z, float* w) {
  clear_error();
  if (!x || !F || !Z || !w || i0 < 0 || n_outer < 1 || i0 + n_outer > x->N)
    return set_error(DPF_E_INVALID, "dpf_record_tuples: bad arguments");
  if (x->t < 2 || !x->dbg_b || !x->anc_prev || x->prec != DPF_F32)
    return set_error(DPF_E_INVALID, "dpf_record_tuples: needs an FP32 filter stepped at least twice with "
                                    "debug recording on");
  const long long t = x->t;  // the last call materialised step t - 1 from step t - 2
  RecordArgs r{};
  r.x_old = (const float*)x->x[t % 2];
  r.z_old = (const float*)x->z[t % 2];
  r.x_new = (const float*)x->x[(t + 1) % 2];
  r.z_new = (const float*)x->z[(t + 1) % 2];
  r.lq_new = (const float*)x->lq[(t + 1) % 2];
  r.y_prev = (const float*)x->yb + ((t + 1) % 2) * x->dy;
  r.anc_prev = x->anc_prev;
  r.bidx = x->dbg_b;
  r.N = x->N;
  r.i0 = i0;
  r.n_outer = n_outer;
  r.M = x->M;
  r.d1 = x->d1;
  r.d2 = x->d2;
  r.dy = x->dy;
  r.xp = x->xp;
  r.din = 2 * x->d1 + x->d2 + x->dy;
  r.F = F;
  r.Z = Z;
  r.w = w;
  const long long n = n_outer * x->M;
  record_kernel<<<(unsigned)((n + 255) / 256), 256, 0, x->stream>>>(r);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  return cuda_error(e, "dpf_record_tuples");
}

}  // extern "C"
