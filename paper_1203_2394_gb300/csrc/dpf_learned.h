// The learned inner proposal object (see dpf_learned.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "dpf_internal.h"

namespace dpf {

constexpr int kLayers = 4;           // three hidden layers and the head
constexpr int kMaxComponents = 8;
constexpr int kMaxDin = 16;          // inputs, padded to one BF16 MMA K step
constexpr int kMaxD2 = 8;
constexpr int kMaxDinAmortised = 160;  // the outer-amortised form: 2 d1 + dy + 2 d2 inputs
constexpr int kMaxD2Amortised = 64;
constexpr int kMaxHidden = 256;
constexpr int kMaxDout = 128;
constexpr float kLogSigMin = -7.f, kLogSigMax = 5.f;

dpf_status proposal_requantize(dpf_proposal& p);
// The network over n feature rows F (n x din) into out (n x dout) on the tensor cores,
// rounded as the training forward pass rounds; hidden holds 2 n x hidden floats. A
// bounded wait that gives up sets ERR_TIMEOUT in *err.
dpf_status proposal_forward_rows(dpf_proposal& p, const float* F, long long n, float* hidden, float* out, int* err,
                                 cudaStream_t s);

}  // namespace dpf

struct dpf_proposal {
  int kind = 0;  // 0: mixture of Gaussians per inner particle; 1: per-group affine map of the prior draws
  int d1 = 0, d2 = 0, dy = 0, din = 0, hidden = 0, C = 0, dout = 0;
  int zw = 0;    // floats per training target row: d2 (kind 0) or 3 d2 (z, prior mean, centre)
  int centre = 0;  // kind 1: the map's centre, 0 the group's mean prior mean m, 1 the particle's own mu
  float qinv[dpf::kMaxD2Amortised * dpf::kMaxD2Amortised] = {};  // kind 1: Q_z^-1 (row-major), the training loss
  float* qinv_d = nullptr;                      // ... its device copy
  float half_logdet = 0.f;                      // kind 1: 1/2 log det(2 pi Q_z)
  long long nparams = 0;
  long long offW[dpf::kLayers] = {}, offB[dpf::kLayers] = {};
  int rows[dpf::kLayers] = {}, cols[dpf::kLayers] = {};
  cudaStream_t stream = nullptr;
  bool bf16 = true;  // the forward pass rounds as the tensor-core pass does
  float* W = nullptr;      // FP32 master parameters
  float* Wq = nullptr;     // what the forward pass uses (bfloat16-rounded matrices when bf16)
  float* am = nullptr;     // Adam moments
  float* av = nullptr;
  float* grad = nullptr;
  double* loss_d = nullptr;
  double* wsum_d = nullptr;
  int* err_d = nullptr;    // device error word of the training products (bounded waits)
  int adam_t = 0;
  // minibatch workspace
  int ws_rows = 0;
  float *Fb = nullptr, *Zb = nullptr, *wb = nullptr, *h1 = nullptr, *h2 = nullptr, *h3 = nullptr;
  float *ob = nullptr, *dA = nullptr, *dB = nullptr, *dO = nullptr;
  int64_t* perm_d = nullptr;
  // weights packed for the tensor-core forward pass (rebuilt when stale)
  bool packed_valid = false;
  void* packed = nullptr;
  size_t packed_bytes = 0;
  std::vector<void*> allocs;
};
