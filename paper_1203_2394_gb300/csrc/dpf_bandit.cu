// Automatic choice of the state decomposition by online bandits (the paper's
// Section "Automatic State Decomposition", Fig. hedge, after Auer et al. 1995):
// Hedge with full reward vectors (every decomposition runs, as in the batched
// form) and Exp3 with the reward of the one decomposition tried. Host code.
#include <cmath>
#include <cstdint>
#include <vector>

#include "dpf_internal.h"

namespace dpf {

// Philox4x32-10 on the host (Salmon et al. 2011), the bandit's own draws.
static void philox_host(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0, n1 = (uint32_t)p1;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1, n3 = (uint32_t)p0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

constexpr uint32_t P_BANDIT = 11;  // Philox purpose of the bandit's action draws

}  // namespace dpf

struct dpf_bandit {
  int kind = 0, K = 0;
  double eta = 0.0, gamma = 0.0;
  uint64_t seed = 0;
  uint32_t t = 0;               // rounds completed
  std::vector<double> G;        // cumulative (simulated) rewards
  int last = -1;                // the action drawn for the current round
  std::vector<double> phat;     // the distribution the last action was drawn from
};

namespace {

// Hedge's p(t): p_i proportional to exp(eta G_i(t-1)) (shifted by the largest for range).
void hedge_p(const dpf_bandit& b, double* p) {
  double mx = -INFINITY;
  for (int i = 0; i < b.K; ++i) mx = std::fmax(mx, b.eta * b.G[i]);
  double s = 0.0;
  for (int i = 0; i < b.K; ++i) s += (p[i] = std::exp(b.eta * b.G[i] - mx));
  for (int i = 0; i < b.K; ++i) p[i] /= s;
}

// The distribution actions are drawn from: Hedge's p(t), or Exp3's
// phat(t) = (1 - gamma) p(t) + gamma / K.
void draw_p(const dpf_bandit& b, double* p) {
  hedge_p(b, p);
  if (b.kind == DPF_EXP3)
    for (int i = 0; i < b.K; ++i) p[i] = (1.0 - b.gamma) * p[i] + b.gamma / b.K;
}

}  // namespace

using namespace dpf;

extern "C" {

dpf_status dpf_bandit_create(int32_t kind, int32_t K, double eta, double gamma, uint64_t seed, dpf_bandit** out) {
  clear_error();
  if (!out) return set_error(DPF_E_INVALID, "dpf_bandit_create: null output");
  *out = nullptr;
  if ((kind != DPF_HEDGE && kind != DPF_EXP3) || K < 1 || K > 4096 || !(eta > 0.0) ||
      (kind == DPF_EXP3 && !(gamma > 0.0 && gamma <= 1.0)))
    return set_error(DPF_E_INVALID, "dpf_bandit_create: kind HEDGE or EXP3, 1 <= K <= 4096, eta > 0, "
                                    "0 < gamma <= 1 for EXP3");
  dpf_bandit* b = new dpf_bandit();
  b->kind = kind;
  b->K = K;
  b->eta = eta;
  b->gamma = gamma;
  b->seed = seed;
  b->G.assign(K, 0.0);
  b->phat.assign(K, 1.0 / K);
  *out = b;
  return DPF_OK;
}

dpf_status dpf_bandit_probs(const dpf_bandit* b, double* p) {
  clear_error();
  if (!b || !p) return set_error(DPF_E_INVALID, "dpf_bandit_probs: null argument");
  draw_p(*b, p);
  return DPF_OK;
}

dpf_status dpf_bandit_choose(dpf_bandit* b, int32_t* action) {
  clear_error();
  if (!b || !action) return set_error(DPF_E_INVALID, "dpf_bandit_choose: null argument");
  draw_p(*b, b->phat.data());
  // one word of the bandit's stream for round t, inverse CDF on the distribution
  uint32_t c[4] = {b->t, 0u, P_BANDIT << 24, 0u};
  philox_host(c, (uint32_t)b->seed, (uint32_t)(b->seed >> 32));
  const double u = (c[0] + 0.5) * 0x1p-32;
  double cum = 0.0;
  int a = b->K - 1;
  for (int i = 0; i < b->K; ++i) {
    cum += b->phat[i];
    if (u < cum) {
      a = i;
      break;
    }
  }
  b->last = a;
  *action = a;
  return DPF_OK;
}

dpf_status dpf_bandit_update(dpf_bandit* b, const double* rewards) {
  clear_error();
  if (!b || !rewards) return set_error(DPF_E_INVALID, "dpf_bandit_update: null argument");
  if (b->kind == DPF_HEDGE) {
    for (int i = 0; i < b->K; ++i)
      if (!(rewards[i] >= 0.0 && rewards[i] <= 1.0))
        return set_error(DPF_E_INVALID, "dpf_bandit_update: rewards must lie in [0, 1]");
    for (int i = 0; i < b->K; ++i) b->G[i] += rewards[i];
  } else {
    if (b->last < 0) return set_error(DPF_E_INVALID, "dpf_bandit_update: Exp3 needs dpf_bandit_choose first");
    if (!(rewards[0] >= 0.0 && rewards[0] <= 1.0))
      return set_error(DPF_E_INVALID, "dpf_bandit_update: the reward must lie in [0, 1]");
    // the simulated reward vector: r / phat for the action tried, 0 for the others
    b->G[b->last] += rewards[0] / b->phat[b->last];
    b->last = -1;
  }
  b->t += 1;
  return DPF_OK;
}

dpf_status dpf_bandit_reward(const double* y, const double* yhat, int32_t dy, double alpha, double* r) {
  clear_error();
  if (!y || !yhat || !r || dy < 1 || !(alpha > 0.0))
    return set_error(DPF_E_INVALID, "dpf_bandit_reward: null argument, dy < 1 or alpha <= 0");
  double e2 = 0.0;
  for (int k = 0; k < dy; ++k) e2 += (y[k] - yhat[k]) * (y[k] - yhat[k]);
  *r = alpha / (alpha + e2);
  return DPF_OK;
}

void dpf_bandit_destroy(dpf_bandit* b) { delete b; }

}  // extern "C"
