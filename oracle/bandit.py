"""Oracle of the automatic state decomposition: Hedge and Exp3 as in the paper's
Fig. hedge (after Auer et al. 1995), written from the figure step by step.

TEST INFRASTRUCTURE ONLY: the tests may use this module; the library path never does.

Hedge: p_i(t) = exp(eta G_i(t-1)) / sum_j exp(eta G_j(t-1)); after the round,
G_i(t) = G_i(t-1) + r_i(t) for every action.
Exp3: phat_j(t) = (1 - gamma) p_j(t) + gamma / K; the action i_t is drawn from phat;
the simulated reward is r_{i_t}(t) / phat_{i_t}(t) for i_t and 0 elsewhere, fed to Hedge.
Draws: u = (w + 1/2) 2^-32 with w the first Philox4x32-10 word at counter
(t, 0, 11 << 24, 0), key (seed_lo, seed_hi); i_t = the first j with u < sum_{i <= j} phat_i.
"""
from __future__ import annotations

import numpy as np

P_BANDIT = 11


def reward(y, yhat, alpha):
    """Section 4.3: alpha / (alpha + eps^2), eps the one-step-ahead prediction error
    (its Euclidean norm for vector observations)."""
    e = np.asarray(y, dtype=np.float64) - np.asarray(yhat, dtype=np.float64)
    return alpha / (alpha + float(e @ e))


class Hedge:
    def __init__(self, K, eta):
        self.K, self.eta = K, eta
        self.G = np.zeros(K)

    def p(self):
        e = np.exp(self.eta * self.G - np.max(self.eta * self.G))
        return e / e.sum()

    def feed(self, r):
        self.G = self.G + np.asarray(r, dtype=np.float64)


class Exp3:
    def __init__(self, K, eta, gamma, seed, philox):
        self.hedge = Hedge(K, eta)
        self.K, self.gamma, self.seed, self.philox = K, gamma, seed, philox
        self.t = 0
        self.last = None

    def phat(self):
        return (1.0 - self.gamma) * self.hedge.p() + self.gamma / self.K

    def choose(self):
        ph = self.phat()
        w = int(self.philox((self.t, 0, P_BANDIT << 24, 0), (self.seed & 0xFFFFFFFF, self.seed >> 32))[0])
        u = (w + 0.5) * 2.0 ** -32
        cum = np.cumsum(ph)
        a = int(np.argmax(u < cum)) if np.any(u < cum) else self.K - 1
        self.last = (a, ph[a])
        return a

    def feed(self, r):
        a, pa = self.last
        rhat = np.zeros(self.K)
        rhat[a] = r / pa
        self.hedge.feed(rhat)
        self.t += 1
        self.last = None
