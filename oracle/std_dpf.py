"""Oracle of the decentralized particle filter without look-ahead (the paper's Fig. dpf,
after Chen et al. 2011), with the prior as both proposals (r = 1), in x-first order.

TEST INFRASTRUCTURE ONLY: the tests may use this module; the library path never does.

One call t, for each outer particle i, in the figure's order (steps 4-7 for the coming
step, then 1 and 3 with y_t; step 2 is the global systematic resampling that follows):
  a = the ancestor the outer resampling of call t-1 gave i (i itself at t = 1);
  (4) x_t ~ sum_j qbar_j p(x_t | x_{t-1}^a, z_{t-1}^(a,j)): the component c by the one-draw
      local systematic rule on qbar with the word (t, i, LA_J, 0), then
      x_t = E[x_t | x_{t-1}^a, z^(a,c)] + chol(Q_x) e with e the normals (t, i, LA_X, 0);
  (5) q_j proportional to qbar_j p(x_t | x_{t-1}^a, z^(a,j));
  (6) b = the local systematic resampling of the M inner particles by q, word (t, i, INNER, 0);
  (7) z_t^(j) = E[z_t | x_{t-1}^a, z^(a,b_j)] + chol(Q_z) e_j, e_j the normals (t, i, PROP, j);
  (1) log w_i = log (1/M) sum_j p(y_t | x_t, z_t^(j));
  (3) log qbar_t^(j) = log p(y_t | x_t, z_t^(j)) - log sum_j p(y_t | x_t, z_t^(j)).
With the Gaussian approximation of the mixture (Section 4.2, Table 2), step (4) draws
x_t = mu + chol(S) e instead, mu = sum_j qbar_j m_j and S = Q_x + sum_j qbar_j (m_j - mu)
(m_j - mu)^T with m_j = E[x_t | x_{t-1}^a, z^(a,j)]: the mixture's first two moments.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle
from oracle.pf import log_gauss, obs_mean, transition_mean


def _word(seed, t, i, purpose, sub=0):
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return int(oracle.philox((t, i, (purpose << 24) | sub, 0), key)[0])


def _lse(v):
    m = np.max(v)
    return m + np.log(np.sum(np.exp(v - m)))


def std_step(model, seed, t, y, x_prev, z_prev, lq_prev, anc, lib, dest=None, gauss=False, comp_in=None,
             bidx_in=None, return_q=False, x_in=None):
    """One call from the state of step t-1: x_prev (N, d1), z_prev (N, M, d2), lq_prev
    (N, M) = log qbar. anc: the ancestors of the destinations (None at t = 1); dest: the
    destinations' indices (their random-number keys; default 0..n-1). comp_in (n,) and
    bidx_in (n, M), optional: replay these mixture components and local resampling
    indices instead of drawing them; x_in (n, d1), optional: take these x_t instead.
    Returns x (n, d1), z (n, M, d2), lq (n, M), lw (n,), bidx (n, M), comp (n,), and with
    return_q also the local resampling weights log q (n, M)."""
    d1, d2 = model.d1, model.d2
    M = z_prev.shape[1]
    n = x_prev.shape[0] if anc is None else len(anc)
    dest = np.arange(n) if dest is None else np.asarray(dest)
    Lq = np.linalg.cholesky(model.Q)
    Lqx, Lqz = Lq[:d1, :d1], Lq[d1:, d1:]
    Qx = model.Q[:d1, :d1]
    y = np.asarray(y, np.float64)
    X = np.zeros((n, d1)); Z = np.zeros((n, M, d2)); LQ = np.zeros((n, M)); LW = np.zeros(n)
    B = np.zeros((n, M), np.int64); COMP = np.zeros(n, np.int64); QW = np.zeros((n, M))
    for r in range(n):
        g = int(dest[r])
        a = g if anc is None else int(anc[r])
        s = np.concatenate([np.repeat(x_prev[a][None, :], M, 0), z_prev[a]], axis=1)
        mean = transition_mean(model, s, t - 1)  # row j: E[s_t | x^a, z^(a,j)]
        qbar = np.exp(lq_prev[a] - lq_prev[a].max())
        e = oracle.normals(seed, 0, t, g, oracle.P_LA_X, 0, d1, lib)
        if gauss:
            qn = qbar / qbar.sum()
            mu = qn @ mean[:, :d1]
            dev = mean[:, :d1] - mu
            S = Qx + (dev * qn[:, None]).T @ dev
            c = -1
            xt = mu + np.linalg.cholesky(S) @ e
        else:
            if comp_in is not None:
                c = int(comp_in[r])
            else:
                c = int(oracle.sys_local(qbar, 1, _word(seed, t, g, oracle.P_LA_J), lib)[0])
            xt = mean[c, :d1] + Lqx @ e
        if x_in is not None:
            xt = np.asarray(x_in[r], np.float64)
        # q_j = qbar_j N(x_t; mean_j, Q_x)
        q = lq_prev[a] + log_gauss(xt[None, :] - mean[:, :d1], Qx)
        QW[r] = q
        if bidx_in is not None:
            b = np.asarray(bidx_in[r], np.int64)
        else:
            b = oracle.sys_local(np.exp(q - q.max()), M, _word(seed, t, g, oracle.P_INNER), lib)
        eps = np.stack([oracle.normals(seed, 0, t, g, oracle.P_PROP, j, d2, lib) for j in range(M)])
        zt = mean[b, d1:] + eps @ Lqz.T
        st = np.concatenate([np.repeat(xt[None, :], M, 0), zt], axis=1)
        ell = log_gauss(y[None, :] - obs_mean(model, st), model.R)
        lse = _lse(ell)
        X[r], Z[r], LQ[r], LW[r], B[r], COMP[r] = xt, zt, ell - lse, lse - np.log(M), b, c
    if return_q:
        return X, Z, LQ, LW, B, COMP, QW
    return X, Z, LQ, LW, B, COMP
