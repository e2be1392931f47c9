"""Oracle of the bootstrap particle filter, the baseline the paper compares the
decentralized filters with (Section 4.1, "PF"; the sampling-importance-resampling filter
of Gordon, Salmond and Smith 1993), over the full state s = (x, z) in x-first order.

TEST INFRASTRUCTURE ONLY: the tests may use this module; the library path never does.

Step t, for particles i = 0..N-1:
  a_i = i at t = 1 (the initial draw is equally weighted), else the ancestor the global
        systematic resampling of step t-1 gave particle i;
  s_t^i = f(s_{t-1}^{a_i}, t-1) + chol(Q) e^i, with f the model's transition mean
        (A s, plus the growth map a x + b x / (1 + x^2) + c cos(w (t-1)) on the x block)
        and e^i the normals of purposes PF_X (x block) and PF_Z (z block) at counter
        (t, i, purpose, 0); Q has no x/z cross-covariance, so chol(Q) is block-diagonal;
  log w^i = log N(y_t; H s_t^i + q (x_t^i)^2 on the first d1 observations, R);
  the evidence increment is LSE_i(log w) - log N, the filtered mean sum_i W_i s_t^i with
  W normalised; the resampling of step t draws from W with the word (t, 0, OUTER, 0).
"""
from __future__ import annotations

import numpy as np

P_PF_X, P_PF_Z = 12, 13


def transition_mean(model, s, t_src):
    """E[s_t | s_{t-1} = s] for rows of s, with t_src = t - 1 the source step."""
    d1 = model.d1
    m = s @ model.A.T
    if model.growth is not None:
        a, b, c, w = model.growth
        x = s[:, :d1]
        m[:, :d1] += a * x + b * x / (1.0 + x * x) + c * np.cos(w * t_src)
    return m


def obs_mean(model, s):
    """E[y | s] for rows of s."""
    d1 = model.d1
    h = s @ model.H.T
    if model.qc is not None:
        h[:, :d1] += model.qc * s[:, :d1] ** 2
    return h


def log_gauss(r, R):
    """log N(r; 0, R) for rows r."""
    Lr = np.linalg.cholesky(R)
    u = np.linalg.solve(Lr, r.T).T
    dy = R.shape[0]
    return -0.5 * np.sum(u * u, 1) - np.sum(np.log(np.diag(Lr))) - 0.5 * dy * np.log(2.0 * np.pi)


def pf_step(model, t, y, x_prev, z_prev, anc, noise, dest=None):
    """One step from the particles of step t-1. anc: the ancestors of the destinations
    (None at t = 1: destination i starts from particle i); noise(t, i, purpose, n) gives n
    standard normals; dest: the destinations' particle indices (their noise keys; default
    0..n-1). Returns the new particles (x, z) and their log-weights."""
    d1, d2 = model.d1, model.d2
    dest = np.arange(x_prev.shape[0] if anc is None else len(anc)) if dest is None else np.asarray(dest)
    idx = dest if anc is None else np.asarray(anc)
    s_prev = np.concatenate([x_prev[idx], z_prev[idx]], axis=1)
    m = transition_mean(model, s_prev, t - 1)
    L = np.linalg.cholesky(model.Q)
    e = np.stack([np.concatenate([noise(t, int(i), P_PF_X, d1), noise(t, int(i), P_PF_Z, d2)]) for i in dest])
    s = m + e @ L.T
    lw = log_gauss(np.asarray(y, np.float64)[None, :] - obs_mean(model, s), model.R)
    return s[:, :d1], s[:, d1:], lw


def summarise(lw, x, z):
    """Evidence increment log(mean_i w_i), the weighted mean of (x, z), and the weights."""
    mx = lw.max()
    W = np.exp(lw - mx)
    W = W / W.sum()
    logz = mx + np.log(np.mean(np.exp(lw - mx)))
    return logz, W @ np.concatenate([x, z], axis=1), W
