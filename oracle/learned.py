"""FP64 oracle of the learned inner proposal: the MLP with a Gaussian-mixture head, its
weighted negative log-likelihood, the gradients (backpropagation written out), Adam,
and the inner update of the look-ahead DPF with the learned proposal.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` may use this module; the library path never does. It imports nothing
from the CUDA package.

The proposal (not in the paper; it replaces the prior proposal of the inner
particles, the paper's step 4 of Fig. 4 with r-tilde of eq. qbar) is

    q_phi(z_t | f) = sum_c pi_c N(z_t; mu_c, diag sigma_c^2),  f = (x_{t-1}, x_t, z_{t-1}, y_t),

with [logits, mu, log sigma] the output of an MLP with `layers` hidden ReLU layers.
Head layout for C components and d2 coordinates: logits o[0:C]; mu_(c,d) =
o[C + c d2 + d]; log sigma_(c,d) = clamp(o[C + C d2 + c d2 + d], -7, 5).

With ``bf16=True`` the forward pass rounds what the GPU keeps in bfloat16 (the inputs,
the weights and every hidden activation after its ReLU: value -> float32 -> bfloat16,
round to nearest even) and accumulates exactly; biases stay full precision. The
backward pass then uses the rounded values (a straight-through rounding).
"""
from __future__ import annotations

import numpy as np

LOGSIG_MIN, LOGSIG_MAX = -7.0, 5.0
LOG2PI = np.log(2.0 * np.pi)
P_LCOMP = 10  # Philox purpose of the mixture-component draw of the learned proposal


def bf16(a):
    """Round to bfloat16 (through float32, round to nearest even); returns float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _q(a, on):
    return bf16(a) if on else np.asarray(a, dtype=np.float64)


def n_layers(W):
    return len([k for k in W if k.startswith("W")])


def forward(W, F, bf16_mode=False):
    """MLP outputs for feature rows F (n x din). Returns (out n x dout, cache)."""
    L = n_layers(W)
    h = _q(F, bf16_mode)
    cache = {"h0": h}
    for l in range(1, L + 1):
        Wl = _q(W[f"W{l}"], bf16_mode)
        pre = h @ Wl.T + W[f"b{l}"]
        cache[f"pre{l}"] = pre
        if l < L:
            h = _q(np.maximum(pre, 0.0), bf16_mode)
            cache[f"h{l}"] = h
    return pre, cache


def head(out, d2, C):
    """Mixture parameters from the head: logits (n, C), mu (n, C, d2), logsig (n, C, d2)
    clamped, and the mask of log-sigmas inside the clamp."""
    n = out.shape[0]
    logits = out[:, :C]
    mu = out[:, C:C + C * d2].reshape(n, C, d2)
    raw = out[:, C + C * d2:C + 2 * C * d2].reshape(n, C, d2)
    logsig = np.clip(raw, LOGSIG_MIN, LOGSIG_MAX)
    inside = (raw > LOGSIG_MIN) & (raw < LOGSIG_MAX)
    return logits, mu, logsig, inside


def _lse(a, axis):
    m = np.max(a, axis=axis, keepdims=True)
    return np.squeeze(m, axis) + np.log(np.sum(np.exp(a - m), axis=axis))


def component_logpdf(z, mu, logsig):
    """log N(z; mu_c, diag sigma_c^2) for every component: (n, C)."""
    u = (z[:, None, :] - mu) * np.exp(-logsig)
    return np.sum(-0.5 * u * u - logsig - 0.5 * LOG2PI, axis=2)


def logq(z, logits, mu, logsig):
    """log q(z) = LSE_c(log softmax(logits)_c + log N(z; mu_c, sigma_c^2))."""
    la = logits - _lse(logits, 1)[:, None]
    return _lse(la + component_logpdf(z, mu, logsig), 1)


def nll_and_grad(W, F, Z, w, d2, C, bf16_mode=False):
    """Weighted mean NLL  L = sum_b w_b (-log q(z_b | f_b)) / sum_b w_b  and dL/dW."""
    out, cache = forward(W, F, bf16_mode)
    logits, mu, logsig, inside = head(out, d2, C)
    n = F.shape[0]
    la = logits - _lse(logits, 1)[:, None]
    lc = la + component_logpdf(Z, mu, logsig)           # (n, C)
    lq = _lse(lc, 1)
    wn = np.asarray(w, dtype=np.float64) / np.sum(w)
    loss = -np.sum(wn * lq)
    gam = np.exp(lc - lq[:, None])                       # responsibilities
    pi = np.exp(la)
    u = (Z[:, None, :] - mu) * np.exp(-logsig)           # standardised residuals
    g_logits = pi - gam                                  # d(-log q)/d logits
    g_mu = -gam[:, :, None] * u * np.exp(-logsig)        # d(-log q)/d mu
    g_ls = -gam[:, :, None] * (u * u - 1.0) * inside     # d(-log q)/d raw log sigma
    dout = np.concatenate([g_logits, g_mu.reshape(n, -1), g_ls.reshape(n, -1)], axis=1)
    dout *= wn[:, None]
    grads = {}
    L = n_layers(W)
    d = dout
    for l in range(L, 0, -1):
        hin = cache[f"h{l - 1}"]
        grads[f"W{l}"] = d.T @ hin
        grads[f"b{l}"] = d.sum(axis=0)
        if l > 1:
            Wl = _q(W[f"W{l}"], bf16_mode)
            d = (d @ Wl) * (cache[f"pre{l - 1}"] > 0)
    return loss, grads


def adam_init(W):
    return {"t": 0, "m": {k: np.zeros_like(v) for k, v in W.items()},
            "v": {k: np.zeros_like(v) for k, v in W.items()}}


def adam_step(W, G, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) in place; returns the new weights."""
    state["t"] += 1
    t = state["t"]
    out = {}
    for k in W:
        m = state["m"][k] = b1 * state["m"][k] + (1 - b1) * G[k]
        v = state["v"][k] = b2 * state["v"][k] + (1 - b2) * G[k] * G[k]
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        out[k] = W[k] - lr * mh / (np.sqrt(vh) + eps)
    return out


def features(x_prev_a, x_new, z_b, y):
    """Input rows (x_{t-1}^(a), x_t, z_{t-1}^(a, b), y_t) of one group's M particles."""
    M = z_b.shape[0]
    return np.concatenate([np.broadcast_to(x_prev_a, (M, x_prev_a.shape[0])),
                           np.broadcast_to(x_new, (M, x_new.shape[0])), z_b,
                           np.broadcast_to(y, (M, y.shape[0]))], axis=1)


def learned_finalize(model, W, C, seed, t, y, anc, x_prev, z_prev, x_new, bidx, normals, sys_local,
                     word, bf16_mode=False, head_out=None, dest=None):
    """The inner update of step t with the learned proposal, for destinations 0..n-1.

    model: the model in x-first order (attributes d1, d2, dy, A, Q, H, R of an
    ``oracle.OracleModel``); anc[i]: the ancestor of destination i; x_new[i]: its
    selected x_t; bidx[i]: its local resampling indices (the plain rule, unchanged);
    normals(t, i, purpose, sub, n), sys_local(W, n_out, u) and word(t, i, purpose,
    sub): the shared random streams and the integer resampling rule. head_out: if
    given (n, M, dout), the MLP outputs to use instead of evaluating the network. dest:
    the destinations' indices in the filter (their random-stream keys; default 0..n-1).
    For particle j of destination i:
      z_b  = z_{t-1}^(a, bidx_j),  f = (x_{t-1}^(a), x_t^(i), z_b, y_t);
      c    = the one-draw local systematic pick over exp(logits - max), word (t, i, LCOMP, j);
      z    = mu_c + sigma_c eps,  eps = normals(t, i, PROP, j) (the prior path's noise);
      log r = log N(z; A_zx x_{t-1}^(a) + A_zz z_b, Q_z) - log q(z | f) + log p(y_t | x_t, z);
      lq   = log r - LSE_j log r.
    Returns z (n, M, d2), lq (n, M), comp (n, M), out (n, M, dout), logr (n, M)."""
    d1, d2, dy = model.d1, model.d2, model.dy
    A, Q, H, R = model.A, model.Q, model.H, model.R
    Azx, Azz = A[d1:, :d1], A[d1:, d1:]
    Qz = Q[d1:, d1:]
    Lqz = np.linalg.cholesky(Qz)
    Hx, Hz = H[:, :d1], H[:, d1:]
    Lr = np.linalg.cholesky(R)
    qc = model.qc
    n = len(anc)
    M = bidx.shape[1]
    dout = C * (1 + 2 * d2)
    zs = np.zeros((n, M, d2)); lqs = np.zeros((n, M)); comps = np.zeros((n, M), np.int32)
    outs = np.zeros((n, M, dout)); logrs = np.zeros((n, M))
    dest = np.arange(n) if dest is None else np.asarray(dest)
    for i in range(n):
        a = anc[i]
        g = int(dest[i])
        zb = z_prev[a][bidx[i]]
        f = features(x_prev[a], x_new[i], zb, y)
        out = head_out[i] if head_out is not None else forward(W, f, bf16_mode)[0]
        logits, mu, logsig, _ = head(out, d2, C)
        z = np.zeros((M, d2))
        for j in range(M):
            wts = np.exp(logits[j] - logits[j].max())
            c = int(sys_local(wts, 1, word(t, g, P_LCOMP, j))[0])
            eps = normals(t, g, 9, j, d2)  # P_PROP
            z[j] = mu[j, c] + np.exp(logsig[j, c]) * eps
            comps[i, j] = c
        lq_prop = logq(z, logits, mu, logsig)
        mp = x_prev[a] @ Azx.T + zb @ Azz.T
        rp = np.linalg.solve(Lqz, (z - mp).T).T
        lprior = -0.5 * np.sum(rp * rp, 1) - np.sum(np.log(np.diag(Lqz))) - 0.5 * d2 * LOG2PI
        hx = Hx @ x_new[i]
        if qc is not None:
            hx = hx + qc * x_new[i][:dy] ** 2
        ry = np.linalg.solve(Lr, (y - hx - z @ Hz.T).T).T
        lpy = -0.5 * np.sum(ry * ry, 1) - np.sum(np.log(np.diag(Lr))) - 0.5 * dy * LOG2PI
        lr_ = lprior - lq_prop + lpy
        zs[i] = z
        logrs[i] = lr_
        lqs[i] = lr_ - _lse(lr_[None, :], 1)[0]
        outs[i] = out
    return dict(z=zs, lq=lqs, comp=comps, out=outs, logr=logrs)


# ---------------------------------------------------------------------------
# The outer-amortised proposal: one network evaluation per outer particle gives
# a diagonal affine map of that group's prior draws.
#   group features g_i = (x_{t-1}^(a), x_t, y_t, m_i, v_i), with mu_ij the prior means
#   A_zx x_{t-1}^(a) + A_zz z_{t-1}^(a, b_ij), m_i their mean and v_i their variance
#   (per coordinate, over j); head (log s_i, c_i) (d2 each, log s clamped to [-7, 5]);
#   zhat_ij = mu_ij + L_qz eps_ij (the prior draw, PROP noise), and
#   z_ij = k_ij + c_i + s_i * (zhat_ij - k_ij),
#   log q(z_ij) = log N(zhat_ij; mu_ij, Q_z) - sum log s_i,
#   with the centre k_ij = m_i (the group's mean prior mean) or k_ij = mu_ij (the
#   particle's own prior mean: the map then scales only the transition noise).
# ---------------------------------------------------------------------------
def inner_ess(lq):
    """Inner effective sample size of each group, (sum_j W_j)^2 / sum_j W_j^2 with
    W = exp(lq) (rows of lq are groups)."""
    lq = np.asarray(lq, dtype=np.float64)
    W = np.exp(lq - lq.max(axis=1, keepdims=True))
    return W.sum(1) ** 2 / (W * W).sum(1)


def fallback_groups(lq, frac):
    """The groups whose learned inner update falls back to the plain rule: inner ESS
    below frac * M (M = the row length)."""
    return inner_ess(lq) < frac * np.asarray(lq).shape[1]


def affine_head(out, d2):
    raw = out[:, :d2]
    ls = np.clip(raw, LOGSIG_MIN, LOGSIG_MAX)
    inside = (raw > LOGSIG_MIN) & (raw < LOGSIG_MAX)
    return ls, out[:, d2:2 * d2], inside


def affine_nll_and_grad(W, G, Z, MU, MG, Qz, w, bf16_mode=False):
    """Weighted mean of -log q(z_b) for rows (group features G_b, target Z_b, prior
    mean MU_b, group centre MG_b) under the affine proposal, and dL/dW."""
    d2 = Z.shape[1]
    out, cache = forward(W, G, bf16_mode)
    ls, c, inside = affine_head(out, d2)
    s = np.exp(ls)
    zhat = MG + (Z - MG - c) / s
    Qinv = np.linalg.inv(Qz)
    r = zhat - MU
    gz = r @ Qinv.T                                            # d(1/2 r^T Q^-1 r)/d zhat
    nll = 0.5 * np.sum(r * gz, 1) + np.sum(ls, 1) + 0.5 * np.linalg.slogdet(2 * np.pi * Qz)[1]
    wn = np.asarray(w, dtype=np.float64) / np.sum(w)
    loss = float(np.sum(wn * nll))
    g_c = -gz / s                                              # dzhat/dc = -1/s
    g_ls = (-gz * (Z - MG - c) / s + 1.0) * inside             # dzhat/dls = -(z - m - c)/s
    dout = np.concatenate([g_ls, g_c], axis=1) * wn[:, None]
    grads = {}
    L = n_layers(W)
    d = dout
    for l in range(L, 0, -1):
        grads[f"W{l}"] = d.T @ cache[f"h{l - 1}"]
        grads[f"b{l}"] = d.sum(axis=0)
        if l > 1:
            d = (d @ _q(W[f"W{l}"], bf16_mode)) * (cache[f"pre{l - 1}"] > 0)
    return loss, grads


def amortised_features(model, x_prev_a, x_new, y, zb):
    """Group features and the per-particle prior means of one group (zb: M x d2 parents)."""
    d1 = model.d1
    A = model.A
    mu = x_prev_a @ A[d1:, :d1].T + zb @ A[d1:, d1:].T
    m = mu.mean(0)
    v = ((mu - m) ** 2).mean(0)
    return np.concatenate([x_prev_a, x_new, y, m, v]), mu, m


def amortised_finalize(model, W, seed, t, y, anc, x_prev, z_prev, x_new, bidx, normals, bf16_mode=False,
                       head_out=None, centre="group"):
    """The inner update of step t with the outer-amortised proposal (see above) for
    destinations 0..n-1, bidx from the plain local resampling. head_out: (n, >= 2 d2)
    network outputs to use instead of evaluating it. centre: "group" (k = m) or
    "particle" (k = mu). Returns z, lq, feats, out."""
    d1, d2, dy = model.d1, model.d2, model.dy
    Q, H, R = model.Q, model.H, model.R
    Qz = Q[d1:, d1:]
    Lqz = np.linalg.cholesky(Qz)
    Hx, Hz = H[:, :d1], H[:, d1:]
    Lr = np.linalg.cholesky(R)
    n, M = len(anc), bidx.shape[1]
    feats = np.zeros((n, 2 * d1 + dy + 2 * d2))
    mus, ms = [], []
    for i in range(n):
        a = anc[i]
        feats[i], mu, m = amortised_features(model, x_prev[a], x_new[i], y, z_prev[a][bidx[i]])
        mus.append(mu)
        ms.append(m)
    out = head_out if head_out is not None else forward(W, feats, bf16_mode)[0]
    ls, c, _ = affine_head(out, d2)
    zs = np.zeros((n, M, d2)); lqs = np.zeros((n, M))
    for i in range(n):
        eps = np.stack([normals(t, i, 9, j, d2) for j in range(M)])  # P_PROP
        zhat = mus[i] + eps @ Lqz.T
        s = np.exp(ls[i])
        k = mus[i] if centre == "particle" else ms[i]
        z = k + c[i] + s * (zhat - k)
        def lgauss(v, L):
            u = np.linalg.solve(L, v.T).T
            return -0.5 * np.sum(u * u, 1) - np.sum(np.log(np.diag(L))) - 0.5 * L.shape[0] * LOG2PI
        lprior = lgauss(z - mus[i], Lqz)
        lq_prop = lgauss(zhat - mus[i], Lqz) - np.sum(ls[i])
        hx = Hx @ x_new[i]
        if model.qc is not None:
            hx = hx + model.qc * x_new[i][:dy] ** 2
        lpy = lgauss(y - hx - z @ Hz.T, Lr)
        lr_ = lprior - lq_prop + lpy
        zs[i] = z
        lqs[i] = lr_ - _lse(lr_[None, :], 1)[0]
    return dict(z=zs, lq=lqs, feats=feats, out=out)
