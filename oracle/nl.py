"""Oracle of the paper's benchmark models (Table 1) with the LA-DPF (Fig. 4) and the
bootstrap particle filter, in FP64 numpy.

TEST INFRASTRUCTURE ONLY: the tests, smoke() and the benchmark's CPU legs may use this
module; the library path never does.

The models, with s = (x, z) and the noise v_t ~ N(0, Sv) of Table 1:
  model 1: x' = x + z / (1 + z^2) + v_x
           z' = x + 0.5 z + 25 z / (1 + z^2) + 8 cos(1.2 t) + v_z
           y  = atan(x) + z^2 / 20 + e,    Sv = [[1, 0.1], [0.1, 1]]
  model 2: x1' = 0.5 x1 + 8 sin t + v_1,   x2' = 0.4 x1 + 0.5 x2 + v_2
           z1' = z1 + z2 / (1 + z2^2) + v_3
           z2' = z1' + 0.5 z2 + 25 z2 / (1 + z2^2) + 8 cos(1.2 t) + v_4
           y   = (x1 + x2) / (1 + x1^2) + atan(z1) + z2^2 / 20 + e,
           Sv = diag(I_2, [[1, 0.1], [0.1, 10]])
  e ~ N(0, 1); s_0 ~ N(0, I).
Readings: t in the sine and cosine is the step the transition leaves (s_{t+1} uses t);
model 2's z2' adds z1' with its noise, so the increment s' - f(s) is J v with J the
identity but J[z2, z1] = 1, and the transition's covariance is Q = J Sv J^T.

Every draw is made x first: x' = f_x + chol(Q_xx) e_x, then z' from its Gaussian
conditional given x', z' = f_z + G (x' - f_x) + chol(S) e_z with G = Q_zx Q_xx^-1 and
S = Q_zz - G Q_xz (the standard partition of a joint Gaussian).

The LA-DPF step t from the state of step t-1 (x, z, lq = log qbar), in Fig. 4's order:
  1. for each outer particle i and draw m = 0..L-1: a component j_m by the one-draw local
     systematic rule on qbar (word (t, i, LA_J, m)), xbb_m = f_x(x_i, z_ij) + chol(Q_xx) e
     (normals (t, i, LA_X, m));
  2. the pair weights over the inner particles k, with the inner draw conditioned on xbb_m
     and the noise e_k (normals (t, i, LA_Z, k)) shared by the draws:
       alpha_mk = lq_ik + log p(xbb_m | x_i, z_ik),
       zhat_mk  = f_z(x_i, z_ik) + G (xbb_m - f_x(x_i, z_ik)) + chol(S) e_k,
       lwhat_m  = LSE_k(alpha + log p(y_t | xbb_m, zhat_mk)) - LSE_k(alpha),
       lw_i     = LSE_m(lwhat_m) - log L;
  3. the outer systematic resampling of exp(lw) (word (t, 0, OUTER, 0));
  4. for each destination i with ancestor a: the draw sel_i by the one-draw local rule on
     exp(lwhat_a) (word (t, i, SEL, 0)) gives x_t = xbb_(a, sel_i); the inner particles of a
     are resampled by lq_ak + log p(x_t | x_a, z_ak) (word (t, i, INNER, 0)), propagated
     from their conditional given x_t (normals (t, i, PROP, j)) and reweighted by y_t.
The filtered mean is the look-ahead's: the pairs (i, m) weighted by exp(lwhat), with the
z part sum_k softmax_k(alpha + ell) zhat_mk.

Also the DPF without look-ahead (std_step) and the bootstrap particle filter (pf_step)
for the same models, the filters the paper compares the LA-DPF with.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle
from oracle.pf import P_PF_X, P_PF_Z


class PaperModel:
    """One of the paper's two benchmark models (kind 1 or 2), vectorised over leading axes.
    swap (model 1 only) decomposes the state the other way, Section 4.3's second action: the
    filter's x is the table's z and its z the table's x."""

    def __init__(self, kind, swap=False):
        self.kind = int(kind)
        self.swap = bool(swap)
        if self.swap and self.kind != 1:
            raise ValueError("only model 1 is decomposed both ways")
        if self.kind == 1:
            self.d1 = self.d2 = 1
            self.J = np.eye(2)
            self.Sv = np.array([[1.0, 0.1], [0.1, 1.0]])
        elif self.kind == 2:
            self.d1 = self.d2 = 2
            self.J = np.eye(4)
            self.J[3, 2] = 1.0
            self.Sv = np.zeros((4, 4))
            self.Sv[:2, :2] = np.eye(2)
            self.Sv[2:, 2:] = [[1.0, 0.1], [0.1, 10.0]]
        else:
            raise ValueError("kind must be 1 or 2")
        d1 = self.d1
        self.d = 2 * d1
        self.Q = self.J @ self.Sv @ self.J.T
        # filter coordinate c is table coordinate perm[c]
        self.perm = np.array([1, 0]) if self.swap else np.arange(self.d)
        self.Q = self.Q[np.ix_(self.perm, self.perm)]
        Qxx, Qxz, Qzz = self.Q[:d1, :d1], self.Q[:d1, d1:], self.Q[d1:, d1:]
        self.Qxx = Qxx
        self.G = Qxz.T @ np.linalg.inv(Qxx)
        self.S = Qzz - self.G @ Qxz
        self.Lqx = np.linalg.cholesky(Qxx)
        self.LS = np.linalg.cholesky(self.S)

    def transition(self, x, z, s, v=None):
        """Table 1's equations from (x, z) at step s with the noise v (None: the mean), in the
        filter's coordinates."""
        x = np.asarray(x, np.float64)
        z = np.asarray(z, np.float64)
        v = np.zeros(np.broadcast_shapes(x.shape[:-1], z.shape[:-1]) + (self.d,)) if v is None else v
        if self.swap:  # the table's (x, z) is the filter's (z, x)
            vt = np.empty_like(v)
            vt[..., self.perm] = v
            xn, zn = self._table_transition(z, x, s, vt)
            return zn, xn
        return self._table_transition(x, z, s, v)

    def _table_transition(self, x, z, s, v):
        if self.kind == 1:
            xs, zs = x[..., 0], z[..., 0]
            xn = xs + zs / (1 + zs ** 2) + v[..., 0]
            zn = xs + 0.5 * zs + 25 * zs / (1 + zs ** 2) + 8 * np.cos(1.2 * s) + v[..., 1]
            return xn[..., None], zn[..., None]
        x1, x2, z1, z2 = x[..., 0], x[..., 1], z[..., 0], z[..., 1]
        x1n = 0.5 * x1 + 8 * np.sin(s) + v[..., 0]
        x2n = 0.4 * x1 + 0.5 * x2 + v[..., 1]
        z1n = z1 + z2 / (1 + z2 ** 2) + v[..., 2]
        z2n = z1n + 0.5 * z2 + 25 * z2 / (1 + z2 ** 2) + 8 * np.cos(1.2 * s) + v[..., 3]
        return np.stack([x1n, x2n], -1), np.stack([z1n, z2n], -1)

    def h(self, x, z):
        if self.swap:
            x, z = z, x
        if self.kind == 1:
            return np.arctan(x[..., 0]) + z[..., 0] ** 2 / 20
        return (x[..., 0] + x[..., 1]) / (1 + x[..., 0] ** 2) + np.arctan(z[..., 0]) + z[..., 1] ** 2 / 20

    def log_py(self, y, x, z):
        """log N(y; h(x, z), 1) (y a scalar)."""
        r = float(y) - self.h(x, z)
        return -0.5 * np.log(2 * np.pi) - 0.5 * r * r

    def log_px(self, xn, fx):
        """log N(xn; fx, Q_xx)."""
        r = np.linalg.solve(self.Lqx, (xn - fx)[..., None])[..., 0]
        return (-0.5 * np.sum(r * r, -1) - np.sum(np.log(np.diag(self.Lqx)))
                - 0.5 * self.d1 * np.log(2 * np.pi))

    def draw_x(self, fx, e):
        return fx + e @ self.Lqx.T

    def draw_z(self, fz, fx, xn, e):
        """z' given x': f_z + G (x' - f_x) + chol(S) e."""
        return fz + (xn - fx) @ self.G.T + e @ self.LS.T


def _word(seed, t, i, purpose, sub=0, lib=None):
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return int(oracle.philox((t, i, (purpose << 24) | sub, 0), key, lib)[0])


def _lse(v, axis=-1):
    m = np.max(v, axis=axis, keepdims=True)
    m = np.where(np.isfinite(m), m, 0.0)
    return np.squeeze(m, axis) + np.log(np.sum(np.exp(v - m), axis=axis))


def init(model, N, M, seed, lib):
    """s_0 ~ N(0, I): x_0 from the normals (0, i, INIT_X, 0), z_0^(i,j) from (0, i, INIT_Z, j)."""
    i = np.arange(N)
    x = oracle.normals_many(seed, 0, 0, i, oracle.P_INIT_X, 0, model.d1, lib)
    z = oracle.normals_many(seed, 0, 0, np.repeat(i, M), oracle.P_INIT_Z, np.tile(np.arange(M), N),
                            model.d2, lib).reshape(N, M, model.d2)
    return x, z, np.full((N, M), -np.log(M))


def lookahead(model, seed, t, y, x, z, lq, L, idx, lib, jla_in=None):
    """Steps 1-2 of Fig. 4 for the outer particles idx from the state of step t-1.
    jla_in (optional, (n, L)): replay these mixture components instead of drawing them.
    Returns lw (n,), lwhat (n, L), xbb (n, L, d1), jla (n, L), mu (n, L, d2)."""
    d1, d2, M = model.d1, model.d2, z.shape[1]
    n = len(idx)
    lw = np.zeros(n); lwhat = np.zeros((n, L)); xbb = np.zeros((n, L, d1))
    jla = np.zeros((n, L), np.int64); mu = np.zeros((n, L, d2))
    for q, i in enumerate(idx):
        i = int(i)
        fx, fz = model.transition(x[i][None, :], z[i], t - 1)  # (M, d1), (M, d2)
        qbar = np.exp(lq[i] - lq[i].max())
        for m in range(L):
            if jla_in is not None:
                jla[q, m] = int(jla_in[q][m])
            else:
                jla[q, m] = oracle.sys_local(qbar, 1, _word(seed, t, i, oracle.P_LA_J, m, lib), lib)[0]
        e = oracle.normals_many(seed, 0, t, np.full(L, i), oracle.P_LA_X, np.arange(L), d1, lib)
        xb = model.draw_x(fx[jla[q]], e)  # (L, d1)
        ek = oracle.normals_many(seed, 0, t, np.full(M, i), oracle.P_LA_Z, np.arange(M), d2, lib)
        alpha = lq[i][None, :] + model.log_px(xb[:, None, :], fx[None, :, :])  # (L, M)
        zh = model.draw_z(fz[None], fx[None], xb[:, None, :], ek[None])  # (L, M, d2)
        a1 = alpha + model.log_py(y, np.broadcast_to(xb[:, None, :], zh.shape[:2] + (d1,)), zh)
        l1 = _lse(a1)
        lwhat[q] = l1 - _lse(alpha)
        lw[q] = _lse(lwhat[q]) - np.log(L)
        xbb[q] = xb
        mu[q] = np.einsum("mk,mkc->mc", np.exp(a1 - l1[:, None]), zh)
    return lw, lwhat, xbb, jla, mu


def finalize(model, seed, t, y, idx, anc, x_prev, z_prev, lq_prev, x_new, lib, bidx_in=None,
             return_alpha=False):
    """Step 4's inner update for the destinations idx with ancestors anc and new x_t.
    bidx_in (optional, (n, M)): replay these local resampling indices.
    Returns z (n, M, d2), lq (n, M), bidx (n, M) and, with return_alpha, the local
    resampling weights alpha (n, M)."""
    d2, M = model.d2, z_prev.shape[1]
    n = len(idx)
    Z = np.zeros((n, M, d2)); LQ = np.zeros((n, M)); B = np.zeros((n, M), np.int64)
    AL = np.zeros((n, M))
    for q in range(n):
        i, a = int(idx[q]), int(anc[q])
        fx, fz = model.transition(x_prev[a][None, :], z_prev[a], t - 1)
        alpha = lq_prev[a] + model.log_px(x_new[q][None, :], fx)
        AL[q] = alpha
        if bidx_in is not None:
            b = np.asarray(bidx_in[q], np.int64)
        else:
            b = oracle.sys_local(np.exp(alpha - alpha.max()), M, _word(seed, t, i, oracle.P_INNER, 0, lib), lib)
        e = oracle.normals_many(seed, 0, t, np.full(M, i), oracle.P_PROP, np.arange(M), d2, lib)
        zt = model.draw_z(fz[b], fx[b], x_new[q][None, :], e)
        ell = model.log_py(y, np.broadcast_to(x_new[q], (M, model.d1)), zt)
        Z[q], LQ[q], B[q] = zt, ell - _lse(ell), b
    if return_alpha:
        return Z, LQ, B, AL
    return Z, LQ, B


def step(model, seed, t, y, x, z, lq, L, lib):
    """One LA-DPF step (Fig. 4) from the state of step t-1; returns the state of step t,
    the filtered mean (d1 + d2), log p(y_t | y_1:t-1) and the intermediate products."""
    N = x.shape[0]
    idx = np.arange(N)
    lw, lwhat, xbb, jla, mu = lookahead(model, seed, t, y, x, z, lq, L, idx, lib)
    logZ = _lse(lw) - np.log(N)
    W = np.exp(lwhat - lwhat.max())
    W /= W.sum()
    mean = np.concatenate([np.einsum("nm,nmc->c", W, xbb), np.einsum("nm,nmc->c", W, mu)])
    anc = oracle.sys_global(np.exp(lw - lw.max()), _word(seed, t, 0, oracle.P_OUTER, 0, lib), lib)
    sel = np.array([oracle.sys_local(np.exp(lwhat[a] - lwhat[a].max()), 1,
                                     _word(seed, t, i, oracle.P_SEL, 0, lib), lib)[0]
                    for i, a in enumerate(anc)])
    x_new = xbb[anc, sel]
    z_new, lq_new, bidx = finalize(model, seed, t, y, idx, anc, x, z, lq, x_new, lib)
    return dict(x=x_new, z=z_new, lq=lq_new, mean=mean, logZ=logZ, lw=lw, lwhat=lwhat, xbb=xbb,
                jla=jla, anc=anc, sel=sel, bidx=bidx)


def run_la_dpf(model, seed, ys, N, M, L, lib):
    """Filtered means (T, d) and log-evidence increments of the LA-DPF over y_1..y_T."""
    x, z, lq = init(model, N, M, seed, lib)
    means, lz = [], []
    for t, y in enumerate(ys, start=1):
        o = step(model, seed, t, float(np.ravel(y)[0]), x, z, lq, L, lib)
        x, z, lq = o["x"], o["z"], o["lq"]
        means.append(o["mean"]); lz.append(o["logZ"])
    return np.array(means), np.array(lz)


def std_step(model, seed, t, y, x_prev, z_prev, lq_prev, anc, lib, dest=None, gauss=False, comp_in=None,
             bidx_in=None, return_picks=False, x_in=None):
    """The DPF without look-ahead (the paper's Fig. dpf with the prior as both proposals),
    call t for the destinations dest (default 0..n-1) with ancestors anc (None at t = 1):
      x_t ~ sum_j qbar_j N(f_x(x_a, z_aj), Q_xx): a component by the one-draw local rule
            (word (t, i, LA_J, 0)), then f_x of it + chol(Q_xx) e (normals (t, i, LA_X, 0));
            with gauss, the mixture's moment-matched Gaussian instead (Section 4.2): mean
            mu = sum_j qbar_j f_x,j, covariance Q_xx + sum_j qbar_j (f_x,j - mu)(f_x,j - mu)^T;
      b = local systematic resampling by lq_aj + log N(x_t; f_x,j, Q_xx) (word (t, i, INNER, 0));
      z_t^j from the transition's conditional given x_t out of z_ab_j (normals (t, i, PROP, j));
      lq = ell - LSE ell with ell = log p(y_t | x_t, z_t^j); log w = LSE ell - log M.
    comp_in (n,) and bidx_in (n, M), optional: replay these components and local indices;
    x_in (n, d1), optional: take these x_t instead of the draws.
    Returns x (n, d1), z (n, M, d2), lq (n, M), lw (n,); with return_picks also the
    components (n,; -1 for the Gaussian form), the local indices (n, M) and the local
    resampling weights alpha (n, M)."""
    d1, d2, M = model.d1, model.d2, z_prev.shape[1]
    n = x_prev.shape[0] if anc is None else len(anc)
    dest = np.arange(n) if dest is None else np.asarray(dest)
    X = np.zeros((n, d1)); Z = np.zeros((n, M, d2)); LQ = np.zeros((n, M)); LW = np.zeros(n)
    COMP = np.full(n, -1, np.int64); B = np.zeros((n, M), np.int64); AL = np.zeros((n, M))
    for r in range(n):
        i = int(dest[r])
        a = i if anc is None else int(anc[r])
        fx, fz = model.transition(x_prev[a][None, :], z_prev[a], t - 1)
        qbar = np.exp(lq_prev[a] - lq_prev[a].max())
        e = oracle.normals(seed, 0, t, i, oracle.P_LA_X, 0, d1, lib)
        if gauss:
            qn = qbar / qbar.sum()
            mu = qn @ fx
            dev = fx - mu
            xt = mu + np.linalg.cholesky(model.Qxx + (dev * qn[:, None]).T @ dev) @ e
        else:
            if comp_in is not None:
                c = int(comp_in[r])
            else:
                c = int(oracle.sys_local(qbar, 1, _word(seed, t, i, oracle.P_LA_J, 0, lib), lib)[0])
            COMP[r] = c
            xt = model.draw_x(fx[c], e)
        if x_in is not None:
            xt = np.asarray(x_in[r], np.float64)
        alpha = lq_prev[a] + model.log_px(xt[None, :], fx)
        AL[r] = alpha
        if bidx_in is not None:
            b = np.asarray(bidx_in[r], np.int64)
        else:
            b = oracle.sys_local(np.exp(alpha - alpha.max()), M, _word(seed, t, i, oracle.P_INNER, 0, lib), lib)
        B[r] = b
        eps = oracle.normals_many(seed, 0, t, np.full(M, i), oracle.P_PROP, np.arange(M), d2, lib)
        zt = model.draw_z(fz[b], fx[b], xt[None, :], eps)
        ell = model.log_py(y, np.broadcast_to(xt, (M, d1)), zt)
        l = _lse(ell)
        X[r], Z[r], LQ[r], LW[r] = xt, zt, ell - l, l - np.log(M)
    if return_picks:
        return X, Z, LQ, LW, COMP, B, AL
    return X, Z, LQ, LW


def run_std(model, seed, ys, N, M, lib, gauss=False):
    """Filtered means (T, d) and log-evidence increments of the DPF without look-ahead,
    resampling the outer particles every call (word (t, 0, OUTER, 0)); the mean weighs
    each outer particle by its weight, with the z part sum_j qbar_j z_j."""
    x, z, lq = init(model, N, M, seed, lib)
    anc = None
    means, lz = [], []
    for t, y in enumerate(ys, start=1):
        x, z, lq, lw = std_step(model, seed, t, float(np.ravel(y)[0]), x, z, lq, anc, lib, gauss=gauss)
        W = np.exp(lw - lw.max())
        zm = np.einsum("nm,nmc->nc", np.exp(lq), z)
        means.append(np.concatenate([W @ x, W @ zm]) / W.sum())
        lz.append(_lse(lw) - np.log(N))
        anc = oracle.sys_global(W, _word(seed, t, 0, oracle.P_OUTER, 0, lib), lib)
    return np.array(means), np.array(lz)


def pf_step(model, seed, t, y, x, z, anc, lib, dest=None):
    """The bootstrap particle filter's step t: each destination i draws from the transition
    out of its ancestor (itself at t = 1), x first (normals (t, i, PF_X, 0)), then z given x
    (normals (t, i, PF_Z, 0)), and is weighted by p(y_t | x, z).
    x (N, d1), z (N, d2); returns x, z, lw of the destinations."""
    n = x.shape[0] if anc is None else len(anc)
    dest = np.arange(n) if dest is None else np.asarray(dest)
    src = dest if anc is None else np.asarray(anc)
    fx, fz = model.transition(x[src], z[src], t - 1)
    ex = oracle.normals_many(seed, 0, t, dest, P_PF_X, 0, model.d1, lib)
    ez = oracle.normals_many(seed, 0, t, dest, P_PF_Z, 0, model.d2, lib)
    xn = model.draw_x(fx, ex)
    zn = model.draw_z(fz, fx, xn, ez)
    return xn, zn, model.log_py(y, xn, zn)


def run_pf(model, seed, ys, N, lib):
    """Filtered means (T, d), log-evidence increments (T,) and posterior standard
    deviations (T, d) of the bootstrap particle filter, resampling every step (word
    (t, 0, OUTER, 0)); its initial particles are the LA-DPF's x_0 with the first inner
    particle z_0^(i,0)."""
    x, z, _ = init(model, N, 1, seed, lib)
    z = z[:, 0, :]
    anc = None
    means, lz, sds = [], [], []
    for t, y in enumerate(ys, start=1):
        x, z, lw = pf_step(model, seed, t, float(np.ravel(y)[0]), x, z, anc, lib)
        W = np.exp(lw - lw.max())
        s = np.concatenate([x, z], 1)
        m = W @ s / W.sum()
        means.append(m)
        sds.append(np.sqrt(W @ (s - m) ** 2 / W.sum()))
        lz.append(_lse(lw) - np.log(N))
        anc = oracle.sys_global(W, _word(seed, t, 0, oracle.P_OUTER, 0, lib), lib)
    return np.array(means), np.array(lz), np.array(sds)
