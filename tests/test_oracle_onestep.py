"""Deterministic pins of the oracle's LA-DPF step (no GPU).

1. One full step at N = 2, M = 3, L = 2 on the linear-Gaussian model lg4 (d = 4,
   x = 2 / z = 2), evaluated independently here in 50-digit arithmetic (mpmath) from
   the definitions of Fig. 4 and the readings the oracle follows, and fed the same
   Philox words (the generator itself is pinned to cuRAND in test_oracle_rng.py):
   every resampling index equal, log w, log w-hat, x_t, z_t, lq_t, the filtered
   mean and the evidence within 1e-13 (relative, floor 1).
2. The projected look-ahead draw (the inner draw enters the observation only through
   H_z zbb, so that projection is drawn with covariance H_z Q_z H_z^T, and the z-mean
   uses E[zbb | H_z zbb]) against the plain draw of the full zbb: the outer weight w
   and the z-mean estimator mu have the same expectation, within Monte Carlo error.
"""
import mpmath as mp
import numpy as np

from oracle import oracle
from paper_1203_2394_gb300 import workloads

P_LA_J, P_LA_X, P_LA_Z, P_OUTER, P_SEL, P_INNER, P_PROP = (
    oracle.P_LA_J, oracle.P_LA_X, oracle.P_LA_Z, oracle.P_OUTER, oracle.P_SEL, oracle.P_INNER, oracle.P_PROP)


# ---------------------------------------------------------------- 50-digit step
class Ref:
    """Fig. 4's step for a linear-Gaussian model, written out in mpmath."""

    def __init__(self, spec, seed):
        mp.mp.dps = 50
        d1, d = spec.d1, spec.d
        self.d1, self.d2, self.dy = d1, d - d1, spec.dy
        M_ = lambda a: mp.matrix([[mp.mpf(float(v)) for v in row] for row in np.atleast_2d(a)])
        A, Q, H, R = spec.A, spec.Q, spec.H, spec.R
        self.Axx, self.Axz = M_(A[:d1, :d1]), M_(A[:d1, d1:])
        self.Azx, self.Azz = M_(A[d1:, :d1]), M_(A[d1:, d1:])
        self.Qx, self.Qz = M_(Q[:d1, :d1]), M_(Q[d1:, d1:])
        self.Hx, self.Hz, self.R = M_(H[:, :d1]), M_(H[:, d1:]), M_(R)
        self.Lqx, self.Lqz = mp.cholesky(self.Qx), mp.cholesky(self.Qz)
        S = self.Hz * self.Qz * self.Hz.T  # covariance of the projected draw
        self.Ls = mp.cholesky(S)
        self.K = self.Qz * self.Hz.T * mp.inverse(S)
        self.key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)

    # random words and normals (Box-Muller on two words, u = ((w >> 9) + 1/2) 2^-23)
    def words(self, t, i, purpose, sub, block=0):
        return [int(v) for v in oracle.philox((t, i, (purpose << 24) | sub, block), self.key)]

    @staticmethod
    def bm(wa, wb):
        ua = (mp.mpf(wa >> 9) + mp.mpf(1) / 2) * mp.mpf(2) ** -23
        ub = (mp.mpf(wb >> 9) + mp.mpf(1) / 2) * mp.mpf(2) ** -23
        r = mp.sqrt(-2 * mp.log(ua))
        return r * mp.cos(2 * mp.pi * ub), r * mp.sin(2 * mp.pi * ub)

    def normals(self, t, i, purpose, sub, n):
        out, w = [], None
        for p in range((n + 1) // 2):
            if p % 2 == 0:
                w = self.words(t, i, purpose, sub, p // 2)
            out += list(self.bm(w[2 * (p % 2)], w[2 * (p % 2) + 1]))
        return mp.matrix(out[:n])

    def la_z_normals(self, t, i, k):
        # dy <= 2: inner particles 2h and 2h+1 share the block of sub = h
        w = self.words(t, i, P_LA_Z, k >> 1)
        q = 2 * (k & 1)
        return mp.matrix(list(self.bm(w[q], w[q + 1]))[:self.dy])

    # the exact integer systematic rule
    @staticmethod
    def systematic(W, n_out, u, rule):
        n = len(W)
        B = max(0, int(np.ceil(np.log2(n)))) if n > 1 else 0
        S = (62 if rule == "global" else 31) - B
        b = 32 if (rule == "global" or n_out == 1) else 16
        ub = u if b == 32 else u >> 16
        e = mp.frexp(max(W))[1] - 1
        cum, acc = [], 0
        for w in W:
            acc += int(mp.floor(mp.ldexp(w, S - e)))
            cum.append(acc)
        C = cum[-1]
        out, i = [], 0
        for k in range(n_out):
            rhs = (k * 2 ** b + ub) * C
            while cum[i] * n_out * 2 ** b <= rhs:
                i += 1
            out.append(i)
        return out

    @staticmethod
    def lse(v):
        m = max(v)
        return m + mp.log(mp.fsum(mp.exp(a - m) for a in v))

    @staticmethod
    def log_normal(v, L):
        # log N(v; 0, L L^T)
        sol = mp.lu_solve(L, v)
        n = v.rows
        return (-mp.mpf(1) / 2 * mp.fsum(sol[q] ** 2 for q in range(n))
                - mp.fsum(mp.log(L[q, q]) for q in range(n)) - n * mp.log(2 * mp.pi) / 2)

    def step(self, t, y, x, z, lq, N, M, L):
        v = lambda a: mp.matrix([mp.mpf(float(q)) for q in np.ravel(a)])
        y = v(y)
        X = [v(x[i]) for i in range(N)]
        Z = [[v(z[i, k]) for k in range(M)] for i in range(N)]
        LQ = [[mp.mpf(float(lq[i, k])) for k in range(M)] for i in range(N)]
        Lr = mp.cholesky(self.R)
        fx = lambda xi, zk: self.Axx * xi + self.Axz * zk
        fz = lambda xi, zk: self.Azx * xi + self.Azz * zk
        xbb, lwhat, mu, lw = [], [], [], []
        for i in range(N):
            mx = max(LQ[i])
            Wq = [mp.exp(a - mx) for a in LQ[i]]
            # step 1: the L draws from the mixture sum_j qbar_j p(x_t | x, z_j)
            xb = []
            for m in range(L):
                j = self.systematic(Wq, 1, self.words(t, i, P_LA_J, m)[0], "local")[0]
                xb.append(fx(X[i], Z[i][j]) + self.Lqx * self.normals(t, i, P_LA_X, m, self.d1))
            # the inner draws, projected: g_k = H_z f^z_k + chol(H_z Q_z H_z^T) e_k
            g, zm = [], []
            for k in range(M):
                f = fz(X[i], Z[i][k])
                e = self.Ls * self.la_z_normals(t, i, k)
                g.append(self.Hz * f + e)
                zm.append(f + self.K * e)  # E[zbb_k | g_k]
            # step 2: the weights (self-normalised over the weighted inner draws)
            lh, mus = [], []
            for m in range(L):
                a = [LQ[i][k] + self.log_normal(xb[m] - fx(X[i], Z[i][k]), self.Lqx) for k in range(M)]
                al = [a[k] + self.log_normal(y - self.Hx * xb[m] - g[k], Lr) for k in range(M)]
                lh.append(self.lse(al) - self.lse(a))
                s = self.lse(al)
                mus.append(sum((mp.exp(al[k] - s) * zm[k] for k in range(M)), mp.matrix(self.d2, 1)))
            xbb.append(xb)
            lwhat.append(lh)
            mu.append(mus)
            lw.append(self.lse(lh) - mp.log(L))
        logZ = self.lse(lw) - mp.log(N)
        # the filtered mean: every (i, m) weighted by exp(lwhat)
        top = max(max(r) for r in lwhat)
        Wim = [[mp.exp(lwhat[i][m] - top) for m in range(L)] for i in range(N)]
        sw = mp.fsum(mp.fsum(r) for r in Wim)
        mean_x = sum((Wim[i][m] * xbb[i][m] for i in range(N) for m in range(L)), mp.matrix(self.d1, 1)) / sw
        mean_z = sum((Wim[i][m] * mu[i][m] for i in range(N) for m in range(L)), mp.matrix(self.d2, 1)) / sw
        # step 3: outer resampling
        lmax = max(lw)
        anc = self.systematic([mp.exp(a - lmax) for a in lw], N, self.words(t, 0, P_OUTER, 0)[0], "global")
        # step 4: selection, local resampling, propagation, measurement update
        sel, bidx, xn, zn, lqn = [], [], [], [], []
        for i in range(N):
            a = anc[i]
            lm = max(lwhat[a])
            ms = self.systematic([mp.exp(q - lm) for q in lwhat[a]], 1, self.words(t, i, P_SEL, 0)[0], "local")[0]
            xt = xbb[a][ms]
            alpha = [LQ[a][k] + self.log_normal(xt - fx(X[a], Z[a][k]), self.Lqx) for k in range(M)]
            am = max(alpha)
            b = self.systematic([mp.exp(q - am) for q in alpha], M, self.words(t, i, P_INNER, 0)[0], "local")
            zt = [fz(X[a], Z[a][b[j]]) + self.Lqz * self.normals(t, i, P_PROP, j, self.d2) for j in range(M)]
            ell = [self.log_normal(y - self.Hx * xt - self.Hz * zt[j], Lr) for j in range(M)]
            s = self.lse(ell)
            sel.append(ms)
            bidx.append(b)
            xn.append(xt)
            zn.append(zt)
            lqn.append([q - s for q in ell])
        f = lambda a: np.array([float(q) for q in a])
        return dict(
            lw=f(lw), lwhat=np.array([f(r) for r in lwhat]), logZ=float(logZ),
            mean=np.concatenate([f(mean_x), f(mean_z)]), anc=np.array(anc), sel=np.array(sel),
            bidx=np.array(bidx), x=np.array([f(q) for q in xn]),
            z=np.array([[f(q) for q in r] for r in zn]), lq=np.array([f(r) for r in lqn]),
            xbb=np.array([[f(q) for q in r] for r in xbb]))


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b)))


def test_one_step_against_50_digit_arithmetic():
    spec = workloads.make_model("lg4", 0)
    N, M, L, seed = 2, 3, 2, 29
    _, ys = workloads.simulate(spec, 2, 4)
    o = oracle.Oracle(oracle.OracleModel.from_spec(spec), N, M, L, seed)
    x, z, lq = o.init()
    s1 = o.step(1, ys[0], x, z, lq)  # a state with unequal inner weights
    ref = Ref(spec, seed)
    for t, (xs, zs, lqs) in ((1, (x, z, lq)), (2, (s1["x"], s1["z"], s1["lq"]))):
        got = o.step(t, ys[t - 1], xs, zs, lqs)
        r = ref.step(t, ys[t - 1], xs, zs, lqs, N, M, L)
        for k in ("anc", "sel", "bidx"):
            np.testing.assert_array_equal(got[k], r[k], err_msg=f"{k} t={t}")
        for k in ("lw", "lwhat", "xbb", "x", "z", "lq", "mean"):
            assert _rel(got[k], r[k]) <= 1e-13, (k, t, _rel(got[k], r[k]))
        assert abs(got["logZ"] - r["logZ"]) <= 1e-13 * max(1.0, abs(r["logZ"])), t
        # the step is not degenerate: distinct inner weights and several distinct ancestors
        assert np.ptp(lqs) > 0 or t == 1


# ---------------------------------------------------------------- the projected draw
def test_projected_draw_matches_the_plain_draw_in_expectation():
    """For a fixed state, the outer weight w = exp(log w) and the z-mean estimator of
    the look-ahead, averaged over R independent step keys: the oracle (projected draw,
    Rao-Blackwellised z-mean) against a plain look-ahead written here that draws the
    full zbb ~ N(f^z, Q_z) and evaluates p(y | xbb, zbb) directly (same x draws). The
    two laws of w are equal, and E[mu] is the same: the means agree within 4.5
    standard errors; a plain draw without the projection's noise is far off."""
    import dataclasses
    base = workloads.make_model("lg4", 0)
    # Q_z = 2 I (instead of 0.1 I): the inner draw's noise then moves the weights enough
    # for the planted mistake below to show
    Q2 = base.Q.copy()
    Q2[base.d1:, base.d1:] = 2.0 * np.eye(base.d - base.d1)
    spec = dataclasses.replace(base, Q=Q2)
    d1, d2 = spec.d1, spec.d2
    N, M, L, R = 1, 16, 4, 3000
    _, ys = workloads.simulate(spec, 1, 9)
    y = ys[0]
    rng = np.random.default_rng(5)
    x = rng.normal(size=(N, d1))
    z = rng.normal(size=(N, M, d2))
    lq = rng.normal(size=(N, M))
    lq -= np.log(np.exp(lq).sum(axis=1, keepdims=True))
    A, Q, H, Rm = spec.A, spec.Q, spec.H, spec.R
    Axx, Axz, Azx, Azz = A[:d1, :d1], A[:d1, d1:], A[d1:, :d1], A[d1:, d1:]
    Qx, Qz = Q[:d1, :d1], Q[d1:, d1:]
    Hx, Hz = H[:, :d1], H[:, d1:]
    Lqz = np.linalg.cholesky(Qz)
    Qxi, Ri = np.linalg.inv(Qx), np.linalg.inv(Rm)
    om = oracle.OracleModel.from_spec(spec)
    w_proj, mu_proj, w_plain, mu_plain, w_bad = [], [], [], [], []
    fz = z[0] @ Azz.T + x[0] @ Azx.T  # f^z of each inner particle
    fxk = z[0] @ Axz.T + x[0] @ Axx.T  # f^x of each inner particle
    for r in range(R):
        o = oracle.Oracle(om, N, M, L, seed=1000 + r)
        out = o.lookahead(1, y, np.arange(N), x, z, lq)
        w_proj.append(np.exp(out["lw"][0]))
        Wm = np.exp(out["lwhat"][0] - out["lwhat"][0].max())
        mu_proj.append((Wm[:, None] * out["mu"][0]).sum(0) / Wm.sum())
        # the plain look-ahead on the oracle's own x draws, full zbb drawn here
        zbb = fz + rng.normal(size=(M, d2)) @ Lqz.T
        lwh, mus, lwh_bad = [], [], []
        for m in range(L):
            xb = out["xbb"][0, m]
            dx = xb - fxk
            a = lq[0] - 0.5 * np.einsum("kc,cd,kd->k", dx, Qxi, dx)
            res = y - Hx @ xb - zbb @ Hz.T
            al = a - 0.5 * np.einsum("kc,cd,kd->k", res, Ri, res)
            lwh.append(np.logaddexp.reduce(al) - np.logaddexp.reduce(a))
            sm = np.exp(al - al.max())
            mus.append((sm[:, None] * zbb).sum(0) / sm.sum())
            res0 = y - Hx @ xb - fz @ Hz.T  # planted: the inner draw without its noise
            al0 = a - 0.5 * np.einsum("kc,cd,kd->k", res0, Ri, res0)
            lwh_bad.append(np.logaddexp.reduce(al0) - np.logaddexp.reduce(a))
        lwh = np.array(lwh)
        # both carry the observation density's constant; the plain sum here omits it
        const = -0.5 * spec.dy * np.log(2 * np.pi) - 0.5 * np.log(np.linalg.det(Rm))
        w_plain.append(np.exp(np.logaddexp.reduce(lwh) - np.log(L) + const))
        w_bad.append(np.exp(np.logaddexp.reduce(np.array(lwh_bad)) - np.log(L) + const))
        Wp = np.exp(lwh - lwh.max())
        mu_plain.append((Wp[:, None] * np.array(mus)).sum(0) / Wp.sum())
    w_proj, w_plain, w_bad = map(np.array, (w_proj, w_plain, w_bad))
    mu_proj, mu_plain = np.array(mu_proj), np.array(mu_plain)

    def agree(a, b, k=4.5):
        se = np.sqrt(a.var(axis=0) / len(a) + b.var(axis=0) / len(b))
        return np.all(np.abs(a.mean(axis=0) - b.mean(axis=0)) <= k * se), np.abs(a.mean(0) - b.mean(0)) / se

    ok, zs = agree(w_proj, w_plain)
    assert ok, zs
    ok, zs = agree(mu_proj, mu_plain)
    assert ok, zs
    bad, zs = agree(w_proj, w_bad, 10.0)
    assert not bad, zs  # the noise-free inner draw is caught
