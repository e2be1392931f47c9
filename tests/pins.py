"""Closed-form pins of the oracle's LA-DPF step, written as reusable checks.

Each ``pin_*`` returns (ok, detail). They are used by the CPU tests directly and
by the planted-mistake tests, which rebuild the oracle with a deliberate error
and require at least one pin to fail.

Pins (all for observations linear in (x, z)):

* look-ahead weight: for a fixed state, the expectation over the step's random
  draws of w^(i) = (1/L) sum_m what^(i,m) equals sum_k qbar^(i,k)
  N(y_t; H f(x^(i), z^(i,k)), H Q H^T + R). (The x draws come from the mixture
  that normalises alpha, so the ratio cancels inside the expectation over
  xbb; the projected inner draw then integrates the z noise exactly.)
* inner step: the weighted inner set after local resampling, propagation and the
  y-update targets the Gaussian-mixture posterior of z_t with component weights
  qbar^k N(x_t; f^x(x_a, z^k), Q_x) N(y_t; H_x x_t + H_z f^z, H_z Q_z H_z^T + R).
* filtered means and log-evidence of the whole filter agree with the Kalman
  filter on a linear-Gaussian model within Monte Carlo error.
"""
import numpy as np

from oracle import oracle
from paper_1203_2394_gb300 import workloads
from tests.kalman import kalman


def _mvn_logpdf(v, S):
    sign, logdet = np.linalg.slogdet(S)
    return -0.5 * np.einsum("...i,ij,...j->...", v, np.linalg.inv(S), v) - 0.5 * logdet - 0.5 * S.shape[0] * np.log(2 * np.pi)


def _state(rng, N, M, d1, d2, scale=1.0, lq_scale=1.0):
    x = rng.standard_normal((N, d1)) * scale
    z = rng.standard_normal((N, M, d2)) * scale
    lq = rng.standard_normal((N, M)) * lq_scale
    lq -= np.log(np.exp(lq).sum(1, keepdims=True))
    return x, z, lq


def _fmean(spec, x, z, s):
    d1 = spec.d1
    st = np.concatenate([np.broadcast_to(x[:, None, :], z.shape[:2] + (d1,)), z], axis=-1)
    out = st @ spec.A.T
    if spec.growth is not None:
        a, b, c, w = spec.growth
        xx = st[..., :d1]
        out[..., :d1] += a * xx + b * xx / (1 + xx * xx) + c * np.cos(w * s)
    return out


def pin_lookahead_weight(lib=None, spec_name="lg4", growth=False, reps=300, seed=11):
    spec = workloads.make_model(spec_name, 0)
    spec.Q = 0.6 * np.eye(spec.d)  # noise large enough that each noise term shows in the weight
    if growth:
        spec.growth = (0.5, 25.0, 8.0, 1.2)
    rng = np.random.default_rng(seed)
    N, M, L, t = 3, 48, 8, 4
    x, z, lq = _state(rng, N, M, spec.d1, spec.d2)
    x = x[:1] + 0.3 * (x - x[:1])  # nearby outer particles, so one y is plausible for all
    f = _fmean(spec, x, z, t - 1)  # (N, M, d)
    S = spec.H @ spec.Q @ spec.H.T + spec.R
    y = spec.H @ f[0, 0] + np.linalg.cholesky(S) @ rng.standard_normal(spec.dy)
    om = oracle.OracleModel.from_spec(spec)
    exact = (np.exp(lq) * np.exp(_mvn_logpdf(y - f @ spec.H.T, S))).sum(1)
    vals = np.zeros((reps, N))
    for r in range(reps):
        o = oracle.Oracle(om, N, M, L, seed=1000 + r, lib=lib).lookahead(t, y, np.arange(N), x, z, lq)
        vals[r] = np.exp(o["lw"])
    mean = vals.mean(0)
    se = vals.std(0, ddof=1) / np.sqrt(reps)
    zsc = np.abs(mean - exact) / se
    return bool(np.all(zsc < 4.5)), dict(mean=mean, exact=exact, z=zsc)


def pin_inner_step(lib=None, reps=60, seed=5):
    spec = workloads.make_model("lg4", 0)
    d1, d2 = spec.d1, spec.d2
    rng = np.random.default_rng(seed)
    M, t = 1024, 3
    x, z, lq = _state(rng, 1, M, d1, d2, lq_scale=0.5)
    Axx, Axz = spec.A[:d1, :d1], spec.A[:d1, d1:]
    Azx, Azz = spec.A[d1:, :d1], spec.A[d1:, d1:]
    Qx, Qz = spec.Q[:d1, :d1], spec.Q[d1:, d1:]
    Hx, Hz = spec.H[:, :d1], spec.H[:, d1:]
    fx = x[0] @ Axx.T + z[0] @ Axz.T
    fz = x[0] @ Azx.T + z[0] @ Azz.T
    # x_t drawn from the predictive mixture, y_t from the model given a nearby z_t
    k0 = rng.integers(M)
    x_new = (fx[k0] + np.linalg.cholesky(Qx) @ rng.standard_normal(d1))[None, :]
    y = Hx @ x_new[0] + Hz @ (fz[k0] + np.linalg.cholesky(Qz) @ rng.standard_normal(d2)) \
        + np.linalg.cholesky(spec.R) @ rng.standard_normal(spec.dy)
    Sy = Hz @ Qz @ Hz.T + spec.R
    r = y - Hx @ x_new[0] - fz @ Hz.T
    logpi = lq[0] + _mvn_logpdf(x_new[0] - fx, Qx) + _mvn_logpdf(r, Sy)
    pi = np.exp(logpi - logpi.max()); pi /= pi.sum()
    G = Qz @ Hz.T @ np.linalg.inv(Sy)
    comp_mean = fz + r @ G.T
    exact = pi @ comp_mean
    om = oracle.OracleModel.from_spec(spec)
    est = np.zeros((reps, d2))
    for rr in range(reps):
        o = oracle.Oracle(om, 1, M, 4, seed=77 + rr, lib=lib).finalize(
            t, y, [0], [0], x, z, lq, x_new)
        wq = np.exp(o["lq"][0])
        if abs(wq.sum() - 1) > 1e-9:
            return False, dict(reason="inner weights not normalised", sum=wq.sum())
        est[rr] = wq @ o["z"][0]
    mean = est.mean(0)
    se = est.std(0, ddof=1) / np.sqrt(reps)
    zsc = np.abs(mean - exact) / np.maximum(se, 1e-12)
    return bool(np.all(zsc < 4.5)), dict(mean=mean, exact=exact, z=zsc)


def pin_kalman(lib=None, T=12, N=384, M=48, L=8, reps=12, nthreads=8):
    spec = workloads.make_model("lg4", 0)
    _, ys = workloads.simulate(spec, T, 0)
    km, kc, kll = kalman(spec.A, spec.Q, spec.H, spec.R, spec.m0, spec.P0, ys)
    om = oracle.OracleModel.from_spec(spec)
    means = np.zeros((reps, T, spec.d))
    logz = np.zeros((reps, T))
    for r in range(reps):
        outs = oracle.Oracle(om, N, M, L, seed=r, nthreads=nthreads, lib=lib).run(ys[:T])
        means[r] = [o["mean"] for o in outs]
        logz[r] = np.cumsum([o["logZ"] for o in outs])
    err = means.mean(0) - km
    se = means.std(0, ddof=1) / np.sqrt(reps)
    sd = np.sqrt(np.einsum("tii->ti", kc))
    ok_mean = np.all(np.abs(err) < 4.5 * se + 0.05 * sd)
    lerr = logz.mean(0) - np.cumsum(kll)
    lse_ = logz.std(0, ddof=1) / np.sqrt(reps)
    ok_logz = np.all(np.abs(lerr) < 4.5 * lse_ + 0.05 * np.sqrt(np.arange(1, T + 1)))
    return bool(ok_mean and ok_logz), dict(err=err, se=se, sd=sd, lerr=lerr, lse=lse_)
