"""The oracle of the DPF without look-ahead (oracle/std_dpf.py) against closed forms (CPU).

On lg4 the filtered means track the Kalman filter within a fraction of the posterior
standard deviation and a transposed transition matrix is caught; on the growth model the
means agree with the bootstrap particle filter's oracle, an independently coded estimator
of the same posterior mean.
"""
import numpy as np

from oracle import oracle, pf, std_dpf
from paper_1203_2394_gb300 import workloads
from tests.gpu_util import word
from tests.kalman import kalman
from tests.test_oracle_pf import run_pf


def run_std(model, seed, N, M, ys, lib):
    o = oracle.Oracle(model, N, M, 1, seed, nthreads=8, lib=lib)
    x, z, lq = o.init()
    anc, means = None, []
    for t in range(1, len(ys) + 1):
        x, z, lq, lw, _, _ = std_dpf.std_step(model, seed, t, ys[t - 1], x, z, lq, anc, lib)
        W = np.exp(lw - lw.max())
        W /= W.sum()
        zmean = np.einsum("nm,nmc->nc", np.exp(lq), z)
        means.append(np.concatenate([W @ x, W @ zmean]))
        anc = oracle.sys_global(W, word(seed, t, 0, oracle.P_OUTER), lib)
    return np.array(means)


def test_std_dpf_tracks_kalman_and_sees_a_transposed_transition(oracle_lib):
    spec = workloads.make_model("lg4", 0)
    om = oracle.OracleModel.from_spec(spec)
    _, ys = workloads.simulate(spec, 10, 3)
    km, kP, _ = kalman(spec.A, spec.Q, spec.H, spec.R, spec.m0, spec.P0, ys)
    sd = np.sqrt(np.stack([np.diag(P) for P in kP]))
    err = np.max(np.abs(run_std(om, 4, 1500, 32, ys, oracle_lib) - km) / sd)
    assert err < 0.25, err
    bad = oracle.OracleModel(om.d1, om.d2, om.dy, om.A.T, om.Q, om.H, om.R, om.m0, om.P0)
    assert np.max(np.abs(run_std(bad, 4, 1500, 32, ys, oracle_lib) - km) / sd) > 0.5


def test_std_dpf_agrees_with_the_pf_oracle_on_the_growth_model(oracle_lib):
    spec = workloads.make_model("growth_clg10", 0)
    om = oracle.OracleModel.from_spec(spec)
    _, ys = workloads.simulate(spec, 6, 0)
    ref, _ = run_pf(om, 21, 20000, ys, oracle_lib)
    sd = run_pf.sd
    got = run_std(om, 5, 1500, 32, ys, oracle_lib)
    z = np.abs(got - ref) / sd
    assert np.max(z) < 0.3, np.round(z.max(axis=0), 3)


def test_gaussian_approximation_moments_and_tracking(oracle_lib):
    """The Gaussian approximation: for a model whose x transition is free of z it draws
    exactly what the mixture does; on lg4 (x depends on z) the drawn x_t over many keys has
    the mixture's mean and covariance (the mixture's, computed by enumerating its
    components), and the filter still tracks the Kalman filter."""
    spec = workloads.make_model("growth_clg10", 0)
    om = oracle.OracleModel.from_spec(spec)
    o = oracle.Oracle(om, 50, 16, 1, 3, lib=oracle_lib)
    x, z, lq = o.init()
    _, ys = workloads.simulate(spec, 1, 0)
    a = std_dpf.std_step(om, 3, 1, ys[0], x, z, lq, None, oracle_lib)
    b = std_dpf.std_step(om, 3, 1, ys[0], x, z, lq, None, oracle_lib, gauss=True)
    np.testing.assert_allclose(a[0], b[0], rtol=0, atol=1e-12)
    # moments on lg4: one ancestor group, many destination keys
    spec = workloads.make_model("lg4", 0)
    om = oracle.OracleModel.from_spec(spec)
    o = oracle.Oracle(om, 1, 8, 1, 5, lib=oracle_lib)
    x, z, lq = o.init()
    lq = np.log(np.array([[0.3, 0.05, 0.1, 0.2, 0.05, 0.1, 0.1, 0.1]]))
    n = 4000
    xs = std_dpf.std_step(om, 5, 1, np.zeros(2), x, z, lq, np.zeros(n, int), oracle_lib, dest=np.arange(n),
                          gauss=True)[0]
    d1 = om.d1
    comp_means = (np.concatenate([np.repeat(x, 8, 0), z[0]], 1) @ om.A.T)[:, :d1]
    q = np.exp(lq[0])
    mu = q @ comp_means
    cov = om.Q[:d1, :d1] + sum(q[j] * np.outer(comp_means[j] - mu, comp_means[j] - mu) for j in range(8))
    se = np.sqrt(np.diag(cov) / n)
    assert np.all(np.abs(xs.mean(0) - mu) < 4 * se), (xs.mean(0), mu)
    np.testing.assert_allclose(np.cov(xs.T), cov, rtol=0.1)
    # tracking
    _, ys = workloads.simulate(spec, 8, 3)
    km, kP, _ = kalman(spec.A, spec.Q, spec.H, spec.R, spec.m0, spec.P0, ys)
    sd = np.sqrt(np.stack([np.diag(P) for P in kP]))
    o = oracle.Oracle(om, 1000, 32, 1, 6, nthreads=8, lib=oracle_lib)
    x, z, lq = o.init()
    anc, means = None, []
    for t in range(1, 9):
        x, z, lq, lw, _, _ = std_dpf.std_step(om, 6, t, ys[t - 1], x, z, lq, anc, oracle_lib, gauss=True)
        W = np.exp(lw - lw.max()); W /= W.sum()
        means.append(np.concatenate([W @ x, W @ np.einsum("nm,nmc->nc", np.exp(lq), z)]))
        anc = oracle.sys_global(W, word(6, t, 0, oracle.P_OUTER), oracle_lib)
    assert np.max(np.abs(np.array(means) - km) / sd) < 0.3
