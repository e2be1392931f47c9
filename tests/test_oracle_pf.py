"""The bootstrap particle filter's oracle (oracle/pf.py) against closed forms (CPU).

On the linear-Gaussian lg4 model the filtered means track the Kalman filter's within a
small fraction of the posterior standard deviation, and a transposed transition matrix
breaks that (the pin sees the mistake); the evidence estimator exp(log Z) is unbiased
(averaged over seeds it matches the Kalman likelihood within its standard error). On the
growth model, where no closed form exists, the filter agrees with the LA-DPF oracle, an
independently coded estimator of the same posterior mean.
"""
import numpy as np
import pytest

from oracle import oracle, pf
from paper_1203_2394_gb300 import workloads
from tests.gpu_util import word
from tests.kalman import kalman


def run_pf(model, seed, N, ys, lib):
    o = oracle.Oracle(model, N, 1, 1, seed, nthreads=8, lib=lib)
    x, z, _ = o.init()
    z = z[:, 0, :]
    noise = lambda t, i, p, n: oracle.normals(seed, 0, t, i, p, 0, n, lib)
    anc, means, sds, logz = None, [], [], 0.0
    for t in range(1, len(ys) + 1):
        x, z, lw = pf.pf_step(model, t, ys[t - 1], x, z, anc, noise)
        lz, mean, W = pf.summarise(lw, x, z)
        s = np.concatenate([x, z], axis=1)
        logz += lz
        means.append(mean)
        sds.append(np.sqrt(W @ (s - mean) ** 2))
        anc = oracle.sys_global(np.exp(lw - lw.max()), word(seed, t, 0, oracle.P_OUTER), lib)
    run_pf.sd = np.array(sds)
    return np.array(means), logz


def _lg4():
    spec = workloads.make_model("lg4", 0)
    return spec, oracle.OracleModel.from_spec(spec)


def test_pf_tracks_kalman_and_sees_a_transposed_transition(oracle_lib):
    spec, om = _lg4()
    _, ys = workloads.simulate(spec, 12, 3)
    km, kP, _ = kalman(spec.A, spec.Q, spec.H, spec.R, spec.m0, spec.P0, ys)
    sd = np.sqrt(np.stack([np.diag(P) for P in kP]))
    means, _ = run_pf(om, 11, 20000, ys, oracle_lib)
    err = np.max(np.abs(means - km) / sd)
    assert err < 0.15, err
    bad = oracle.OracleModel(om.d1, om.d2, om.dy, om.A.T, om.Q, om.H, om.R, om.m0, om.P0)
    means_bad, _ = run_pf(bad, 11, 20000, ys, oracle_lib)
    assert np.max(np.abs(means_bad - km) / sd) > 0.5


def test_pf_evidence_is_unbiased(oracle_lib):
    spec, om = _lg4()
    _, ys = workloads.simulate(spec, 4, 5)
    _, _, kll = kalman(spec.A, spec.Q, spec.H, spec.R, spec.m0, spec.P0, ys)
    ratios = np.array([np.exp(run_pf(om, 100 + r, 100, ys, oracle_lib)[1] - kll.sum()) for r in range(200)])
    se = ratios.std(ddof=1) / np.sqrt(len(ratios))
    assert abs(ratios.mean() - 1.0) <= 4 * se + 1e-3, (ratios.mean(), se)


def test_pf_agrees_with_the_ladpf_oracle_on_the_growth_model(oracle_lib):
    spec = workloads.make_model("growth_clg10", 0)
    om = oracle.OracleModel.from_spec(spec)
    _, ys = workloads.simulate(spec, 6, 0)
    means, _ = run_pf(om, 21, 20000, ys, oracle_lib)
    o = oracle.Oracle(om, 2000, 64, 16, 22, nthreads=8, lib=oracle_lib)
    sd = run_pf.sd
    ladpf = np.array([r["mean"] for r in o.run(ys)])
    # both are Monte Carlo estimates of the same posterior mean: their difference is a small
    # fraction of the posterior standard deviation (the x block is near-bimodal: y sees x^2)
    z = np.abs(means - ladpf) / sd
    assert np.max(z) < 0.25, np.round(z.max(axis=0), 3)
    # a growth term with the wrong sign is seen
    g = list(om.growth)
    g[1] = -g[1]
    bad = oracle.OracleModel(om.d1, om.d2, om.dy, om.A, om.Q, om.H, om.R, om.m0, om.P0, tuple(g), om.qc)
    means_bad, _ = run_pf(bad, 21, 20000, ys, oracle_lib)
    assert np.max(np.abs(means_bad - ladpf) / sd) > 1.0
