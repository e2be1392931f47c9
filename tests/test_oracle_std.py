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
