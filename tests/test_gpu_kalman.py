"""The CUDA filter against the exact Kalman posterior on the linear-Gaussian
workload: filtered means and log-evidence within Monte Carlo error, in FP64
and FP32, with the error shrinking as N and M grow."""
import numpy as np
import pytest

from paper_1203_2394_gb300 import workloads
from tests.kalman import kalman

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run(prec, N, M, L, reps, T):
    from paper_1203_2394_gb300 import dpf
    spec = workloads.make_model("lg4", 0)
    _, ys = workloads.simulate(spec, T, 0)
    km, kc, kll = kalman(spec.A, spec.Q, spec.H, spec.R, spec.m0, spec.P0, ys)
    dt = np.float64 if prec == dpf.DPF_F64 else np.float32
    means = np.zeros((reps, T, spec.d)); logz = np.zeros((reps, T))
    for r in range(reps):
        f = dpf.Filter(dpf.Model.from_spec(spec, prec), 2, 2, N, M, L, seed=1000 + r)
        for t in range(T):
            means[r, t], logz[r, t] = f.step(ys[t].astype(dt))
        f.close()
    err = means.mean(0) - km
    se = means.std(0, ddof=1) / np.sqrt(reps)
    sd = np.sqrt(np.einsum("tii->ti", kc))
    lerr = logz.mean(0) - np.cumsum(kll)
    lse = logz.std(0, ddof=1) / np.sqrt(reps)
    return err, se, sd, lerr, lse


@pytest.mark.parametrize("prec", [0, 1], ids=["f32", "f64"])
def test_gpu_filter_tracks_kalman(prec):
    err, se, sd, lerr, lse = _run(prec, 2048, 64, 8, 24, 30)
    assert np.all(np.abs(err) < 4.5 * se + 0.03 * sd), np.max(np.abs(err) / (se + 1e-12))
    assert np.all(np.abs(lerr) < 4.5 * lse + 0.03 * np.sqrt(np.arange(1, 31)))


def test_error_shrinks_with_particles():
    small = _run(1, 128, 16, 4, 24, 20)
    large = _run(1, 4096, 128, 8, 24, 20)
    rms = lambda r: np.sqrt(np.mean(r[0] ** 2 + r[1] ** 2 * 24))  # bias^2 + variance of one run
    assert rms(large) < rms(small)
