"""The bootstrap particle filter on the GPU (dpf_create_pf) against its oracle.

* Teacher-forced, step by step (lg4 in FP64, the growth model in FP32): from the GPU's
  particles and ancestors of step t-1 the oracle's step gives the same particles (1e-12 /
  1e-5) and log-weights, the ancestors of step t equal the oracle's systematic resampling
  of the GPU's quantised weights bit for bit, and the weighted mean matches.
* FP64 with many particles tracks the Kalman filter on lg4.
* The comparison workload's size (N = 65536 x 129 particles, FP32): sampled particles of
  one step against the oracle.
"""
import numpy as np
import pytest

from oracle import oracle, pf
from paper_1203_2394_gb300 import workloads
from tests.gpu_util import rel, word
from tests.kalman import kalman

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _filter(name, prec, N, seed):
    from paper_1203_2394_gb300 import dpf
    spec = workloads.make_model(name, 0)
    p = dpf.DPF_F64 if prec == "f64" else dpf.DPF_F32
    return spec, dpf.ParticleFilter(dpf.Model.from_spec(spec, p), spec.d1, spec.d2, N, seed)


def _state(f):
    return f.read("x").astype(np.float64), f.read("z")[:, :, 0].T.astype(np.float64)


@pytest.mark.parametrize("name,prec", [("lg4", "f64"), ("growth_clg10", "f32")])
def test_pf_teacher_forced(name, prec):
    N, seed = 3000, 7
    spec, f = _filter(name, prec, N, seed)
    om = oracle.OracleModel.from_spec(spec)
    lib = oracle.load()
    tol = 1e-12 if prec == "f64" else 2e-5
    dt = np.float64 if prec == "f64" else np.float32
    ox, oz, _ = oracle.Oracle(om, N, 1, 1, seed, lib=lib).init()
    x, z = _state(f)
    np.testing.assert_allclose(x, ox, rtol=0, atol=tol)
    np.testing.assert_allclose(z, oz[:, 0, :], rtol=0, atol=tol)
    _, ys = workloads.simulate(spec, 6, 1)
    noise = lambda t, i, p, n: oracle.normals(seed, 0, t, i, p, 0, n, lib)
    anc = None
    for t in range(1, 6):
        y = ys[t - 1].astype(dt)
        mean, _ = f.step(y)
        gx, gz = _state(f)
        lw = f.read("lw").astype(np.float64)
        ex, ez, elw = pf.pf_step(om, t, y.astype(np.float64), x, z, anc, noise)
        np.testing.assert_allclose(gx, ex, rtol=0, atol=tol * max(1.0, np.abs(ex).max()))
        np.testing.assert_allclose(gz, ez, rtol=0, atol=tol * max(1.0, np.abs(ez).max()))
        assert np.max(rel(lw, elw)) <= (1e-11 if prec == "f64" else 1e-5)
        _, emean, _ = pf.summarise(lw, gx, gz)
        assert np.max(rel(mean, emean[np.argsort(spec.perm())])) <= (1e-11 if prec == "f64" else 1e-5)
        anc = f.read("anc")
        wout = f.read("wout").astype(np.float64)
        np.testing.assert_array_equal(anc, oracle.sys_global(wout, word(seed, t, 0, oracle.P_OUTER), lib))
        x, z = gx, gz


def test_pf_f64_tracks_kalman():
    spec, f = _filter("lg4", "f64", 200000, 3)
    _, ys = workloads.simulate(spec, 20, 2)
    km, kP, kll = kalman(spec.A, spec.Q, spec.H, spec.R, spec.m0, spec.P0, ys)
    means = []
    for t in range(20):
        m, lz = f.step(ys[t])
        means.append(m)
    sd = np.sqrt(np.stack([np.diag(P) for P in kP]))
    err = np.max(np.abs(np.array(means) - km) / sd)
    assert err < 0.1, err
    assert abs(lz - kll.sum()) < 1.0, (lz, kll.sum())


def test_pf_comparison_size_sampled():
    N, seed = 65536 * 129, 5
    spec, f = _filter("growth_clg10", "f32", N, seed)
    om = oracle.OracleModel.from_spec(spec)
    lib = oracle.load()
    _, ys = workloads.simulate(spec, 2, 0)
    f.step(ys[0].astype(np.float32))
    x, z = _state(f)
    anc = f.read("anc")  # step 1's resampling: the ancestors step 2 starts from
    wout = f.read("wout").astype(np.float64)
    np.testing.assert_array_equal(anc, oracle.sys_global(wout, word(seed, 1, 0, oracle.P_OUTER), lib))
    f.step(ys[1].astype(np.float32))
    gx, gz = _state(f)
    lw = f.read("lw").astype(np.float64)
    idx = np.sort(np.random.default_rng(1).choice(N, 64, replace=False))
    noise = lambda t, i, p, n: oracle.normals(seed, 0, t, i, p, 0, n, lib)
    ex, ez, elw = pf.pf_step(om, 2, ys[1].astype(np.float32).astype(np.float64), x, z, anc[idx], noise,
                             dest=idx)
    np.testing.assert_allclose(gx[idx], ex, rtol=0, atol=2e-5 * max(1.0, np.abs(ex).max()))
    np.testing.assert_allclose(gz[idx], ez, rtol=0, atol=2e-5 * max(1.0, np.abs(ez).max()))
    assert np.max(rel(lw[idx], elw)) <= 1e-5
