"""Pins of the oracle of the paper's benchmark models (Table 1): oracle/nl.py.

* The transition means and the observation function at points evaluated by hand from the
  table's equations.
* The x-first draw's noise factor reproduces the table's noise covariance, with model 2's
  z2' carrying z1' and its noise: T T^T = J Sv J^T.
* The observation density against scipy's normal density.
* A look-ahead draw's weight, for an inner set of equal particles, is the Monte Carlo mean
  of p(y_t | xbb, z) over z from the transition's conditional given xbb: against that
  integral by quadrature of the joint Gaussian, within four standard errors.
* The grid filter itself (tests/grid_filter.py) against the Kalman filter on a linear
  two-dimensional model with correlated noise: means, standard deviations and evidence.
* Model 1's filtered means and log-evidence increments, from the bootstrap particle filter
  and the LA-DPF, against the exact filter on a grid (tests/grid_filter.py), and planted
  mistakes (the p(x | x, z) factor of the pair weights dropped, the x-z coupling G dropped,
  the time index off by one, the inner noise dropped, the observation variance wrong) make
  the LA-DPF miss it.
* Model 2: the LA-DPF agrees with a bootstrap particle filter of many particles, in the
  filtered means and the log-evidence increments.
* Model 1 decomposed the other way (the table's z outer, its x inner; Section 4.3's second
  action): the transition at a hand-evaluated point in the swapped coordinates, and the
  LA-DPF and the particle filter against the grid filter, mapped back to the table's order.
* The DPF without look-ahead: model 1 against the grid filter, with the Monte Carlo
  mixture prior and with its Gaussian approximation, and planted mistakes miss it; on model
  2, whose x transition is free of z, the Gaussian approximation is the mixture itself, so
  both forms give the same particles; on model 1 the two forms' draws of x_t for one group
  over 4000 seeds have the same mean and variance (the moments the Gaussian form matches).
"""
import numpy as np
import pytest

from oracle import nl, oracle
from paper_1203_2394_gb300 import workloads
from tests.grid_filter import model1_posterior_means, posterior_means
from tests.kalman import kalman

scipy_stats = pytest.importorskip("scipy.stats")
scipy_integrate = pytest.importorskip("scipy.integrate")


@pytest.fixture(scope="module")
def lib():
    return oracle.load()


def test_model_special_points():
    m1, m2 = nl.PaperModel(1), nl.PaperModel(2)
    # model 1 at x = 2, z = 1, s = 0: 2 + 1/2; 2 + 0.5 + 12.5 + 8
    fx, fz = m1.transition(np.array([2.0]), np.array([1.0]), 0)
    np.testing.assert_allclose([fx[0], fz[0]], [2.5, 23.0], rtol=1e-15)
    # at x = 0, z = 0, s = pi / 1.2: cos = -1
    fx, fz = m1.transition(np.array([0.0]), np.array([0.0]), np.pi / 1.2)
    np.testing.assert_allclose([fx[0], fz[0]], [0.0, -8.0], atol=1e-14)
    np.testing.assert_allclose(m1.h(np.array([0.0]), np.array([2.0])), 0.2, rtol=1e-15)
    np.testing.assert_allclose(m1.h(np.array([1.0]), np.array([0.0])), np.pi / 4, rtol=1e-15)
    # model 2 at x = (2, 2), z = (1, 1), s = 0: (1, 0.8 + 1), z1' = 1.5, z2' = 1.5 + 0.5 + 12.5 + 8
    fx, fz = m2.transition(np.array([2.0, 2.0]), np.array([1.0, 1.0]), 0)
    np.testing.assert_allclose(np.r_[fx, fz], [1.0, 1.8, 1.5, 22.5], rtol=1e-15)
    # s = pi / 2: 8 sin = 8
    fx, _ = m2.transition(np.array([0.0, 0.0]), np.array([0.0, 0.0]), np.pi / 2)
    np.testing.assert_allclose(fx, [8.0, 0.0], atol=1e-14)
    np.testing.assert_allclose(m2.h(np.array([1.0, 1.0]), np.array([0.0, 0.0])), 1.0, rtol=1e-15)
    np.testing.assert_allclose(m2.h(np.array([0.0, 0.0]), np.array([1.0, 2.0])), np.pi / 4 + 0.2, rtol=1e-15)


@pytest.mark.parametrize("kind,Q", [
    (1, [[1, 0.1], [0.1, 1]]),
    # v_z = (v3, v4) ~ N(0, [[1, 0.1], [0.1, 10]]) enters as (v3, v3 + v4)
    (2, [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 1.1], [0, 0, 1.1, 11.2]]),
])
def test_noise_factor_is_the_table_covariance(kind, Q):
    m = nl.PaperModel(kind)
    d1 = m.d1
    T = np.zeros((m.d, m.d))
    T[:d1, :d1] = m.Lqx
    T[d1:, :d1] = m.G @ m.Lqx
    T[d1:, d1:] = m.LS
    np.testing.assert_allclose(T @ T.T, np.array(Q, float), atol=1e-14)
    # the same factor through the draw functions, column by column
    e = np.eye(m.d)
    xs = m.draw_x(np.zeros(d1), e[:, :d1])
    zs = m.draw_z(np.zeros(d1), np.zeros(d1), xs, e[:, d1:])
    np.testing.assert_allclose(np.c_[xs, zs].T, T, atol=1e-15)


def test_log_py_is_the_normal_density():
    m = nl.PaperModel(2)
    rng = np.random.default_rng(0)
    x, z = rng.normal(size=(50, 2)), rng.normal(size=(50, 2))
    y = 0.7
    ref = scipy_stats.norm.logpdf(y, loc=m.h(x, z), scale=1.0)
    np.testing.assert_allclose(m.log_py(y, x, z), ref, rtol=1e-13)


def test_lookahead_weight_is_the_conditional_integral(lib):
    m = nl.PaperModel(1)
    M, L, seed, t, y = 1024, 4, 11, 3, 1.3
    x = np.array([[0.4]])
    z = np.full((1, M, 1), 1.7)
    lq = np.full((1, M), -np.log(M))
    lw, lwhat, xbb, _, _ = nl.lookahead(m, seed, t, y, x, z, lq, L, [0], lib)
    fx, fz = m.transition(x[0], z[0, 0], t - 1)
    Qi = np.linalg.inv(m.Q)
    for k in range(L):
        xb = xbb[0, k, 0]
        # p(z' | xb) from the joint Gaussian N((fx, fz), Q) divided by its x marginal
        def joint(zp):
            r = np.array([xb - fx[0], zp - fz[0]])
            return np.exp(-0.5 * r @ Qi @ r) / (2 * np.pi * np.sqrt(np.linalg.det(m.Q)))
        px = scipy_stats.norm.pdf(xb, fx[0], np.sqrt(m.Q[0, 0]))
        f = lambda zp: scipy_stats.norm.pdf(y, np.arctan(xb) + zp * zp / 20, 1.0) * joint(zp) / px
        c = fz[0] + m.Q[1, 0] / m.Q[0, 0] * (xb - fx[0])
        ref, _ = scipy_integrate.quad(f, c - 12, c + 12, epsabs=1e-13, limit=200)
        # the Monte Carlo standard error of the mean of p(y | xb, z_k) over the draws
        ek = oracle.normals_many(seed, 0, t, np.zeros(M, int), oracle.P_LA_Z, np.arange(M), 1, lib)[:, 0]
        zk = m.draw_z(fz, fx, np.array([xb]), ek[:, None])[:, 0]
        pk = scipy_stats.norm.pdf(y, np.arctan(xb) + zk * zk / 20, 1.0)
        se = pk.std() / np.sqrt(M) / pk.mean()
        assert abs(lwhat[0, k] - np.log(ref)) < 4 * se + 1e-12, (k, lwhat[0, k], np.log(ref), se)
    np.testing.assert_allclose(lw[0], np.log(np.mean(np.exp(lwhat[0]))), rtol=1e-13)


def test_grid_filter_is_the_kalman_filter_on_a_linear_model():
    A = np.array([[0.9, 0.3], [-0.2, 0.8]])
    Q = np.array([[1.0, 0.3], [0.3, 0.5]])
    H = np.array([[1.0, -0.7]])
    rng = np.random.default_rng(3)
    s = rng.normal(size=2)
    ys = []
    for _ in range(6):
        s = A @ s + np.linalg.cholesky(Q) @ rng.normal(size=2)
        ys.append(H @ s + np.sqrt(0.5) * rng.normal(size=1))
    ys = np.array(ys)
    km, kP, kll = kalman(A, Q, H, 0.5 * np.eye(1), np.zeros(2), np.eye(2), ys)
    gm, gs, glz, edge = posterior_means(
        ys, np.arange(-12, 12 + 1e-9, 0.2), np.arange(-12, 12 + 1e-9, 0.2),
        lambda x, z, t: (A[0, 0] * x + A[0, 1] * z, A[1, 0] * x + A[1, 1] * z),
        lambda x, z: H[0, 0] * x + H[0, 1] * z, Q, r_var=0.5)
    assert edge < 1e-12
    np.testing.assert_allclose(gm, km, atol=1e-6)
    np.testing.assert_allclose(gs, np.sqrt(np.stack([np.diag(P) for P in kP])), atol=1e-6)
    np.testing.assert_allclose(glz, kll, atol=1e-6)


GRID = dict(xg=np.arange(-15, 15 + 1e-9, 0.2), zg=np.arange(-36, 36 + 1e-9, 0.1), cut=1e-10)


@pytest.fixture(scope="module")
def grid1():
    _, ys = workloads.simulate_paper(1, 6, 0)
    gm, gs, glz, edge = model1_posterior_means(ys, **GRID)
    assert edge < 1e-10
    return ys, gm, gs, glz


def test_pf_matches_the_grid_filter(grid1, lib):
    ys, gm, gs, glz = grid1
    mp, lp, _ = nl.run_pf(nl.PaperModel(1), 3, ys, 50000, lib)
    assert np.abs((mp - gm) / gs).max() < 0.1
    assert np.abs(lp - glz).max() < 0.1


def _la_dpf_errors(model, ys, gm, gs, glz, lib):
    ml, lz = nl.run_la_dpf(model, 3, ys, 600, 32, 8, lib)
    return np.abs((ml - gm) / gs).max(), np.abs(lz - glz).max()


def test_la_dpf_matches_the_grid_filter(grid1, lib):
    ys, gm, gs, glz = grid1
    em, ez = _la_dpf_errors(nl.PaperModel(1), ys, gm, gs, glz, lib)
    assert em < 0.2 and ez < 0.2, (em, ez)


def _plant(name):
    m = nl.PaperModel(1)
    if name == "no_px_factor":
        f = m.log_px
        m.log_px = lambda xn, fx: 0.0 * f(xn, fx)
    elif name == "no_coupling":
        m.G = 0.0 * m.G
    elif name == "time_off_by_one":
        tr = m.transition
        m.transition = lambda x, z, s, v=None: tr(x, z, s + 1, v)
    elif name == "no_inner_noise":
        m.LS = 0.0 * m.LS
    elif name == "obs_variance":
        h = m.h
        m.log_py = lambda y, x, z: -0.5 * np.log(2 * np.pi) - 2.0 * (float(y) - h(x, z)) ** 2
    return m


@pytest.mark.parametrize("name", ["no_px_factor", "no_coupling", "time_off_by_one", "no_inner_noise",
                                  "obs_variance"])
def test_planted_mistake_misses_the_grid_filter(grid1, lib, name):
    ys, gm, gs, glz = grid1
    em, ez = _la_dpf_errors(_plant(name), ys, gm, gs, glz, lib)
    assert em >= 0.2 or ez >= 0.2, (name, em, ez)


def test_model2_la_dpf_agrees_with_pf(lib):
    m = nl.PaperModel(2)
    _, ys = workloads.simulate_paper(2, 8, 0)
    mp, lp, sp = nl.run_pf(m, 4, ys, 200000, lib)
    # M = 128: with 32 inner particles the ratio estimate of a draw's weight is still
    # visibly biased on this model (z2 has variance 11.2 under a likelihood in z2^2 / 20)
    ml, ll = nl.run_la_dpf(m, 4, ys, 600, 128, 8, lib)
    assert np.abs((ml - mp) / sp).max() < 0.15
    assert np.abs(ll - lp).max() < 0.15


def _std_errors(model, ys, gm, gs, glz, lib, N=600, gauss=False):
    ms, lz = nl.run_std(model, 3, ys, N, 32, lib, gauss=gauss)
    return np.abs((ms - gm) / gs).max(), np.abs(lz - glz).max()


@pytest.mark.parametrize("gauss", [False, True])
def test_dpf_matches_the_grid_filter(grid1, lib, gauss):
    ys, gm, gs, glz = grid1
    # the Gaussian form approximates the mixture prior of x_t: more outer particles
    em, ez = _std_errors(nl.PaperModel(1), ys, gm, gs, glz, lib, N=2000 if gauss else 600, gauss=gauss)
    assert em < 0.2 and ez < 0.2, (em, ez)


@pytest.mark.parametrize("name", ["no_px_factor", "no_coupling", "time_off_by_one"])
def test_dpf_planted_mistake_misses_the_grid_filter(grid1, lib, name):
    ys, gm, gs, glz = grid1
    em, ez = _std_errors(_plant(name), ys, gm, gs, glz, lib)
    assert em >= 0.2 or ez >= 0.2, (name, em, ez)


def test_dpf_gaussian_form_is_exact_when_x_is_free_of_z(lib):
    m = nl.PaperModel(2)
    N, M, seed = 40, 16, 5
    x, z, lq = nl.init(m, N, M, seed, lib)
    lq = lq + np.random.default_rng(0).normal(size=lq.shape)  # unequal inner weights
    lq -= np.log(np.exp(lq).sum(1, keepdims=True))
    anc = np.random.default_rng(1).integers(0, N, N)
    a = nl.std_step(m, seed, 3, 0.4, x, z, lq, anc, lib, gauss=False)
    b = nl.std_step(m, seed, 3, 0.4, x, z, lq, anc, lib, gauss=True)
    for u, v in zip(a, b):
        np.testing.assert_allclose(u, v, rtol=0, atol=1e-12)


def test_swapped_model1_coordinates():
    m = nl.PaperModel(1, swap=True)
    # filter x = table z = 1, filter z = table x = 2, s = 0: table x' = 2.5, table z' = 23
    fx, fz = m.transition(np.array([1.0]), np.array([2.0]), 0)
    np.testing.assert_allclose([fx[0], fz[0]], [23.0, 2.5], rtol=1e-15)
    np.testing.assert_allclose(m.h(np.array([2.0]), np.array([0.0])), 0.2, rtol=1e-15)
    np.testing.assert_allclose(m.Q, [[1, 0.1], [0.1, 1]], atol=1e-15)


def test_swapped_decomposition_matches_the_grid_filter(grid1, lib):
    ys, gm, gs, glz = grid1
    m = nl.PaperModel(1, swap=True)
    mp, lp, _ = nl.run_pf(m, 3, ys, 50000, lib)
    # the swapped LA-DPF needs more inner particles (the table's x given its z) to reach the
    # same error: with M = 32 it is 0.5 posterior standard deviations off, with 256 within 0.2
    ml, ll = nl.run_la_dpf(m, 3, ys, 600, 256, 8, lib)
    for mean, lz, tm, tz in ((mp, lp, 0.1, 0.1), (ml, ll, 0.2, 0.3)):
        table = np.empty_like(mean)
        table[:, m.perm] = mean
        assert np.abs((table - gm) / gs).max() < tm
        assert np.abs(lz - glz).max() < tz


def test_dpf_gaussian_form_matches_the_mixture_moments(lib):
    m = nl.PaperModel(1)
    M, seeds = 8, 4000
    x = np.array([[0.3]])
    z = np.array([[[-2.0], [-0.5], [0.2], [0.9], [1.5], [3.0], [-4.0], [0.0]]])
    lq = np.log(np.array([[0.05, 0.2, 0.1, 0.15, 0.2, 0.1, 0.1, 0.1]]))
    draws = {False: [], True: []}
    for seed in range(seeds):
        for gauss in (False, True):
            xt = nl.std_step(m, seed, 2, 0.1, x, z, lq, np.array([0]), lib, gauss=gauss)[0]
            draws[gauss].append(xt[0, 0])
    a, b = np.array(draws[False]), np.array(draws[True])
    se = np.sqrt(a.var() / seeds + b.var() / seeds)
    assert abs(a.mean() - b.mean()) < 4 * se, (a.mean(), b.mean(), se)
    assert abs(a.var() / b.var() - 1) < 4 * np.sqrt(2 / seeds) * 1.5, (a.var(), b.var())
