"""Pins of the learned-proposal oracle (``oracle/learned.py``), none of which reuses its
own formulas:

* gradients of the weighted NLL against central finite differences (FP64), with some
  log-sigmas outside the clamp (zero gradient there);
* one component: log q equals scipy's multivariate normal log-density;
* the mixture density integrates to one on a grid; identical components give the
  single-component density whatever the logits;
* Adam's first step equals -lr g / (|g| + eps) (bias correction cancels), and Adam
  minimises a convex quadratic;
* bfloat16 rounding agrees with torch's float32 -> bfloat16 conversion;
* a network that outputs exactly the prior (a ReLU pair per input, identity hidden
  layers, four equal components with sigma^2 = Q_z) makes the learned inner update
  reproduce the plain one of the C oracle (which the Kalman pins hold), z and lq.
"""
import numpy as np
import pytest

from oracle import learned, oracle
from paper_1203_2394_gb300 import workloads


def _small(seed=0, din=8, hidden=12, d2=2, C=3, n=40):
    rng = np.random.default_rng(seed)
    W = workloads.init_mlp_weights(din, hidden, C * (1 + 2 * d2), seed=seed)
    for k in W:
        W[k] = W[k] + 0.05 * rng.standard_normal(W[k].shape)
    F = rng.standard_normal((n, din))
    Z = rng.standard_normal((n, d2))
    w = rng.uniform(0.1, 1.0, n)
    return W, F, Z, w


def test_gradients_match_finite_differences():
    W, F, Z, w = _small()
    d2, C = 2, 3
    # push a few raw log-sigmas outside the clamp
    W["b4"][C + C * d2 + 0] = 9.0
    W["b4"][C + C * d2 + 3] = -11.0
    loss, G = learned.nll_and_grad(W, F, Z, w, d2, C)
    h = 1e-6
    rng = np.random.default_rng(1)
    for k in W:
        flat = W[k].reshape(-1)
        picks = rng.choice(flat.size, min(flat.size, 25), replace=False)
        for p in picks:
            old = flat[p]
            flat[p] = old + h
            lp, _ = learned.nll_and_grad(W, F, Z, w, d2, C)
            flat[p] = old - h
            lm, _ = learned.nll_and_grad(W, F, Z, w, d2, C)
            flat[p] = old
            fd = (lp - lm) / (2 * h)
            g = G[k].reshape(-1)[p]
            assert abs(fd - g) <= 1e-6 * max(1.0, abs(fd)), (k, p, fd, g)
    assert G["b4"][C + C * d2 + 0] == 0.0 and G["b4"][C + C * d2 + 3] == 0.0


def test_one_component_is_the_gaussian_density():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(2)
    n, d2 = 30, 3
    z = rng.standard_normal((n, d2))
    mu = rng.standard_normal((n, 1, d2))
    ls = rng.uniform(-1, 1, (n, 1, d2))
    lq = learned.logq(z, rng.standard_normal((n, 1)), mu, ls)
    for b in range(n):
        ref = stats.multivariate_normal.logpdf(z[b], mu[b, 0], np.diag(np.exp(2 * ls[b, 0])))
        assert lq[b] == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_mixture_integrates_to_one_and_equal_components_collapse():
    rng = np.random.default_rng(3)
    C = 4
    logits = rng.standard_normal((1, C))
    mu = rng.uniform(-1, 1, (1, C, 2))
    ls = rng.uniform(-0.7, 0.2, (1, C, 2))
    g = np.linspace(-9, 9, 721)
    X, Y = np.meshgrid(g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel()], 1)
    lq = learned.logq(pts, np.repeat(logits, len(pts), 0), np.repeat(mu, len(pts), 0),
                      np.repeat(ls, len(pts), 0))
    mass = np.exp(lq).sum() * (g[1] - g[0]) ** 2
    assert mass == pytest.approx(1.0, abs=1e-6)
    same_mu = np.repeat(mu[:, :1], C, 1)
    same_ls = np.repeat(ls[:, :1], C, 1)
    z = rng.standard_normal((1, 2))
    a = learned.logq(z, logits, same_mu, same_ls)
    b = learned.logq(z, np.zeros((1, 1)), mu[:, :1], ls[:, :1])
    assert a[0] == pytest.approx(b[0], rel=1e-13, abs=1e-13)


def test_adam_first_step_and_convergence():
    rng = np.random.default_rng(4)
    W = {"a": rng.standard_normal(7)}
    G = {"a": rng.standard_normal(7)}
    st = learned.adam_init(W)
    lr, eps = 3e-3, 1e-8
    W1 = learned.adam_step(W, G, st, lr=lr, eps=eps)
    np.testing.assert_allclose(W1["a"] - W["a"], -lr * G["a"] / (np.abs(G["a"]) + eps), rtol=1e-9)
    # minimise 0.5 (w - c)^T D (w - c)
    c = rng.standard_normal(5)
    D = rng.uniform(0.5, 3.0, 5)
    W = {"a": np.zeros(5)}
    st = learned.adam_init(W)
    for _ in range(3000):
        W = learned.adam_step(W, {"a": D * (W["a"] - c)}, st, lr=1e-2)
    np.testing.assert_allclose(W["a"], c, atol=1e-3)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.standard_normal(4000) * 10 ** rng.uniform(-6, 6, 4000),
                        [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.0 - 2.0 ** -8, 0.0, -0.0]])
    ref = torch.tensor(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(learned.bf16(v), ref)


def _prior_net(model, hidden=16, C=4):
    """An MLP whose mixture is exactly the prior N(A_zx x_a + A_zz z_b, Q_z)."""
    d1, d2, dy = model.d1, model.d2, model.dy
    din = 2 * d1 + d2 + dy
    A = model.A
    P = np.zeros((d2, din))
    P[:, :d1] = A[d1:, :d1]             # A_zx x_{t-1}
    P[:, 2 * d1:2 * d1 + d2] = A[d1:, d1:]  # A_zz z_b
    W = {}
    W1 = np.zeros((hidden, din))
    W1[:din] = np.eye(din)
    W1[din:2 * din] = -np.eye(din)
    W["W1"], W["b1"] = W1, np.zeros(hidden)
    for l in (2, 3):
        W[f"W{l}"], W[f"b{l}"] = np.eye(hidden), np.zeros(hidden)
    dout = C * (1 + 2 * d2)
    W4 = np.zeros((dout, hidden))
    b4 = np.zeros(dout)
    sig = np.sqrt(np.diag(model.Q[d1:, d1:]))
    for c in range(C):
        rows = slice(C + c * d2, C + (c + 1) * d2)
        W4[rows, :din] = P
        W4[rows, din:2 * din] = -P
        b4[C + C * d2 + c * d2:C + C * d2 + (c + 1) * d2] = np.log(sig)
    W["W4"], W["b4"] = W4, b4
    return W


def test_prior_network_reproduces_the_plain_inner_update():
    spec = workloads.make_model("lg4", 0)
    om = oracle.OracleModel.from_spec(spec)
    N, M, L, seed = 12, 16, 4, 3
    o = oracle.Oracle(om, N, M, L, seed)
    _, ys = workloads.simulate(spec, 3, 0)
    x, z, lq = o.init()
    r1 = o.step(1, ys[0], x, z, lq)
    x1, z1, lq1 = r1["x"], r1["z"], r1["lq"]
    r2 = o.step(2, ys[1], x1, z1, lq1)
    anc, xn = r2["anc"], r2["x"]
    fin = o.finalize(2, ys[1], np.arange(N), anc, x1, z1, lq1, xn)
    W = _prior_net(om)
    lib = oracle.load()
    got = learned.learned_finalize(
        om, W, 4, seed, 2, ys[1], anc, x1, z1, xn, fin["bidx"],
        normals=lambda t, i, p, j, n: oracle.normals(seed, 0, t, i, p, j, n, lib),
        sys_local=lambda w, k, u: oracle.sys_local(w, k, u, lib),
        word=lambda t, i, p, j: int(oracle.philox((t, i, (p << 24) | j, 0), (seed, 0), lib)[0]))
    np.testing.assert_allclose(got["z"], fin["z"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(got["lq"], fin["lq"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(fin["z"], r2["z"], rtol=0, atol=0)


def test_affine_gradients_match_finite_differences():
    rng = np.random.default_rng(20)
    din, d2, n = 10, 2, 30
    W = workloads.init_mlp_weights(din, 12, 2 * d2, seed=21)
    for k in W:
        W[k] = W[k] + 0.05 * rng.standard_normal(W[k].shape)
    W["b4"][0] = 8.0  # one log-scale outside the clamp
    G = rng.standard_normal((n, din))
    Z = rng.standard_normal((n, d2)); MU = rng.standard_normal((n, d2)); MG = rng.standard_normal((n, d2))
    Qz = np.array([[0.2, 0.05], [0.05, 0.1]])
    w = rng.uniform(0.1, 1, n)
    loss, Gr = learned.affine_nll_and_grad(W, G, Z, MU, MG, Qz, w)
    h = 1e-6
    for k in W:
        flat = W[k].reshape(-1)
        for p in rng.choice(flat.size, min(flat.size, 20), replace=False):
            old = flat[p]
            flat[p] = old + h
            lp, _ = learned.affine_nll_and_grad(W, G, Z, MU, MG, Qz, w)
            flat[p] = old - h
            lm, _ = learned.affine_nll_and_grad(W, G, Z, MU, MG, Qz, w)
            flat[p] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - Gr[k].reshape(-1)[p]) <= 1e-6 * max(1.0, abs(fd)), (k, p)
    assert Gr["b4"][0] == 0.0


def test_affine_density_is_the_change_of_variables():
    # q(z) of the affine map equals N(z; m + c + s (mu - m), S Qz S), by scipy
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(22)
    d2 = 2
    Qz = np.array([[0.2, 0.05], [0.05, 0.1]])
    mu, m = rng.standard_normal(d2), rng.standard_normal(d2)
    ls, c = rng.uniform(-0.5, 0.5, d2), rng.standard_normal(d2)
    s = np.exp(ls)
    W = {"W1": np.zeros((4, 1)), "b1": np.zeros(4), "W2": np.zeros((2 * d2, 4)),
         "b2": np.concatenate([ls, c])}
    for _ in range(5):
        z = rng.standard_normal(d2)
        loss, _ = learned.affine_nll_and_grad(W, np.zeros((1, 1)), z[None], mu[None], m[None], Qz, [1.0])
        S = np.diag(s)
        ref = stats.multivariate_normal.logpdf(z, m + c + s * (mu - m), S @ Qz @ S)
        assert -loss == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_identity_affine_map_reproduces_the_plain_inner_update():
    spec = workloads.make_model("lg4", 0)
    om = oracle.OracleModel.from_spec(spec)
    N, M, L, seed = 10, 16, 4, 3
    o = oracle.Oracle(om, N, M, L, seed)
    _, ys = workloads.simulate(spec, 3, 0)
    x, z, lq = o.init()
    r1 = o.step(1, ys[0], x, z, lq)
    r2 = o.step(2, ys[1], r1["x"], r1["z"], r1["lq"])
    fin = o.finalize(2, ys[1], np.arange(N), r2["anc"], r1["x"], r1["z"], r1["lq"], r2["x"])
    din = 2 * om.d1 + om.dy + 2 * om.d2
    W = workloads.init_mlp_weights(din, 16, 2 * om.d2, seed=1)
    W["W4"][:] = 0.0
    W["b4"][:] = 0.0  # s = 1, c = 0
    lib = oracle.load()
    got = learned.amortised_finalize(om, W, seed, 2, ys[1], r2["anc"], r1["x"], r1["z"], r2["x"], fin["bidx"],
                                     normals=lambda t, i, p, j, n: oracle.normals(seed, 0, t, i, p, j, n, lib))
    np.testing.assert_allclose(got["z"], fin["z"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(got["lq"], fin["lq"], rtol=1e-10, atol=1e-10)


def test_inner_ess_and_the_fallback_rule():
    """Inner ESS: M for equal weights, k for k equal weights and the rest zero, shift
    invariant; weights (1, 1, 1, 3) give 6^2 / 12 = 3, so the strict rule ESS < frac M
    falls back at frac 0.8 (3 < 3.2) and not at 0.75 (3 = 3)."""
    M = 64
    assert learned.inner_ess(np.zeros((1, M)))[0] == pytest.approx(M, rel=1e-15)
    for k in (1, 5, 32):
        lq = np.full((1, M), -np.inf)
        lq[0, :k] = -3.0
        assert learned.inner_ess(lq)[0] == pytest.approx(k, rel=1e-15)
    rng = np.random.default_rng(0)
    lq = rng.standard_normal((7, M))
    np.testing.assert_allclose(learned.inner_ess(lq + 17.5), learned.inner_ess(lq), rtol=1e-13)
    lq4 = np.log(np.array([[1.0, 1.0, 1.0, 3.0]]))
    assert learned.inner_ess(lq4)[0] == pytest.approx(3.0, rel=1e-15)
    assert learned.fallback_groups(lq4, 0.8)[0]
    assert not learned.fallback_groups(lq4, 0.75)[0]


def test_particle_centred_map_weights_by_its_density():
    """With the centre at the particle's own prior mean the map's draw is
    z = mu_j + c + s (zhat - mu_j), zhat ~ N(mu_j, Q_z), so its proposal density is
    N(z; mu_j + c, S Q_z S): the oracle's log-weights, evaluated by change of
    variables, must equal log N(z; mu_j, Q_z) - log N(z; mu_j + c, S Q_z S)
    + log N(y; H_x x + H_z z, R) normalised over the group (scipy's densities); the
    identity map (s = 1, c = 0) reproduces the plain inner update."""
    stats = pytest.importorskip("scipy.stats")
    spec = workloads.make_model("lg4", 0)
    om = oracle.OracleModel.from_spec(spec)
    N, M, L, seed = 6, 16, 4, 5
    o = oracle.Oracle(om, N, M, L, seed)
    _, ys = workloads.simulate(spec, 3, 0)
    x, z, lq = o.init()
    r1 = o.step(1, ys[0], x, z, lq)
    r2 = o.step(2, ys[1], r1["x"], r1["z"], r1["lq"])
    fin = o.finalize(2, ys[1], np.arange(N), r2["anc"], r1["x"], r1["z"], r1["lq"], r2["x"])
    lib = oracle.load()
    d1, d2 = om.d1, om.d2
    din = 2 * d1 + om.dy + 2 * d2
    W = workloads.init_mlp_weights(din, 16, 2 * d2, seed=1)
    W["W4"][:] = 0.0
    W["b4"][:] = 0.0
    nrm = lambda t, i, p, j, n: oracle.normals(seed, 0, t, i, p, j, n, lib)  # noqa: E731
    ident = learned.amortised_finalize(om, W, seed, 2, ys[1], r2["anc"], r1["x"], r1["z"], r2["x"], fin["bidx"],
                                       normals=nrm, centre="particle")
    np.testing.assert_allclose(ident["z"], fin["z"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(ident["lq"], fin["lq"], rtol=1e-10, atol=1e-10)
    rng = np.random.default_rng(8)
    head = np.concatenate([rng.uniform(-0.4, 0.4, (N, d2)), 0.3 * rng.standard_normal((N, d2))], axis=1)
    got = learned.amortised_finalize(om, W, seed, 2, ys[1], r2["anc"], r1["x"], r1["z"], r2["x"], fin["bidx"],
                                     normals=nrm, head_out=head, centre="particle")
    Qz, Hx, Hz = om.Q[d1:, d1:], om.H[:, :d1], om.H[:, d1:]
    for i in range(N):
        a = r2["anc"][i]
        mu = r1["x"][a] @ om.A[d1:, :d1].T + r1["z"][a][fin["bidx"][i]] @ om.A[d1:, d1:].T
        s, c = np.exp(head[i, :d2]), head[i, d2:]
        S = np.diag(s)
        lr = np.array([stats.multivariate_normal.logpdf(got["z"][i, j], mu[j], Qz)
                       - stats.multivariate_normal.logpdf(got["z"][i, j], mu[j] + c, S @ Qz @ S)
                       + stats.multivariate_normal.logpdf(ys[1], Hx @ r2["x"][i] + Hz @ got["z"][i, j], om.R)
                       for j in range(M)])
        lr -= lr.max()
        np.testing.assert_allclose(got["lq"][i], lr - np.log(np.exp(lr).sum()), rtol=1e-9, atol=1e-9)


def test_particle_centred_map_at_d2_56():
    """The same density check at the high-dimensional size (growth_clg64: d1 = 8,
    d2 = 56, dy = 8, observations quadratic in x), on three groups of 16."""
    stats = pytest.importorskip("scipy.stats")
    spec = workloads.make_model("growth_clg64", 0)
    om = oracle.OracleModel.from_spec(spec)
    N, M, L, seed = 3, 16, 4, 7
    o = oracle.Oracle(om, N, M, L, seed)
    _, ys = workloads.simulate(spec, 3, 0)
    x, z, lq = o.init()
    r1 = o.step(1, ys[0], x, z, lq)
    r2 = o.step(2, ys[1], r1["x"], r1["z"], r1["lq"])
    fin = o.finalize(2, ys[1], np.arange(N), r2["anc"], r1["x"], r1["z"], r1["lq"], r2["x"])
    lib = oracle.load()
    d1, d2 = om.d1, om.d2
    W = workloads.init_mlp_weights(2 * d1 + om.dy + 2 * d2, 16, 2 * d2, seed=1)
    rng = np.random.default_rng(9)
    head = np.concatenate([rng.uniform(-0.2, 0.2, (N, d2)), 0.1 * rng.standard_normal((N, d2))], axis=1)
    got = learned.amortised_finalize(om, W, seed, 2, ys[1], r2["anc"], r1["x"], r1["z"], r2["x"], fin["bidx"],
                                     normals=lambda t, i, p, j, n: oracle.normals(seed, 0, t, i, p, j, n, lib),
                                     head_out=head, centre="particle")
    Qz, Hz = om.Q[d1:, d1:], om.H[:, d1:]
    for i in range(N):
        a = r2["anc"][i]
        mu = r1["x"][a] @ om.A[d1:, :d1].T + r1["z"][a][fin["bidx"][i]] @ om.A[d1:, d1:].T
        s, c = np.exp(head[i, :d2]), head[i, d2:]
        S = np.diag(s)
        xn = r2["x"][i]
        hx = om.H[:, :d1] @ xn + (om.qc * xn[:om.dy] ** 2 if om.qc is not None else 0.0)
        lr = np.array([stats.multivariate_normal.logpdf(got["z"][i, j], mu[j], Qz)
                       - stats.multivariate_normal.logpdf(got["z"][i, j], mu[j] + c, S @ Qz @ S)
                       + stats.multivariate_normal.logpdf(ys[1], hx + Hz @ got["z"][i, j], om.R)
                       for j in range(M)])
        lr -= lr.max()
        np.testing.assert_allclose(got["lq"][i], lr - np.log(np.exp(lr).sum()), rtol=1e-8, atol=1e-8)
