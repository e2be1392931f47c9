"""Automatic state decomposition: Hedge and Exp3 (CPU; the library's host code).

Oracle pins (none retypes the oracle's update): Exp3's simulated reward is unbiased,
computed exactly over the K possible draws; Hedge's expected reward stays within the
Freund-Schapire regret bound ln K / eta + eta T / 8 of the best fixed action; Exp3's
average over seeds within Auer et al.'s bound (e - 1) gamma G_max + K ln K / gamma.
Library against oracle: the same probabilities (1e-12) and the same Exp3 action
sequence for the same rewards and seed; invalid inputs refused.
"""
import numpy as np
import pytest

from oracle import bandit, oracle


def _philox(c, k):
    return oracle.philox(c, k)


def test_exp3_simulated_reward_is_unbiased():
    rng = np.random.default_rng(0)
    K = 5
    for _ in range(20):
        e = bandit.Exp3(K, 0.1, 0.3, 7, _philox)
        e.hedge.G = rng.uniform(0, 5, K)
        ph = e.phat()
        r = rng.uniform(0, 1, K)
        # E[rhat_j] = sum_i phat_i rhat_j(i) with rhat_j(i) = r_j / phat_j if i == j else 0
        expect = np.array([sum(ph[i] * (r[j] / ph[j] if i == j else 0.0) for i in range(K)) for j in range(K)])
        np.testing.assert_allclose(expect, r, rtol=1e-12)


def test_hedge_regret_bound():
    rng = np.random.default_rng(1)
    K, T = 4, 2000
    eta = np.sqrt(8 * np.log(K) / T)
    R = rng.uniform(0, 1, (T, K)) * np.array([0.5, 0.6, 0.7, 0.55])
    h = bandit.Hedge(K, eta)
    gained = 0.0
    for t in range(T):
        gained += h.p() @ R[t]
        h.feed(R[t])
    regret = R.sum(0).max() - gained
    assert regret <= np.log(K) / eta + eta * T / 8
    assert h.p().argmax() == 2


def test_exp3_regret_bound_on_average():
    rng = np.random.default_rng(2)
    K, T = 3, 3000
    means = np.array([0.3, 0.5, 0.8])
    gmax = means.max() * T
    gamma = min(1.0, np.sqrt(K * np.log(K) / ((np.e - 1) * gmax)))
    regrets = []
    for seed in range(20):
        e = bandit.Exp3(K, gamma / K, gamma, seed, _philox)
        R = (rng.uniform(0, 1, (T, K)) < means).astype(float)
        got = 0.0
        for t in range(T):
            a = e.choose()
            got += R[t, a]
            e.feed(R[t, a])
        regrets.append(R.sum(0).max() - got)
    assert np.mean(regrets) <= (np.e - 1) * gamma * gmax + K * np.log(K) / gamma


def test_library_matches_oracle():
    from paper_1203_2394_gb300 import dpf
    rng = np.random.default_rng(3)
    K, T = 4, 300
    R = rng.uniform(0, 1, (T, K))
    h = dpf.Bandit(dpf.DPF_HEDGE, K, 0.5)
    ho = bandit.Hedge(K, 0.5)
    for t in range(T):
        np.testing.assert_allclose(h.probs(), ho.p(), rtol=1e-12, atol=1e-15)
        h.update(R[t])
        ho.feed(R[t])
    e = dpf.Bandit(dpf.DPF_EXP3, K, 0.05, 0.2, seed=12345678901)
    eo = bandit.Exp3(K, 0.05, 0.2, 12345678901, _philox)
    for t in range(T):
        np.testing.assert_allclose(e.probs(), eo.phat(), rtol=1e-12, atol=1e-15)
        a, ao = e.choose(), eo.choose()
        assert a == ao
        e.update(R[t, a])
        eo.feed(R[t, a])


def test_reward_values():
    from paper_1203_2394_gb300 import dpf
    y = np.array([0.3, -1.0, 2.0])
    # a perfect prediction earns 1; an error of squared norm alpha earns 1/2
    assert bandit.reward(y, y, 1e-3) == 1.0
    yh = y + np.array([0.0, np.sqrt(0.25), 0.0])
    assert abs(bandit.reward(y, yh, 0.25) - 0.5) < 1e-15
    # |eps|^2 = 3^2 + 4^2 = 25 for a 3-4-5 error, alpha = 5: 5 / 30
    yh = y + np.array([3.0, 0.0, -4.0])
    assert abs(bandit.reward(y, yh, 5.0) - 1.0 / 6.0) < 1e-15
    rng = np.random.default_rng(4)
    for _ in range(50):
        a, b, al = rng.standard_normal(4), rng.standard_normal(4), rng.uniform(1e-3, 2)
        assert dpf.bandit_reward(a, b, al) == pytest.approx(bandit.reward(a, b, al), rel=1e-14)
        assert 0.0 < dpf.bandit_reward(a, b, al) <= 1.0


def test_invalid_inputs_refused():
    from paper_1203_2394_gb300 import dpf
    with pytest.raises(dpf.DpfError):
        dpf.Bandit(dpf.DPF_EXP3, 3, 0.1, 0.0)
    with pytest.raises(dpf.DpfError):
        dpf.Bandit(5, 3, 0.1)
    h = dpf.Bandit(dpf.DPF_HEDGE, 2, 0.1)
    with pytest.raises(dpf.DpfError):
        h.update([0.5, 1.5])
    e = dpf.Bandit(dpf.DPF_EXP3, 2, 0.1, 0.5)
    with pytest.raises(dpf.DpfError):
        e.update([0.5])  # no choose before
