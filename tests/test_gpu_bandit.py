"""Automatic state decomposition over the batched form: the arms are decompositions
of one system (lg16 split x = the first d1 coordinates, d1 in {1, 2, 4, 8}), all
stepped together as members of one batch (Hedge's full-information setting, Fig.
hedge). Each step every arm earns alpha / (alpha + |y_t - H A m_{t-1}|^2) from its own
filtered mean (Section 4.3); Hedge takes the whole reward vector, Exp3 only its
chosen arm's reward.

Checks: the library's Hedge and Exp3 reproduce the oracle's probabilities (1e-12)
and Exp3's action sequence on the same rewards; Hedge's expected gain is within the
Freund-Schapire bound ln K / eta + eta T / 8 of the best arm's; the arm Hedge favours
at the end has the largest cumulative reward.
"""
import numpy as np
import pytest

from oracle import bandit, oracle
from paper_1203_2394_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

D1S = [1, 2, 4, 8]
N, M, L, T = 2048, 64, 8, 120
ALPHA, ETA, GAMMA = 1.0, 0.5, 0.2


def test_hedge_and_exp3_over_batched_decompositions():
    from paper_1203_2394_gb300 import dpf
    K = len(D1S)
    specs = [workloads.make_model("lg16", 10, d1=d1) for d1 in D1S]
    models = [dpf.Model.from_spec(s, dpf.DPF_F32) for s in specs]
    spec = specs[0]
    _, ys = workloads.simulate(spec, T, 31)
    b = dpf.Batch(models, D1S, [N] * K, [M] * K, L, [500 + k for k in range(K)])
    yd = torch.tensor(np.repeat(ys[:, None, :], K, axis=1).astype(np.float32), device="cuda")
    means = torch.zeros((K, spec.d), dtype=torch.float64, device="cuda")
    hedge = dpf.Bandit(dpf.DPF_HEDGE, K, ETA)
    exp3 = dpf.Bandit(dpf.DPF_EXP3, K, ETA, GAMMA, seed=77)
    ho = bandit.Hedge(K, ETA)
    eo = bandit.Exp3(K, ETA, GAMMA, 77, lambda c, k: oracle.philox(c, k))
    prev = np.tile(spec.m0, (K, 1))
    R = np.zeros((T, K))
    gain = 0.0
    for t in range(T):
        b.step_device(yd[t].data_ptr(), means.data_ptr())
        b.sync()
        m = means.cpu().numpy()
        assert np.all(np.isfinite(m))
        yhat = prev @ spec.A.T @ spec.H.T
        R[t] = [dpf.bandit_reward(ys[t], yhat[k], ALPHA) for k in range(K)]
        for k in range(K):
            assert R[t, k] == pytest.approx(bandit.reward(ys[t], yhat[k], ALPHA), rel=1e-14)
        p = hedge.probs()
        np.testing.assert_allclose(p, ho.p(), rtol=1e-12, atol=1e-15)
        gain += p @ R[t]
        hedge.update(R[t])
        ho.feed(R[t])
        np.testing.assert_allclose(exp3.probs(), eo.phat(), rtol=1e-12, atol=1e-15)
        a = exp3.choose()
        assert a == eo.choose()
        exp3.update(R[t, a])
        eo.feed(R[t, a])
        prev = m
    b.close()
    G = R.sum(0)
    print("cumulative rewards", G, "Hedge p", hedge.probs(), "Exp3 phat", exp3.probs())
    assert G.max() - gain <= np.log(K) / ETA + ETA * T / 8
    assert int(np.argmax(hedge.probs())) == int(np.argmax(G))
