"""What the trained proposal gains: on the linear-Gaussian model lg4 (FP32), a proposal
trained on the GPU on rows the plain filter recorded raises the inner effective sample
size of every step, at an accuracy (RMSE of the filtered mean against the Kalman
filter) no worse than the plain filter's beyond Monte Carlo noise.

Inner ESS of a group: (sum_j W_j)^2 / sum_j W_j^2 with W = exp(lq) of the materialised
inner set, as a fraction of M, averaged over the groups and the steps.
"""
import numpy as np
import pytest

from paper_1203_2394_gb300 import workloads
from tests.kalman import kalman

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

D1, D2, DY, C, H = 2, 2, 2, 4, 256
DIN, DOUT = 2 * D1 + D2 + DY, C * (1 + 2 * D2)


def inner_ess(f):
    lq = f.read("lq").astype(np.float64)
    W = np.exp(lq - lq.max(axis=1, keepdims=True))
    return float(np.mean(W.sum(1) ** 2 / (W * W).sum(1)) / lq.shape[1])


def test_trained_proposal_raises_inner_ess_at_equal_accuracy():
    from paper_1203_2394_gb300 import dpf
    spec = workloads.make_model("lg4", 0)
    model = dpf.Model.from_spec(spec, dpf.DPF_F32)
    N, M, L = 2048, 64, 8
    # ---- training rows from the plain filter on its own trajectory ----
    _, ys_tr = workloads.simulate(spec, 10, 100)
    f = dpf.Filter(model, D1, D2, N, M, L, seed=1)
    f.set_debug(True)
    rows = []
    for t in range(10):
        f.step(ys_tr[t].astype(np.float32))
        if t >= 1:
            rows.append(f.record())
    F = torch.cat([r[0] for r in rows]); Z = torch.cat([r[1] for r in rows]); w = torch.cat([r[2] for r in rows])
    assert F.shape[0] == 9 * N * M
    f.close()
    p = dpf.Proposal(D1, D2, DY, hidden=H, components=C)
    W0 = workloads.init_mlp_weights(DIN, H, DOUT, seed=0)
    W0["b4"][C + C * D2:] = np.log(np.sqrt(0.1))
    p.set_weights(W0)
    losses = p.train(F, Z, w, batch=1024, epochs=3, lr=1e-3, seed=2)
    assert losses[-1] < losses[0]
    # ---- plain against learned on a fresh trajectory ----
    T = 25
    s_true, ys = workloads.simulate(spec, T, 200)
    km, _, _ = kalman(spec.A, spec.Q, spec.H, spec.R, spec.m0, spec.P0, ys)
    plain = dpf.Filter(model, D1, D2, N, M, L, seed=5)
    lrn = dpf.Filter(model, D1, D2, N, M, L, seed=5)
    lrn.set_proposal(p)
    ess_p, ess_l, err_p, err_l = [], [], [], []
    for t in range(T):
        y = ys[t].astype(np.float32)
        mp, _ = plain.step(y)
        ml, _ = lrn.step(y)
        if t >= 1:
            ess_p.append(inner_ess(plain))
            ess_l.append(inner_ess(lrn))
        err_p.append(mp - km[t])
        err_l.append(ml - km[t])
    rmse_p = float(np.sqrt(np.mean(np.square(err_p))))
    rmse_l = float(np.sqrt(np.mean(np.square(err_l))))
    mp_, ml_ = float(np.mean(ess_p)), float(np.mean(ess_l))
    print(f"inner ESS plain {mp_:.3f} learned {ml_:.3f}; RMSE vs Kalman plain {rmse_p:.4f} "
          f"learned {rmse_l:.4f}; training losses {losses}")
    assert ml_ > 1.1 * mp_, (mp_, ml_)
    assert rmse_l <= 1.25 * rmse_p + 0.01, (rmse_p, rmse_l)
