"""The outer-amortised proposal (one network row per outer particle, a diagonal affine
map of the group's prior draws) on the GPU against the oracle.

* Training: loss and gradients of the affine head against the oracle (plain FP32).
* The filter's inner update with it, teacher-forced per step: selection and local
  resampling bit-exact, the group features within 1e-5, the network outputs within
  the bfloat16 bound, z and lq within 1e-5 of the oracle fed the GPU's outputs.
* The trained form raises the inner ESS at an equal RMSE against the Kalman filter.
"""
import numpy as np
import pytest

from oracle import learned, oracle
from paper_1203_2394_gb300 import workloads
from tests.gpu_util import check_fallback, check_selection, rel, state_from_gpu, word
from tests.kalman import kalman

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

D1, D2, DY, H = 2, 2, 2, 256
DIN, DOUT = 2 * D1 + DY + 2 * D2, 2 * D2


def _spec():
    return workloads.make_model("lg4", 0)


def _prop(spec):
    from paper_1203_2394_gb300 import dpf
    om = oracle.OracleModel.from_spec(spec)
    return dpf.Proposal(D1, D2, DY, hidden=H, amortised_Qz=om.Q[D1:, D1:]), om


def test_affine_loss_and_gradients_match_the_oracle():
    spec = _spec()
    p, om = _prop(spec)
    W = workloads.init_mlp_weights(DIN, H, DOUT, seed=30)
    W["b4"] = 0.2 * np.random.default_rng(31).standard_normal(DOUT)
    p.set_weights(W)
    p.set_bf16(False)
    Wf = p.get_weights()
    rng = np.random.default_rng(32)
    n = 500
    G = rng.standard_normal((n, DIN)).astype(np.float32).astype(np.float64)
    Z = rng.standard_normal((n, 3 * D2)).astype(np.float32).astype(np.float64)
    w = rng.uniform(0.1, 1, n).astype(np.float32).astype(np.float64)
    dev = [torch.tensor(a, dtype=torch.float32, device="cuda") for a in (G, Z, w)]
    loss, g = p.loss_grad(*dev)
    ref_loss, ref_g = learned.affine_nll_and_grad(Wf, G, Z[:, :D2], Z[:, D2:2 * D2], Z[:, 2 * D2:],
                                                  om.Q[D1:, D1:], w)
    assert loss == pytest.approx(ref_loss, rel=1e-5, abs=1e-6)
    Gg = p.unflatten(g.cpu().numpy().astype(np.float64))
    for k in Gg:
        d = np.max(np.abs(Gg[k] - ref_g[k]))
        assert d <= 1e-4 * np.max(np.abs(ref_g[k])) + 1e-7, (k, d)


@pytest.mark.parametrize("centre", ["group", "particle"])
def test_amortised_inner_update_teacher_forced(centre):
    from paper_1203_2394_gb300 import dpf
    spec = _spec()
    N, M, L, seed = 200, 64, 4, 3
    f = dpf.Filter(dpf.Model.from_spec(spec, dpf.DPF_F32), D1, D2, N, M, L, seed)
    f.set_debug(True)
    p, om = _prop(spec)
    W = workloads.init_mlp_weights(DIN, H, DOUT, seed=33)
    p.set_weights(W)
    p.set_centre(centre == "particle")
    Wq = p.get_weights()
    o = oracle.Oracle(om, N, M, L, seed, nthreads=8)
    lib = oracle.load()
    _, ys = workloads.simulate(spec, 6, 0)
    prev = None
    for t in range(1, 6):
        if t == 2:
            f.set_proposal(p)
        y = ys[t - 1].astype(np.float32)
        f.step(y)
        x, z, lq = state_from_gpu(f)
        ref = o.lookahead(t, y, np.arange(N), x, z, lq)
        assert np.max(rel(f.read("lw"), ref["lw"])) <= 1e-5
        if prev is not None:
            pa, px, pz, plq, plwhat, pxbb = prev
            sel = f.read("sel")
            check_selection(seed, t - 1, pa, plwhat, sel)  # every flip explained
            np.testing.assert_array_equal(x, pxbb[pa, sel])
            fin = o.finalize(t - 1, ys[t - 2].astype(np.float32), np.arange(N), pa, px, pz, plq, x)
            bidx = f.read("bidx")
            np.testing.assert_array_equal(bidx, fin["bidx"])
            feats = f.read("afeat").astype(np.float64)
            head = f.read("ahead").astype(np.float64)
            yprev = ys[t - 2].astype(np.float32).astype(np.float64)
            got = learned.amortised_finalize(
                om, Wq, seed, t - 1, yprev, pa, px, pz, x, bidx,
                normals=lambda tt, i, pp, j, n: oracle.normals(seed, 0, tt, i, pp, j, n, lib), head_out=head,
                centre=centre)
            assert np.max(rel(feats, got["feats"])) <= 1e-5
            href, cache = learned.forward(Wq, feats, bf16_mode=True)
            scale = np.abs(cache["h3"]) @ np.abs(learned.bf16(Wq["W4"])).T + np.abs(Wq["b4"])
            assert np.all(np.abs(head - href) <= 2.0 ** -6 * scale + 1e-5)
            check_fallback(f.read("fallback"), z, lq, got, fin)
        prev = (f.read("anc"), x, z, lq, f.read("lwhat").astype(np.float64), f.read("xbb").astype(np.float64))


def _inner_ess(f):
    lq = f.read("lq").astype(np.float64)
    W = np.exp(lq - lq.max(axis=1, keepdims=True))
    return float(np.mean(W.sum(1) ** 2 / (W * W).sum(1)) / lq.shape[1])


def test_trained_amortised_proposal_raises_inner_ess():
    from paper_1203_2394_gb300 import dpf
    spec = _spec()
    model = dpf.Model.from_spec(spec, dpf.DPF_F32)
    N, M, L = 2048, 64, 8
    _, ys_tr = workloads.simulate(spec, 10, 100)
    f = dpf.Filter(model, D1, D2, N, M, L, seed=1)
    f.set_debug(True)
    rows = []
    for t in range(10):
        f.step(ys_tr[t].astype(np.float32))
        if t >= 1:
            rows.append(f.record_amortised())
    G = torch.cat([r[0] for r in rows]); Z = torch.cat([r[1] for r in rows]); w = torch.cat([r[2] for r in rows])
    f.close()
    p, om = _prop(spec)
    W0 = workloads.init_mlp_weights(DIN, H, DOUT, seed=0)
    W0["W4"][:] = 0.0
    W0["b4"][:] = 0.0  # start at the identity map (the prior)
    p.set_weights(W0)
    losses = p.train(G, Z, w, batch=1024, epochs=3, lr=1e-3, seed=2)
    assert losses[-1] < losses[0]
    T = 25
    _, ys = workloads.simulate(spec, T, 200)
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
            ess_p.append(_inner_ess(plain))
            ess_l.append(_inner_ess(lrn))
        err_p.append(mp - km[t])
        err_l.append(ml - km[t])
    rmse_p = float(np.sqrt(np.mean(np.square(err_p))))
    rmse_l = float(np.sqrt(np.mean(np.square(err_l))))
    print(f"amortised: inner ESS plain {np.mean(ess_p):.3f} learned {np.mean(ess_l):.3f}; RMSE plain "
          f"{rmse_p:.4f} learned {rmse_l:.4f}; losses {losses}")
    assert np.mean(ess_l) > 1.05 * np.mean(ess_p)
    assert rmse_l <= 1.25 * rmse_p + 0.01
