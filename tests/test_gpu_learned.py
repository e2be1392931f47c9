"""The learned inner proposal on the GPU against the FP64 oracle (``oracle/learned.py``).

* Tensor-core forward pass: bit-exact on a network whose weights, inputs and
  activations are small integers (exact in bfloat16 and in FP32 sums), over several
  tiles and a ragged tail; on random networks within a bound derived from the
  bfloat16 rounding of the activations.
* Training kernels: loss and gradients against the oracle's backpropagation, in
  plain FP32 (tight) and with the bfloat16 forward pass; one Adam step; training
  reaches the analytic optimum of a conditional-Gaussian problem.
* Recording: the training rows of an inner update against the filter's own arrays.
* The filter's inner update with a proposal, teacher-forced per step: selection and
  local resampling bit-exact, the head outputs within the bfloat16 bound, and z and
  lq within 1e-5 of the oracle's learned update fed the GPU's head outputs; the
  look-ahead after it as in the plain tests.
"""
import numpy as np
import pytest

from oracle import learned, oracle
from paper_1203_2394_gb300 import workloads
from tests.gpu_util import check_fallback, check_lwhat, check_selection, rel, state_from_gpu, word

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

D1, D2, DY, C, H = 2, 2, 2, 4, 256
DIN, DOUT = 2 * D1 + D2 + DY, C * (1 + 2 * D2)


def _prop():
    from paper_1203_2394_gb300 import dpf
    return dpf.Proposal(D1, D2, DY, hidden=H, components=C)


def _integer_net(seed):
    rng = np.random.default_rng(seed)

    def sparse(rows, cols, nnz, vals):
        W = np.zeros((rows, cols))
        for r in range(rows):
            W[r, rng.choice(cols, nnz, replace=False)] = rng.choice(vals, nnz)
        return W
    W = {"W1": sparse(H, DIN, 4, [-1.0, 1.0]), "b1": rng.choice([-1.0, 0.0, 1.0], H),
         "W2": sparse(H, H, 4, [-1.0, 1.0]), "b2": rng.choice([-1.0, 0.0, 1.0], H),
         "W3": sparse(H, H, 4, [-1.0, 1.0]), "b3": rng.choice([-1.0, 0.0, 1.0], H),
         "W4": sparse(DOUT, H, 8, [-1.0, 1.0, 2.0]), "b4": rng.choice([-0.5, 0.0, 0.5], DOUT)}
    return W


def test_forward_exact_on_an_integer_network():
    p = _prop()
    W = _integer_net(0)
    p.set_weights(W)
    n = 1000  # 8 tiles, the last one ragged
    F = np.random.default_rng(1).integers(0, 2, (n, DIN)).astype(np.float64)
    got = p.forward(torch.tensor(F, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    ref, _ = learned.forward(W, F, bf16_mode=True)
    np.testing.assert_array_equal(got, ref)


def test_forward_random_network_within_bf16_bound():
    p = _prop()
    W = workloads.init_mlp_weights(DIN, H, DOUT, seed=3)
    rng = np.random.default_rng(4)
    for k in W:
        if k.startswith("b"):
            W[k] = 0.1 * rng.standard_normal(W[k].shape)
    p.set_weights(W)
    n = 777
    F = rng.standard_normal((n, DIN))
    got = p.forward(torch.tensor(F, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    ref, cache = learned.forward(W, F, bf16_mode=True)
    # an activation that rounds the other way moves by one bfloat16 ulp (2^-8 relative);
    # bound the output change by a few such ulps of the head's absolute dot products
    scale = np.abs(cache["h3"]) @ np.abs(learned.bf16(W["W4"])).T + np.abs(W["b4"])
    err = np.abs(got - ref)
    assert np.all(err <= 2.0 ** -6 * scale + 1e-5), float(np.max(err / (scale + 1e-9)))
    assert np.median(err / (scale + 1e-9)) < 1e-5  # most rows see no rounding flip at all


def _data(n, seed):
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((n, DIN))
    Z = rng.standard_normal((n, D2))
    w = rng.uniform(0.05, 1.0, n)
    return F, Z, w


def _dev(*arrs):
    return [torch.tensor(a, dtype=torch.float32, device="cuda") for a in arrs]


@pytest.mark.parametrize("bf16", [False, True])
def test_loss_and_gradients_match_the_oracle(bf16):
    p = _prop()
    W = workloads.init_mlp_weights(DIN, H, DOUT, seed=5)
    W["b4"] = 0.3 * np.random.default_rng(6).standard_normal(DOUT)
    p.set_weights(W)
    p.set_bf16(bf16)
    Wf = p.get_weights()  # the FP32 values the GPU holds
    F, Z, w = _data(600, 7)
    # the GPU sees FP32 inputs
    F32, Z32, w32 = (a.astype(np.float32).astype(np.float64) for a in (F, Z, w))
    loss, g = p.loss_grad(*_dev(F, Z, w))
    ref_loss, ref_g = learned.nll_and_grad(Wf, F32, Z32, w32, D2, C, bf16_mode=bf16)
    gflat = g.cpu().numpy().astype(np.float64)
    G = p.unflatten(gflat)
    if not bf16:
        assert loss == pytest.approx(ref_loss, rel=1e-5)
        for k in G:
            d = np.max(np.abs(G[k] - ref_g[k]))
            assert d <= 1e-4 * np.max(np.abs(ref_g[k])) + 1e-7, (k, d, np.max(np.abs(ref_g[k])))
    else:
        # activations that round the other way change single rows' terms by a
        # bfloat16 ulp; the sums stay close and point the same way
        assert loss == pytest.approx(ref_loss, rel=1e-3)
        for k in G:
            a, b = G[k].ravel(), ref_g[k].ravel()
            cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30)
            assert cos >= 0.999, (k, cos)
            assert np.max(np.abs(a - b)) <= 2e-2 * np.max(np.abs(b)) + 1e-7, k


def test_adam_step_matches_the_oracle():
    p = _prop()
    W = workloads.init_mlp_weights(DIN, H, DOUT, seed=8)
    p.set_weights(W)
    p.set_bf16(False)
    Wf = p.get_weights()
    rng = np.random.default_rng(9)
    gflat = rng.standard_normal(p.nparams).astype(np.float32)
    st = learned.adam_init(Wf)
    ref = Wf
    g = torch.tensor(gflat, device="cuda")
    G = p.unflatten(gflat.astype(np.float64))
    for _ in range(3):
        p.adam_step(g, 1e-3)
        ref = learned.adam_step(ref, G, st, lr=1e-3)
    got = p.get_weights()
    for k in got:
        np.testing.assert_allclose(got[k], ref[k], rtol=1e-5, atol=1e-7)


def test_training_reaches_the_conditional_optimum():
    """z = B f + s eps: the best mixture puts all components on B f with sigma = s,
    so the NLL approaches d2 (1/2 log(2 pi e) + log s)."""
    p = _prop()
    p.set_weights(workloads.init_mlp_weights(DIN, H, DOUT, seed=10))
    rng = np.random.default_rng(11)
    n = 100_000
    F = rng.standard_normal((n, DIN))
    B = rng.standard_normal((D2, DIN)) * 0.5
    s = 0.3
    Z = F @ B.T + s * rng.standard_normal((n, D2))
    w = np.ones(n)
    losses = p.train(*_dev(F, Z, w), batch=1024, epochs=8, lr=1e-3, seed=12)
    opt = D2 * (0.5 * np.log(2 * np.pi * np.e) + np.log(s))
    assert losses[0] > losses[-1]
    assert losses[-1] < opt + 0.1, (losses, opt)


def _lg4_filter(N, M, L, seed=3):
    from paper_1203_2394_gb300 import dpf
    spec = workloads.make_model("lg4", 0)
    f = dpf.Filter(dpf.Model.from_spec(spec, dpf.DPF_F32), 2, 2, N, M, L, seed)
    return spec, f


def test_recorded_rows_match_the_filter_arrays():
    N, M, L = 64, 32, 4
    spec, f = _lg4_filter(N, M, L)
    f.set_debug(True)
    _, ys = workloads.simulate(spec, 4, 0)
    for t in range(3):
        x_prev, z_prev, _ = state_from_gpu(f)
        anc = f.read("anc")
        f.step(ys[t].astype(np.float32))
    F, Z, w = (a.cpu().numpy().astype(np.float64) for a in f.record())
    x, z, lq = state_from_gpu(f)
    bidx = f.read("bidx")
    for i in (0, 17, 63):
        a = anc[i]
        for j in (0, 5, M - 1):
            e = i * M + j
            np.testing.assert_array_equal(F[e], np.concatenate([x_prev[a], x[i], z_prev[a, bidx[i, j]],
                                                                ys[1].astype(np.float32)]))
            np.testing.assert_array_equal(Z[e], z[i, j])
            assert w[e] == pytest.approx(np.exp(lq[i, j]) / N, rel=1e-6)


def test_learned_inner_update_teacher_forced():
    N, M, L, seed = 128, 64, 4, 3
    spec, f = _lg4_filter(N, M, L, seed)
    f.set_debug(True)
    om = oracle.OracleModel.from_spec(spec)
    o = oracle.Oracle(om, N, M, L, seed, nthreads=8)
    lib = oracle.load()
    p = _prop()
    W = workloads.init_mlp_weights(DIN, H, DOUT, seed=13)
    W["b4"][C + C * D2:] = np.log(np.sqrt(0.1))  # start near the prior's spread
    p.set_weights(W)
    Wq = p.get_weights()
    _, ys = workloads.simulate(spec, 6, 0)
    T = 5
    prev = None
    nfb = []
    for t in range(1, T + 1):
        if t == 2:
            f.set_proposal(p)
        y = ys[t - 1].astype(np.float32)
        f.step(y)
        x, z, lq = state_from_gpu(f)
        ref = o.lookahead(t, y, np.arange(N), x, z, lq)
        assert np.max(rel(f.read("lw"), ref["lw"])) <= 1e-5
        check_lwhat(f.read("lwhat").astype(np.float64), ref["lwhat"], 1e-5)
        if prev is not None and t >= 2:
            pa, px, pz, plq, plwhat, pxbb = prev
            sel = f.read("sel")
            check_selection(seed, t - 1, pa, plwhat, sel)  # every flip explained
            np.testing.assert_array_equal(x, pxbb[pa, sel])
            fin = o.finalize(t - 1, ys[t - 2].astype(np.float32), np.arange(N), pa, px, pz, plq, x)
            bidx = f.read("bidx")
            np.testing.assert_array_equal(bidx, fin["bidx"])
            head = f.read("head").astype(np.float64)
            # head outputs against the oracle's bfloat16 forward pass
            feats = np.concatenate([np.repeat(px[pa], M, 0), np.repeat(x, M, 0),
                                    pz[np.repeat(pa, M), bidx.ravel()],
                                    np.repeat(ys[t - 2][None].astype(np.float32), N * M, 0)], 1)
            href, cache = learned.forward(Wq, feats, bf16_mode=True)
            scale = np.abs(cache["h3"]) @ np.abs(learned.bf16(Wq["W4"])).T + np.abs(Wq["b4"])
            assert np.all(np.abs(head.reshape(-1, DOUT) - href) <= 2.0 ** -6 * scale + 1e-5)
            # the draw and the weights given the GPU's head outputs
            got = learned.learned_finalize(
                om, Wq, C, seed, t - 1, ys[t - 2].astype(np.float32), pa, px, pz, x, bidx,
                normals=lambda tt, i, pp, j, n: oracle.normals(seed, 0, tt, i, pp, j, n, lib),
                sys_local=lambda wv, k, u: oracle.sys_local(wv, k, u, lib),
                word=lambda tt, i, pp, j: word(seed, tt, i, pp, j), head_out=head)
            nfb.append(check_fallback(f.read("fallback"), z, lq, got, fin))
        prev = (f.read("anc"), x, z, lq, f.read("lwhat").astype(np.float64), f.read("xbb").astype(np.float64))
    print("groups that fell back, per step:", nfb)
    assert 0 < sum(nfb) < N * len(nfb)  # both forms of the inner update were checked


def test_learned_full_size_sampled():
    """The learned workload's launch (N = 262144, M = 64, L = 1): on sampled groups the
    head outputs within the bfloat16 bound and the draws and weights within 1e-5 of the
    oracle fed the GPU's outputs."""
    N, M, L, seed = 262144, 64, 1, 3
    spec, f = _lg4_filter(N, M, L, seed)
    f.set_debug(True)
    om = oracle.OracleModel.from_spec(spec)
    lib = oracle.load()
    p = _prop()
    W = workloads.init_mlp_weights(DIN, H, DOUT, seed=14)
    W["b4"][C + C * D2:] = np.log(np.sqrt(0.1))
    p.set_weights(W)
    Wq = p.get_weights()
    o = oracle.Oracle(om, N, M, L, seed, nthreads=8)
    _, ys = workloads.simulate(spec, 3, 0)
    f.step(ys[0].astype(np.float32))
    px, pz, plq = state_from_gpu(f)
    pa = f.read("anc")
    f.set_proposal(p)
    f.step(ys[1].astype(np.float32))
    x, z, lq = state_from_gpu(f)
    bidx = f.read("bidx")
    head = f.read("head").astype(np.float64)
    idx = np.sort(np.random.default_rng(5).choice(N, 48, replace=False))
    feats = np.concatenate([np.repeat(px[pa[idx]], M, 0), np.repeat(x[idx], M, 0),
                            pz[np.repeat(pa[idx], M), bidx[idx].ravel()],
                            np.repeat(ys[0][None].astype(np.float32), len(idx) * M, 0)], 1)
    href, cache = learned.forward(Wq, feats, bf16_mode=True)
    scale = np.abs(cache["h3"]) @ np.abs(learned.bf16(Wq["W4"])).T + np.abs(Wq["b4"])
    assert np.all(np.abs(head[idx].reshape(-1, DOUT) - href) <= 2.0 ** -6 * scale + 1e-5)
    got = learned.learned_finalize(
        om, Wq, C, seed, 1, ys[0].astype(np.float32), pa[idx], px, pz, x[idx], bidx[idx],
        normals=lambda tt, i, pp, j, n: oracle.normals(seed, 0, tt, i, pp, j, n, lib),
        sys_local=lambda wv, k, u: oracle.sys_local(wv, k, u, lib),
        word=lambda tt, i, pp, j: word(seed, tt, i, pp, j), head_out=head[idx], dest=idx)
    fin = o.finalize(1, ys[0].astype(np.float32), idx, pa[idx], px, pz, plq, x[idx])
    np.testing.assert_array_equal(bidx[idx], fin["bidx"])
    check_fallback(f.read("fallback")[idx], z[idx], lq[idx], got, fin)


@pytest.mark.parametrize("L", [4, 1])
def test_fallback_everywhere_is_the_plain_filter(L):
    """With the threshold at M (every group whose weights are not all equal falls back),
    the filter with a learned proposal steps exactly like the plain filter with the same
    seed: the same means and evidence bit for bit, and every flag set. With the
    threshold at 0 no group falls back. L = 1 runs the block step, L = 4 the warp step."""
    from paper_1203_2394_gb300 import dpf
    N, M, seed = 300, 64, 9
    spec, plain = _lg4_filter(N, M, L, seed)
    _, lrn = _lg4_filter(N, M, L, seed)
    p = _prop()
    W = workloads.init_mlp_weights(DIN, H, DOUT, seed=21)
    W["b4"][C + C * D2:] = np.log(np.sqrt(0.1))
    p.set_weights(W)
    lrn.set_proposal(p)
    lrn.set_fallback(1.0)
    _, ys = workloads.simulate(spec, 6, 0)
    for t in range(6):
        y = ys[t].astype(np.float32)
        mp, zp = plain.step(y)
        ml, zl = lrn.step(y)
        np.testing.assert_array_equal(mp, ml)
        assert zp == zl
        if t >= 1:
            assert np.all(lrn.read("fallback") == 1)
    np.testing.assert_array_equal(plain.read("z"), lrn.read("z"))
    lrn.set_fallback(0.0)
    lrn.step(ys[5].astype(np.float32))
    assert np.all(lrn.read("fallback") == 0)
    with pytest.raises(dpf.DpfError):
        lrn.set_fallback(1.5)
