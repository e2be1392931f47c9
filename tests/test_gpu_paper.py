"""The paper's benchmark models (Table 1) on the GPU (dpf_create and dpf_create_pf with
DPF_MODEL_PAPER1 / DPF_MODEL_PAPER2, FP32) against the oracle of oracle/nl.py.

* The initial particles equal the oracle's draws.
* LA-DPF, teacher-forced call by call: from the GPU's state of step t-1, every mixture
  component the GPU picked for a look-ahead draw equals the oracle's pick or is an
  explained flip (tests/gpu_util.explain_flips), and with the GPU's picks replayed the
  oracle gives the same draws xbb, per-draw and outer log-weights within 1e-5 and the
  filtered mean within 1e-4 (relative, floor 1); the outer ancestors equal the oracle's
  systematic resampling of the GPU's weights bit for bit; the next call's selection and
  local resampling indices equal the oracle's or are explained flips, its x_t is the
  selected draw exactly, and the inner state of every group (z and lq within 1e-5)
  matches the oracle's given the GPU's indices.
  Cases with ragged M (45, 20 threads of a warp) and L (7), the largest L (32), and edge
  sizes (N = M = L = 1; M = 1 with L = 32; M = 700).
* The filtered mean equals the oracle's weighted look-ahead estimate.
* The bootstrap particle filter, teacher-forced: the same particles and weights.
* The DPF without look-ahead (dpf_create_std), teacher-forced, with the Monte Carlo mixture
  prior and its Gaussian approximation: components and local indices equal or explained
  flips, x_t within 1e-5 with the components replayed, z and log w within 1e-5 and lq within
  1e-4 (one FP32 log-sum-exp a group normalises it) in every group with x_t and the indices
  replayed, the outer ancestors bit for bit.
* Model 1 decomposed the other way (perm = (1, 0)): the LA-DPF and the particle filter as
  above, the filtered mean returned in the table's order.
* The benchmark's size (N = 65536, M = 128, L = 16): sampled groups of two calls.
"""
import numpy as np
import pytest

from oracle import nl, oracle
from paper_1203_2394_gb300 import workloads
from tests.gpu_util import (LOG2E, check_lwhat, check_selection, explain_flips, fp32_weight_relerr, rel,
                            state_from_gpu, word)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    return oracle.load()


def _la(kind, N, M, L, seed, swap=False):
    from paper_1203_2394_gb300 import dpf
    pm = dpf.PaperModel(kind, perm=(1, 0) if swap else None)
    return dpf.Filter(pm, pm.d1, pm.d2, N, M, L, seed)


def _explain_picks(seed, t, idx, lq, jla, ejla, lib):
    """The look-ahead's mixture components: the GPU's pick for draw m of outer particle i
    (one systematic draw on qbar = exp(lq), key (t, i, LA_J, m)) equals the oracle's or is
    an explained flip; lq is the GPU's own state, so only the FP32 weights differ."""
    n = 0
    for q, m_ in zip(*np.nonzero(jla != ejla)):
        i = int(idx[q])
        v = (lq[i] - lq[i].max()) * LOG2E
        explain_flips(np.exp(lq[i] - lq[i].max()), [jla[q, m_]], [ejla[q, m_]],
                      word(seed, t, i, oracle.P_LA_J, int(m_)), 1, fp32_weight_relerr(v))
        n += 1
    return n


def _inner_step(m, seed, t, y, idx, pa, px, pz, plq, xt, z, lq, bidx, lib):
    """Step 4's inner update of the destinations idx: every local resampling index the GPU
    took equals the oracle's or is an explained flip (alpha carries log p(x_t | x, z),
    computed in FP32: bound 2^-18 (1 + |alpha - lq|)), and with the GPU's indices the
    oracle gives the same z and lq (1e-5) in every group."""
    ez, elq, eb, al = nl.finalize(m, seed, t, y, idx, pa, px, pz, plq, xt, lib, return_alpha=True)
    for q in np.nonzero(np.any(bidx != eb, axis=1))[0]:
        a = al[q]
        explain_flips(np.exp(a - a.max()), bidx[q], eb[q], word(seed, t, int(idx[q]), oracle.P_INNER),
                      bidx.shape[1], fp32_weight_relerr((a - a.max()) * LOG2E,
                                                        2.0 ** -18 * (1.0 + np.abs(a - plq[pa[q]]))))
    rz, rlq, _ = nl.finalize(m, seed, t, y, idx, pa, px, pz, plq, xt, lib, bidx_in=bidx)
    assert np.max(rel(z, rz)) <= 1e-5, ("z", np.max(rel(z, rz)))
    assert np.max(rel(lq, rlq)) <= 1e-5, ("lq", np.max(rel(lq, rlq)))


def _oracle_mean(lwhat, xbb, mu):
    W = np.exp(lwhat - lwhat.max())
    W /= W.sum()
    return np.concatenate([np.einsum("nm,nmc->c", W, xbb), np.einsum("nm,nmc->c", W, mu)])


CASES = [
    # (kind, N, M, L, calls)
    (1, 300, 64, 8, 6),
    (1, 200, 45, 7, 5),
    (2, 300, 64, 8, 6),
    (2, 150, 20, 32, 4),
    # edge sizes: one outer particle with one inner particle and one draw; one inner
    # particle with the largest L; M = 700 (704 threads, 197 KB of shared memory)
    (1, 1, 1, 1, 3),
    (2, 5, 1, 32, 3),
    (1, 3, 700, 32, 3),
    # model 1 decomposed the other way (perm = (1, 0): the table's z outer)
    (-1, 200, 64, 8, 5),
]


@pytest.mark.parametrize("case", CASES, ids=[f"model{c[0]}-N{c[1]}-M{c[2]}-L{c[3]}".replace("model-1", "model1swap")
                                              for c in CASES])
def test_paper_la_dpf_teacher_forced(case, lib):
    kind, N, M, L, T = case
    swap, kind = kind < 0, abs(kind)
    seed = 7
    m = nl.PaperModel(kind, swap=swap)
    f = _la(kind, N, M, L, seed, swap)
    f.set_debug(True)
    _, ys = workloads.simulate_paper(kind, T, 0)
    x0, z0, lq0 = state_from_gpu(f)
    ox, oz, olq = nl.init(m, N, M, seed, lib)
    assert np.max(rel(x0, ox)) <= 2e-6 and np.max(rel(z0, oz)) <= 2e-6
    assert np.max(rel(lq0, olq)) <= 1e-6
    prev = None
    idx = np.arange(N)
    for t in range(1, T + 1):
        y = np.float32(ys[t - 1, 0])
        mean, _ = f.step(np.array([y]))
        x, z, lq = state_from_gpu(f)  # the state of step t-1
        lw = f.read("lw").astype(np.float64)
        lwhat = f.read("lwhat").astype(np.float64)
        xbb = f.read("xbb").astype(np.float64)
        jla = f.read("jla")
        _, _, _, ejla, _ = nl.lookahead(m, seed, t, float(y), x, z, lq, L, idx, lib)
        _explain_picks(seed, t, idx, lq, jla, ejla, lib)
        elw, elwhat, exbb, _, emu = nl.lookahead(m, seed, t, float(y), x, z, lq, L, idx, lib, jla_in=jla)
        assert np.max(rel(xbb, exbb)) <= 1e-5, (t, np.max(rel(xbb, exbb)))
        assert np.max(rel(lw, elw)) <= 1e-5, (t, np.max(rel(lw, elw)))
        check_lwhat(lwhat, elwhat, 1e-5)
        em = np.empty(m.d)
        em[m.perm] = _oracle_mean(elwhat, exbb, emu)  # the mean comes back in the table's order
        assert np.max(rel(mean, em)) <= 1e-4, (t, mean, em)
        wout = f.read("wout").astype(np.float64)
        anc = f.read("anc")
        np.testing.assert_array_equal(anc, oracle.sys_global(wout, word(seed, t, 0, oracle.P_OUTER), lib))
        if prev is not None:  # this call ran the inner update of step t-1 first
            pa, px, pz, plq, plwhat, pxbb = prev
            sel = f.read("sel")
            check_selection(seed, t - 1, pa, plwhat, sel)
            np.testing.assert_array_equal(x, pxbb[pa, sel])
            _inner_step(m, seed, t - 1, float(np.float32(ys[t - 2, 0])), idx, pa, px, pz, plq, x, z, lq,
                        f.read("bidx"), lib)
        prev = (anc, x, z, lq, lwhat, xbb)


@pytest.mark.parametrize("kind", [1, 2, -1])
def test_paper_pf_teacher_forced(kind, lib):
    from paper_1203_2394_gb300 import dpf
    N, seed, T = 4000, 5, 6
    swap, kind = kind < 0, abs(kind)
    m = nl.PaperModel(kind, swap=swap)
    pm = dpf.PaperModel(kind, perm=(1, 0) if swap else None)
    f = dpf.ParticleFilter(pm, pm.d1, pm.d2, N, seed)
    _, ys = workloads.simulate_paper(kind, T, 1)
    ox, oz, _ = nl.init(m, N, 1, seed, lib)
    x = f.read("x").astype(np.float64)
    z = f.read("z")[:, :, 0].T.astype(np.float64)
    assert np.max(rel(x, ox)) <= 2e-6 and np.max(rel(z, oz[:, 0])) <= 2e-6
    anc = None
    for t in range(1, T + 1):
        y = np.float32(ys[t - 1, 0])
        mean, _ = f.step(np.array([y]))
        gx = f.read("x").astype(np.float64)
        gz = f.read("z")[:, :, 0].T.astype(np.float64)
        lw = f.read("lw").astype(np.float64)
        ex, ez, elw = nl.pf_step(m, seed, t, float(y), x, z, anc, lib)
        assert np.max(rel(gx, ex)) <= 2e-5 and np.max(rel(gz, ez)) <= 2e-5
        assert np.max(rel(lw, elw)) <= 2e-4
        W = np.exp(lw - lw.max())
        em = np.empty(m.d)
        em[m.perm] = np.concatenate([W @ gx, W @ gz]) / W.sum()
        assert np.max(rel(mean, em)) <= 1e-4
        anc = f.read("anc")
        wout = f.read("wout").astype(np.float64)
        np.testing.assert_array_equal(anc, oracle.sys_global(wout, word(seed, t, 0, oracle.P_OUTER), lib))
        x, z = gx, gz


@pytest.mark.parametrize("kind", [1, 2])
def test_paper_benchmark_size_sampled(kind, lib):
    N, M, L, seed = 65536, 128, 16, 3
    m = nl.PaperModel(kind)
    f = _la(kind, N, M, L, seed)
    _, ys = workloads.simulate_paper(kind, 3, 0)
    idx = np.sort(np.random.default_rng(4).choice(N, 48, replace=False))
    f.set_debug(True)
    prev = None
    for t in range(1, 4):
        y = np.float32(ys[t - 1, 0])
        f.step(np.array([y]))
        x, z, lq = state_from_gpu(f)
        lw = f.read("lw").astype(np.float64)
        xbb = f.read("xbb").astype(np.float64)
        jla = f.read("jla")[idx]
        _, _, _, ejla, _ = nl.lookahead(m, seed, t, float(y), x, z, lq, L, idx, lib)
        _explain_picks(seed, t, idx, lq, jla, ejla, lib)
        elw, elwhat, exbb, _, _ = nl.lookahead(m, seed, t, float(y), x, z, lq, L, idx, lib, jla_in=jla)
        assert np.max(rel(xbb[idx], exbb)) <= 1e-5
        assert np.max(rel(lw[idx], elw)) <= 1e-5
        check_lwhat(f.read("lwhat").astype(np.float64)[idx], elwhat, 1e-5)
        wout = f.read("wout").astype(np.float64)
        anc = f.read("anc")
        np.testing.assert_array_equal(anc, oracle.sys_global(wout, word(seed, t, 0, oracle.P_OUTER), lib))
        if prev is not None:
            pa, px, pz, plq, plwhat, pxbb = prev
            sel = f.read("sel")
            check_selection(seed, t - 1, pa[idx], plwhat, sel[idx], idx)
            np.testing.assert_array_equal(x[idx], pxbb[pa[idx], sel[idx]])
            _inner_step(m, seed, t - 1, float(np.float32(ys[t - 2, 0])), idx, pa[idx], px, pz, plq, x[idx],
                        z[idx], lq[idx], f.read("bidx")[idx], lib)
        prev = (anc, x, z, lq, f.read("lwhat").astype(np.float64), xbb)
        assert np.all(np.isfinite(lw))


@pytest.mark.parametrize("kind,M,gauss", [(1, 32, False), (1, 32, True), (2, 19, False), (2, 64, True)])
def test_paper_dpf_teacher_forced(kind, M, gauss, lib):
    from paper_1203_2394_gb300 import dpf
    N, seed, T = 300, 9, 5
    m = nl.PaperModel(kind)
    pm = dpf.PaperModel(kind)
    f = dpf.StandardDPF(pm, pm.d1, pm.d2, N, M, seed)
    f.set_gaussian_approx(gauss)
    f.set_debug(True)
    _, ys = workloads.simulate_paper(kind, T, 2)
    x, z, lq = state_from_gpu(f)
    ox, oz, olq = nl.init(m, N, M, seed, lib)
    assert np.max(rel(x, ox)) <= 2e-6 and np.max(rel(z, oz)) <= 2e-6
    anc = None
    for t in range(1, T + 1):
        y = np.float32(ys[t - 1, 0])
        mean, _ = f.step(np.array([y]))
        gx, gz, glq = state_from_gpu(f)
        glw = f.read("lw").astype(np.float64)
        comp, bidx = f.read("jla")[:, 0], f.read("bidx")
        # the components (none for the Gaussian form): equal or explained flips
        own = nl.std_step(m, seed, t, float(y), x, z, lq, anc, lib, gauss=gauss, return_picks=True)
        if not gauss:
            for r in np.nonzero(comp != own[4])[0]:
                a = r if anc is None else int(anc[r])
                explain_flips(np.exp(lq[a] - lq[a].max()), [comp[r]], [own[4][r]],
                              word(seed, t, int(r), oracle.P_LA_J), 1,
                              fp32_weight_relerr((lq[a] - lq[a].max()) * LOG2E))
        cin = None if gauss else comp
        r1 = nl.std_step(m, seed, t, float(y), x, z, lq, anc, lib, gauss=gauss, comp_in=cin)
        assert np.max(rel(gx, r1[0])) <= 1e-5, ("x", t, np.max(rel(gx, r1[0])))
        # given the GPU's x_t: the local indices equal or explained, then the inner update
        r2 = nl.std_step(m, seed, t, float(y), x, z, lq, anc, lib, gauss=gauss, comp_in=cin, x_in=gx,
                         return_picks=True)
        for r in np.nonzero(np.any(bidx != r2[5], axis=1))[0]:
            al = r2[6][r]
            a = r if anc is None else int(anc[r])
            explain_flips(np.exp(al - al.max()), bidx[r], r2[5][r], word(seed, t, int(r), oracle.P_INNER), M,
                          fp32_weight_relerr((al - al.max()) * LOG2E, 2.0 ** -18 * (1.0 + np.abs(al - lq[a]))))
        r3 = nl.std_step(m, seed, t, float(y), x, z, lq, anc, lib, gauss=gauss, comp_in=cin, x_in=gx, bidx_in=bidx)
        # lq: one FP32 log-sum-exp a group over terms holding z^2 / 20 (up to about 30)
        # normalises it, which shifts a group's lq by up to a few 1e-5: held to 1e-4
        for name, g, e, tl in (("z", gz, r3[1], 1e-5), ("lq", glq, r3[2], 1e-4), ("lw", glw, r3[3], 1e-5)):
            assert np.max(rel(g, e)) <= tl, (name, t, np.max(rel(g, e)))
        W = np.exp(glw - glw.max())
        W /= W.sum()
        zmean = np.einsum("nm,nmc->nc", np.exp(glq), gz)
        assert np.max(rel(mean, np.concatenate([W @ gx, W @ zmean]))) <= 1e-4
        anc = f.read("anc")
        wout = f.read("wout").astype(np.float64)
        np.testing.assert_array_equal(anc, oracle.sys_global(wout, word(seed, t, 0, oracle.P_OUTER), lib))
        x, z, lq = gx, gz, glq


@pytest.mark.parametrize("kind", [1, 2])
def test_paper_dpf_and_pf_single_particle(kind, lib):
    from paper_1203_2394_gb300 import dpf
    m = nl.PaperModel(kind)
    pm = dpf.PaperModel(kind)
    _, ys = workloads.simulate_paper(kind, 3, 3)
    f = dpf.StandardDPF(pm, pm.d1, pm.d2, 1, 1, 4)
    x, z, lq = state_from_gpu(f)
    anc = None
    for t in range(1, 4):
        y = np.float32(ys[t - 1, 0])
        f.step(np.array([y]))
        gx, gz, glq = state_from_gpu(f)
        ex, ez, elq, elw = nl.std_step(m, 4, t, float(y), x, z, lq, anc, lib)
        assert np.max(rel(gx, ex)) <= 2e-5 and np.max(rel(gz, ez)) <= 2e-5
        assert np.max(rel(f.read("lw").astype(np.float64), elw)) <= 2e-4
        anc = f.read("anc")
        assert anc.tolist() == [0]
        x, z, lq = gx, gz, glq
    p = dpf.ParticleFilter(pm, pm.d1, pm.d2, 1, 4)
    x = p.read("x").astype(np.float64)
    z = p.read("z")[:, :, 0].T.astype(np.float64)
    anc = None
    for t in range(1, 4):
        y = np.float32(ys[t - 1, 0])
        mean, _ = p.step(np.array([y]))
        gx = p.read("x").astype(np.float64)
        gz = p.read("z")[:, :, 0].T.astype(np.float64)
        ex, ez, elw = nl.pf_step(m, 4, t, float(y), x, z, anc, lib)
        assert np.max(rel(gx, ex)) <= 2e-5 and np.max(rel(gz, ez)) <= 2e-5
        assert np.max(rel(mean, np.concatenate([gx[0], gz[0]]))) <= 1e-6
        anc = p.read("anc")
        x, z = gx, gz


def test_paper_model_rejections():
    from paper_1203_2394_gb300 import dpf
    pm = dpf.PaperModel(1)
    with pytest.raises(dpf.DpfError):
        dpf.Filter(pm, 1, 1, 100, 32, 33, 0)  # L > 32: the draws' weights are one warp's
    with pytest.raises(dpf.DpfError):
        dpf.Filter(pm, 2, 0, 100, 32, 8, 0)  # d1 = d2 = 1 for model 1
    with pytest.raises(dpf.DpfError):
        dpf.Filter(pm, 1, 1, 10, 1000, 32, 0)  # the pair arrays exceed the shared memory
    p2 = dpf.PaperModel(2, perm=(2, 3, 0, 1))
    with pytest.raises(dpf.DpfError):
        dpf.Filter(p2, 2, 2, 10, 32, 8, 0)  # model 2 takes the table's order only
