"""The paper's benchmark models (Table 1) on the GPU (dpf_create and dpf_create_pf with
DPF_MODEL_PAPER1 / DPF_MODEL_PAPER2, FP32) against the oracle of oracle/nl.py.

* The initial particles equal the oracle's draws.
* LA-DPF, teacher-forced call by call: from the GPU's state of step t-1 the oracle's
  look-ahead gives the same draws xbb (2e-5), per-draw weights and outer weights (2e-4,
  the FP32 rounding of the growth terms amplified by the z^2 / 20 observation); the outer
  ancestors equal the oracle's systematic resampling of the GPU's weights bit for bit; the
  next call's selection equals the oracle's (all but 0.2%), its x_t is the selected draw
  exactly, and its inner update matches the oracle's in all but 1% of the groups (an FP32
  weight that lands on the other side of a systematic point moves one inner particle).
  Cases with ragged M (45, 20 threads of a warp) and L (7), the largest L (32), and edge
  sizes (N = M = L = 1; M = 1 with L = 32; M = 700).
* The filtered mean equals the oracle's weighted look-ahead estimate.
* The bootstrap particle filter, teacher-forced: the same particles and weights.
* The DPF without look-ahead (dpf_create_std), teacher-forced, with the Monte Carlo mixture
  prior and its Gaussian approximation: the same particles and weights in all but 1% of
  the groups, the outer ancestors bit for bit.
* Model 1 decomposed the other way (perm = (1, 0)): the LA-DPF and the particle filter as
  above, the filtered mean returned in the table's order.
* The benchmark's size (N = 65536, M = 128, L = 16): sampled groups of two calls.
"""
import numpy as np
import pytest

from oracle import nl, oracle
from paper_1203_2394_gb300 import workloads
from tests.gpu_util import check_lwhat, rel, state_from_gpu, word

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    return oracle.load()


def _la(kind, N, M, L, seed, swap=False):
    from paper_1203_2394_gb300 import dpf
    pm = dpf.PaperModel(kind, perm=(1, 0) if swap else None)
    return dpf.Filter(pm, pm.d1, pm.d2, N, M, L, seed)


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
    _, ys = workloads.simulate_paper(kind, T, 0)
    x0, z0, lq0 = state_from_gpu(f)
    ox, oz, olq = nl.init(m, N, M, seed, lib)
    assert np.max(rel(x0, ox)) <= 2e-6 and np.max(rel(z0, oz)) <= 2e-6
    assert np.max(rel(lq0, olq)) <= 1e-6
    prev, bad_groups, bad_draws, bad_sel = None, 0, 0, 0
    for t in range(1, T + 1):
        y = np.float32(ys[t - 1, 0])
        mean, _ = f.step(np.array([y]))
        x, z, lq = state_from_gpu(f)  # the state of step t-1
        lw = f.read("lw").astype(np.float64)
        lwhat = f.read("lwhat").astype(np.float64)
        xbb = f.read("xbb").astype(np.float64)
        elw, elwhat, exbb, _, emu = nl.lookahead(m, seed, t, float(y), x, z, lq, L, np.arange(N), lib)
        # a component pick decided the other way in FP32 moves one draw of a group
        same = np.all(rel(xbb, exbb) <= 2e-5, axis=(1, 2))
        bad_draws += int((~same).sum())
        assert np.max(rel(lw[same], elw[same])) <= 2e-4, (t, np.max(rel(lw[same], elw[same])))
        check_lwhat(lwhat[same], elwhat[same], 2e-4)
        em = np.empty(m.d)
        em[m.perm] = _oracle_mean(elwhat, exbb, emu)  # the mean comes back in the table's order
        assert np.max(rel(mean, em)) <= 2e-3, (t, mean, em)
        wout = f.read("wout").astype(np.float64)
        anc = f.read("anc")
        np.testing.assert_array_equal(anc, oracle.sys_global(wout, word(seed, t, 0, oracle.P_OUTER), lib))
        if prev is not None:  # this call ran the inner update of step t-1 first
            pa, px, pz, plq, plwhat, pxbb = prev
            sel = f.read("sel")
            ref_sel = np.array([oracle.sys_local(np.exp(plwhat[a] - plwhat[a].max()), 1,
                                                 word(seed, t - 1, i, oracle.P_SEL), lib)[0]
                                for i, a in enumerate(pa)])
            bad_sel += int((sel != ref_sel).sum())
            np.testing.assert_array_equal(x, pxbb[pa, sel])
            ez, elq, _ = nl.finalize(m, seed, t - 1, float(np.float32(ys[t - 2, 0])), np.arange(N), pa, px, pz,
                                     plq, x, lib)
            ok = np.all(rel(z, ez) <= 2e-5, axis=(1, 2)) & np.all(rel(lq, elq) <= 2e-4, axis=1)
            bad_groups += int((~ok).sum())
        prev = (anc, x, z, lq, lwhat, xbb)
    assert bad_sel <= max(1, N * T // 500), bad_sel
    assert bad_draws <= max(2, N * T // 100), bad_draws
    assert bad_groups <= max(2, N * T // 100), bad_groups


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
    prev, bad = None, 0
    for t in range(1, 4):
        y = np.float32(ys[t - 1, 0])
        f.step(np.array([y]))
        x, z, lq = state_from_gpu(f)
        lw = f.read("lw").astype(np.float64)
        xbb = f.read("xbb").astype(np.float64)
        elw, elwhat, exbb, _, _ = nl.lookahead(m, seed, t, float(y), x, z, lq, L, idx, lib)
        same = np.all(rel(xbb[idx], exbb) <= 2e-5, axis=(1, 2))
        bad += int((~same).sum())
        assert np.max(rel(lw[idx][same], elw[same])) <= 2e-4
        check_lwhat(f.read("lwhat").astype(np.float64)[idx][same], elwhat[same], 2e-4)
        wout = f.read("wout").astype(np.float64)
        anc = f.read("anc")
        np.testing.assert_array_equal(anc, oracle.sys_global(wout, word(seed, t, 0, oracle.P_OUTER), lib))
        if prev is not None:
            pa, px, pz, plq = prev
            ez, elq, _ = nl.finalize(m, seed, t - 1, float(np.float32(ys[t - 2, 0])), idx, pa[idx], px, pz, plq,
                                     x[idx], lib)
            ok = np.all(rel(z[idx], ez) <= 2e-5, axis=(1, 2)) & np.all(rel(lq[idx], elq) <= 2e-4, axis=1)
            bad += int((~ok).sum())
        prev = (anc, x, z, lq)
        assert np.all(np.isfinite(lw))
    assert bad <= 3, bad


@pytest.mark.parametrize("kind,M,gauss", [(1, 32, False), (1, 32, True), (2, 19, False), (2, 64, True)])
def test_paper_dpf_teacher_forced(kind, M, gauss, lib):
    from paper_1203_2394_gb300 import dpf
    N, seed, T = 300, 9, 5
    m = nl.PaperModel(kind)
    pm = dpf.PaperModel(kind)
    f = dpf.StandardDPF(pm, pm.d1, pm.d2, N, M, seed)
    f.set_gaussian_approx(gauss)
    _, ys = workloads.simulate_paper(kind, T, 2)
    x, z, lq = state_from_gpu(f)
    ox, oz, olq = nl.init(m, N, M, seed, lib)
    assert np.max(rel(x, ox)) <= 2e-6 and np.max(rel(z, oz)) <= 2e-6
    anc, bad = None, 0
    for t in range(1, T + 1):
        y = np.float32(ys[t - 1, 0])
        mean, _ = f.step(np.array([y]))
        gx, gz, glq = state_from_gpu(f)
        glw = f.read("lw").astype(np.float64)
        ex, ez, elq, elw = nl.std_step(m, seed, t, float(y), x, z, lq, anc, lib, gauss=gauss)
        ok = (np.all(rel(gx, ex) <= 2e-5, axis=1) & np.all(rel(gz, ez) <= 2e-5, axis=(1, 2))
              & np.all(rel(glq, elq) <= 2e-4, axis=1) & (rel(glw, elw) <= 2e-4))
        bad += int((~ok).sum())
        W = np.exp(glw - glw.max())
        W /= W.sum()
        zmean = np.einsum("nm,nmc->nc", np.exp(glq), gz)
        assert np.max(rel(mean, np.concatenate([W @ gx, W @ zmean]))) <= 1e-4
        anc = f.read("anc")
        wout = f.read("wout").astype(np.float64)
        np.testing.assert_array_equal(anc, oracle.sys_global(wout, word(seed, t, 0, oracle.P_OUTER), lib))
        x, z, lq = gx, gz, glq
    assert bad <= max(2, N * T // 100), bad


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
