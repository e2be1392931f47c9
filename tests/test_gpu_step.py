"""The CUDA LA-DPF step against the FP64 oracle (same Philox streams).

FP64 (the linear-Gaussian workload lg4 at its full size, N=256, M=32, L=8,
T=50): free-running, every resampling index identical and every continuous
output within 1e-9.
FP32 (the growth/linear-Gaussian workload and lg4 in FP32, several tiles and a
ragged M): teacher-forced per step, i.e. the oracle starts each step from the
GPU's state: log-weights within 1e-5 relative (floor 1), means within 1e-4,
outer ancestors bit-exact given the weights the GPU fed to the resampler. Every
selection and local resampling index the GPU took equals the oracle's, or its
systematic point lies within the derived FP32 bound of a cumulative-weight
boundary (an explained flip; tests/gpu_util.explain_flips); the inner state of
every group matches the oracle's given the GPU's indices.
Replay (FP32, 10 steps): the oracle runs free from its own FP64 state but takes
the GPU's outer ancestors, selections and local resampling indices; the GPU's
filtered means stay within 1e-4 relative of the oracle's.
"""
import numpy as np
import pytest

from oracle import oracle
from paper_1203_2394_gb300 import workloads
from tests.gpu_util import (LOG2E, check_inner_step, check_lwhat, check_selection, explain_flips,
                            fp32_weight_relerr, rel, state_from_gpu, word)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _mk(spec, prec, N, M, L, seed, d1=None):
    from paper_1203_2394_gb300 import dpf
    d1 = spec.d1 if d1 is None else d1
    f = dpf.Filter(dpf.Model.from_spec(spec, prec), d1, spec.d - d1, N, M, L, seed)
    o = oracle.Oracle(oracle.OracleModel.from_spec(spec), N, M, L, seed, nthreads=8)
    return f, o


def test_init_matches_oracle():
    from paper_1203_2394_gb300 import dpf
    spec = workloads.make_model("lg4", 0)
    f, o = _mk(spec, dpf.DPF_F64, 100, 40, 4, 123)
    x, z, lq = state_from_gpu(f)
    xo, zo, lqo = o.init()
    np.testing.assert_allclose(x, xo, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(z, zo, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(lq, lqo, rtol=1e-14)


def test_fp64_free_running_lg4_full_size():
    from paper_1203_2394_gb300 import dpf
    spec = workloads.make_model("lg4", 0)
    sz = spec.sizes
    T, N, M, L, seed = sz["T"], sz["N"], sz["M"], sz["L"], 0
    _, ys = workloads.simulate(spec, T, 0)
    f, o = _mk(spec, dpf.DPF_F64, N, M, L, seed)
    x, z, lq = o.init()
    prev = None
    logz_ref = 0.0
    for t in range(1, T + 1):
        mean, logz = f.step(ys[t - 1])
        r = o.step(t, ys[t - 1], x, z, lq)
        logz_ref += r["logZ"]
        assert logz == pytest.approx(logz_ref, rel=1e-10, abs=1e-9)
        np.testing.assert_array_equal(f.read("anc"), r["anc"], err_msg=f"anc t={t}")
        np.testing.assert_allclose(f.read("lw"), r["lw"], rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(f.read("lwhat"), r["lwhat"], rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(mean, r["mean"], rtol=1e-9, atol=1e-9)
        if t >= 2:  # the inner step of t-1 has now run on the GPU
            np.testing.assert_array_equal(f.read("sel"), prev["sel"], err_msg=f"sel t={t - 1}")
            xg, zg, lqg = state_from_gpu(f)
            np.testing.assert_allclose(xg, prev["x"], rtol=1e-9, atol=1e-9)
            np.testing.assert_allclose(zg, prev["z"], rtol=1e-9, atol=1e-9)
            np.testing.assert_allclose(lqg, prev["lq"], rtol=1e-9, atol=1e-9)
        x, z, lq = r["x"], r["z"], r["lq"]
        prev = r


CASES = [
    # (workload, d1, N, M, L, steps)
    ("growth_clg10", 2, 384, 128, 16, 10),
    ("growth_clg10", 2, 300, 100, 8, 10),  # ragged M: 100 of 128 threads active
    ("lg4", 2, 256, 64, 8, 8),             # x transition depends on z (the general path)
    ("lg4", 2, 200, 20, 5, 6),             # M below a warp
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-N{c[2]}-M{c[3]}-L{c[4]}" for c in CASES])
def test_fp32_teacher_forced(case):
    from paper_1203_2394_gb300 import dpf
    name, d1, N, M, L, T = case
    spec = workloads.make_model(name, 0)
    _, ys = workloads.simulate(spec, T + 1, 0)
    seed = 7
    f, o = _mk(spec, dpf.DPF_F32, N, M, L, seed)
    f.set_debug(True)
    prev = None
    for t in range(1, T + 1):
        mean, _ = f.step(ys[t - 1].astype(np.float32))
        x, z, lq = state_from_gpu(f)  # the state of step t-1
        ref = o.lookahead(t, ys[t - 1].astype(np.float32), np.arange(N), x, z, lq)
        lw = f.read("lw").astype(np.float64)
        assert np.max(rel(lw, ref["lw"])) <= 1e-5, (t, np.max(rel(lw, ref["lw"])))
        check_lwhat(f.read("lwhat").astype(np.float64), ref["lwhat"], 1e-5)
        xbb = f.read("xbb").astype(np.float64)
        assert np.max(rel(xbb, ref["xbb"])) <= 1e-5
        full = o.step(t, ys[t - 1].astype(np.float32), x, z, lq)
        assert np.max(rel(mean, full["mean"])) <= 1e-4, (t, mean, full["mean"])
        # outer resampling: bit-exact given the weights the GPU used
        wout = f.read("wout").astype(np.float64)
        anc = f.read("anc")
        np.testing.assert_array_equal(anc, oracle.sys_global(wout, word(seed, t, 0, oracle.P_OUTER)))
        if prev is not None:
            # the inner step of t-1 ran at the start of this call
            pa, px, pz, plq, plwhat, pxbb = prev
            sel = f.read("sel")
            check_selection(seed, t - 1, pa, plwhat, sel)
            np.testing.assert_allclose(x, pxbb[pa, sel], rtol=0, atol=0)
            check_inner_step(o, seed, t - 1, ys[t - 2].astype(np.float32), pa, px, pz, plq, x, z, lq,
                             f.read("bidx"), x_in_alpha=(name == "lg4"))
        prev = (anc, x, z, lq, f.read("lwhat").astype(np.float64), xbb)


REPLAY = [  # (workload, N, M, L)
    ("growth_clg10", 384, 128, 16),
    ("lg4", 256, 64, 8),
]


@pytest.mark.parametrize("case", REPLAY, ids=[f"{c[0]}-N{c[1]}-M{c[2]}-L{c[3]}" for c in REPLAY])
def test_fp32_replay_10_steps(case):
    """The FP32 GPU filter against the FP64 oracle over the first 10 steps: the oracle keeps
    its own state and takes only the GPU's discrete decisions (outer ancestors, selected
    draws, local resampling indices); the filtered means stay within 1e-4 relative."""
    from paper_1203_2394_gb300 import dpf
    name, N, M, L = case
    T = 10
    spec = workloads.make_model(name, 0)
    _, ys = workloads.simulate(spec, T + 2, 0)
    ys = ys.astype(np.float32)
    seed = 3
    f, o = _mk(spec, dpf.DPF_F32, N, M, L, seed)
    f.set_debug(True)
    means, anc, sel, bidx = {}, {}, {}, {}
    for t in range(1, T + 2):
        mean, _ = f.step(ys[t - 1])
        if t <= T:
            means[t], anc[t] = mean, f.read("anc")
        if t >= 2:  # the inner step of t-1 ran at the start of call t
            sel[t - 1], bidx[t - 1] = f.read("sel"), f.read("bidx")
    x, z, lq = o.init()
    worst = 0.0
    for t in range(1, T + 1):
        r = o.step(t, ys[t - 1], x, z, lq, anc=anc[t], sel=sel[t], bidx=bidx[t])
        err = np.max(rel(means[t], r["mean"]))
        worst = max(worst, err)
        assert err <= 1e-4, (t, err, means[t], r["mean"])
        x, z, lq = r["x"], r["z"], r["lq"]
    assert worst > 0.0  # FP32 against FP64: the two really differ


def test_full_size_growth_clg10_sampled():
    """The benchmark's own workload and launch shape (N=65536, M=128, L=16): sampled
    groups against the oracle (look-ahead weights, then their selection, local
    resampling, propagation and update one call later), the outer resampling
    bit-exact on all N."""
    from paper_1203_2394_gb300 import dpf
    spec = workloads.make_model("growth_clg10", 0)
    sz = spec.sizes
    N, M, L, seed = sz["N"], sz["M"], sz["L"], 0
    _, ys = workloads.simulate(spec, 4, 0)
    f, o = _mk(spec, dpf.DPF_F32, N, M, L, seed)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(N, 256, replace=False))
    f.set_debug(True)
    prev = None
    for t in range(1, 5):
        f.step(ys[t - 1].astype(np.float32))
        x, z, lq = state_from_gpu(f)
        if t <= 3:
            ref = o.lookahead(t, ys[t - 1].astype(np.float32), idx, x, z, lq)
            lw = f.read("lw").astype(np.float64)
            assert np.max(rel(lw[idx], ref["lw"])) <= 1e-5
            check_lwhat(f.read("lwhat").astype(np.float64)[idx], ref["lwhat"], 1e-5)
            wout = f.read("wout").astype(np.float64)
            np.testing.assert_array_equal(f.read("anc"),
                                          oracle.sys_global(wout, word(seed, t, 0, oracle.P_OUTER)))
            assert np.all(np.isfinite(lw))
        if prev is not None:
            # the inner step of t-1 (selection, local resampling, propagation, update) of
            # the sampled destinations, from the full state of t-2
            pa, px, pz, plq, plwhat, pxbb = prev
            sel = f.read("sel")
            check_selection(seed, t - 1, pa[idx], plwhat, sel[idx], idx)
            np.testing.assert_allclose(x[idx], pxbb[pa[idx], sel[idx]], rtol=0, atol=0)
            bidx = f.read("bidx")[idx]
            own = o.finalize(t - 1, ys[t - 2].astype(np.float32), idx, pa[idx], px, pz, plq, x[idx])
            rep = o.finalize(t - 1, ys[t - 2].astype(np.float32), idx, pa[idx], px, pz, plq, x[idx],
                             bidx=bidx)
            for q in np.nonzero(np.any(bidx != own["bidx"], axis=1))[0]:
                al = own["alpha"][q]
                explain_flips(np.exp(al - al.max()), bidx[q], own["bidx"][q],
                              word(seed, t - 1, int(idx[q]), oracle.P_INNER), M,
                              fp32_weight_relerr((al - al.max()) * LOG2E))
            assert np.max(rel(z[idx], rep["z"])) <= 1e-5
            assert np.max(rel(lq[idx], rep["lq"])) <= 1e-5
        if t <= 3:
            prev = (f.read("anc"), x, z, lq, f.read("lwhat").astype(np.float64),
                    f.read("xbb").astype(np.float64))


def test_errors_are_status_codes():
    from paper_1203_2394_gb300 import dpf
    spec = workloads.make_model("lg4", 0)
    m = dpf.Model.from_spec(spec, dpf.DPF_F64)
    with pytest.raises(dpf.DpfError) as e:
        dpf.Filter(m, 2, 2, 0, 32, 8)
    assert e.value.status == dpf.DPF_E_INVALID
    with pytest.raises(dpf.DpfError) as e:
        dpf.Filter(m, 2, 2, 16, 2000, 8)
    assert e.value.status == dpf.DPF_E_INVALID
    with pytest.raises(dpf.DpfError) as e:
        dpf.Filter(m, 1, 3, 16, 32, 8)  # no compiled (f64, 1, 3, 2) variant
    assert e.value.status == dpf.DPF_E_UNSUPPORTED
    bad = dpf.Model(4, 2, spec.A, spec.Q + 0.05, spec.H, spec.R, spec.m0, spec.P0, dpf.DPF_F64)
    with pytest.raises(dpf.DpfError) as e:
        dpf.Filter(bad, 2, 2, 16, 32, 8)  # x/z cross-covariance in Q
    assert e.value.status == dpf.DPF_E_INVALID
