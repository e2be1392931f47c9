"""The CUDA LA-DPF step against the FP64 oracle (same Philox streams).

FP64 (the linear-Gaussian workload lg4 at its full size, N=256, M=32, L=8,
T=50): free-running, every resampling index identical and every continuous
output within 1e-9.
FP32 (the growth/linear-Gaussian workload and lg4 in FP32, several tiles and a
ragged M): teacher-forced per step, i.e. the oracle starts each step from the
GPU's state: log-weights within 1e-5 relative (floor 1), means within 1e-4,
outer ancestors bit-exact given the weights the GPU fed to the resampler,
inner steps exact wherever the local resampling indices agree.
"""
import numpy as np
import pytest

from oracle import oracle
from paper_1203_2394_gb300 import workloads
from tests.gpu_util import check_lwhat, rel, state_from_gpu, word

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
    ("growth_clg10", 2, 384, 128, 16, 8),
    ("growth_clg10", 2, 300, 100, 8, 6),   # ragged M: 100 of 128 threads active
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
    flips_inner = 0
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
            ref_sel = np.array([oracle.sys_local(np.exp(plwhat[pa[i]] - plwhat[pa[i]].max()), 1,
                                                 word(seed, t - 1, i, oracle.P_SEL))[0]
                                for i in range(N)])
            assert np.mean(sel != ref_sel) <= 0.002
            xsel = pxbb[pa, sel]
            np.testing.assert_allclose(x, xsel, rtol=0, atol=0)
            fin = o.finalize(t - 1, ys[t - 2].astype(np.float32), np.arange(N), pa, px, pz, plq, x)
            bidx = f.read("bidx")
            same = np.all(bidx == fin["bidx"], axis=1)
            flips_inner += int((~same).sum())
            assert np.max(rel(z[same], fin["z"][same])) <= 1e-5
            assert np.max(rel(lq[same], fin["lq"][same])) <= 1e-5
        prev = (anc, x, z, lq, f.read("lwhat").astype(np.float64), xbb)
    assert flips_inner <= max(2, N * T // 200), flips_inner


def test_full_size_growth_clg10_sampled():
    """The benchmark's own workload and launch shape (N=65536, M=128, L=16): sampled
    groups against the oracle, the outer resampling bit-exact on all N."""
    from paper_1203_2394_gb300 import dpf
    spec = workloads.make_model("growth_clg10", 0)
    sz = spec.sizes
    N, M, L, seed = sz["N"], sz["M"], sz["L"], 0
    _, ys = workloads.simulate(spec, 4, 0)
    f, o = _mk(spec, dpf.DPF_F32, N, M, L, seed)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(N, 256, replace=False))
    for t in range(1, 4):
        f.step(ys[t - 1].astype(np.float32))
        x, z, lq = state_from_gpu(f)
        ref = o.lookahead(t, ys[t - 1].astype(np.float32), idx, x, z, lq)
        lw = f.read("lw").astype(np.float64)
        assert np.max(rel(lw[idx], ref["lw"])) <= 1e-5
        check_lwhat(f.read("lwhat").astype(np.float64)[idx], ref["lwhat"], 1e-5)
        wout = f.read("wout").astype(np.float64)
        np.testing.assert_array_equal(f.read("anc"),
                                      oracle.sys_global(wout, word(seed, t, 0, oracle.P_OUTER)))
        assert np.all(np.isfinite(lw))


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
