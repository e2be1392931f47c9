"""The wide variant (d1 = 8, d2 = 56, dy = 8; growth_clg64) against the FP64 oracle.

Its propagation z_new = A_zz z runs on the tensor cores (tcgen05, 3xTF32, TMEM
accumulator) or, when switched off, on the CUDA cores. Both are checked
teacher-forced per step against the oracle at the FP32 tolerances of the other
FP32 variants (log-weights 1e-5 relative with floor 1, means 1e-4; every
selection and local resampling index equal or an explained flip; inner states
of every group within the tolerances given the GPU's indices; outer ancestors
bit-exact given the weights fed to the resampler), at both accepted M (128: one MMA tile
a group; 256: two) and with a ragged number of groups per CTA. The full-size
launch (N = 32768, M = 256, L = 16) is checked on sampled groups, and the two
paths are compared with each other.

The inner log-weights lq take a wider bound than at d2 = 8: lq is -1/2 |r|^2 (up
to its normaliser) with r = L_R^-1 (y - h(x) - C z), each of the dy = 8
components a 56-term FP32 dot product. With |r| about 3 and an FP32 rounding of
about 56 u |C_qc z_c| ~ 1e-6 per component, 2 dy |r| dr ~ 5e-5 absolute, so lq
is held to 1e-4 (relative, floor 1); the outer per-step log-weights stay at 1e-5.
"""
import numpy as np
import pytest

from oracle import oracle
from paper_1203_2394_gb300 import workloads
from tests.gpu_util import check_inner_step, check_lwhat, check_selection, rel, state_from_gpu, word

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LQ_TOL = 1e-4  # inner log-weights at d2 = 56 (see the module docstring)


def _mk(spec, N, M, L, seed, tc=True):
    from paper_1203_2394_gb300 import dpf
    f = dpf.Filter(dpf.Model.from_spec(spec, dpf.DPF_F32), spec.d1, spec.d2, N, M, L, seed)
    f.set_tensor_cores(tc)
    o = oracle.Oracle(oracle.OracleModel.from_spec(spec), N, M, L, seed, nthreads=16)
    return f, o


CASES = [  # (N, M, L, steps, tensor cores)
    (160, 256, 16, 5, True),
    (203, 128, 8, 4, True),
    (96, 256, 16, 4, False),
]


@pytest.mark.parametrize("case", CASES, ids=[f"N{c[0]}-M{c[1]}-L{c[2]}-{'tc' if c[4] else 'cc'}"
                                             for c in CASES])
def test_wide_teacher_forced(case):
    N, M, L, T, tc = case
    spec = workloads.make_model("growth_clg64", 0)
    _, ys = workloads.simulate(spec, T + 1, 0)
    seed = 11
    f, o = _mk(spec, N, M, L, seed, tc)
    f.set_debug(True)
    prev = None
    for t in range(1, T + 1):
        y = ys[t - 1].astype(np.float32)
        mean, _ = f.step(y)
        x, z, lq = state_from_gpu(f)
        ref = o.lookahead(t, y, np.arange(N), x, z, lq)
        lw = f.read("lw").astype(np.float64)
        assert np.max(rel(lw, ref["lw"])) <= 1e-5, (t, np.max(rel(lw, ref["lw"])))
        check_lwhat(f.read("lwhat").astype(np.float64), ref["lwhat"], 1e-5)
        xbb = f.read("xbb").astype(np.float64)
        assert np.max(rel(xbb, ref["xbb"])) <= 1e-5
        full = o.step(t, y, x, z, lq)
        assert np.max(rel(mean, full["mean"])) <= 1e-4, (t, np.max(rel(mean, full["mean"])))
        wout = f.read("wout").astype(np.float64)
        anc = f.read("anc")
        np.testing.assert_array_equal(anc, oracle.sys_global(wout, word(seed, t, 0, oracle.P_OUTER)))
        if prev is not None:
            pa, px, pz, plq, plwhat, pxbb = prev
            sel = f.read("sel")
            check_selection(seed, t - 1, pa, plwhat, sel)
            np.testing.assert_allclose(x, pxbb[pa, sel], rtol=0, atol=0)
            check_inner_step(o, seed, t - 1, ys[t - 2].astype(np.float32), pa, px, pz, plq, x, z, lq,
                             f.read("bidx"), lq_tol=LQ_TOL)
        prev = (anc, x, z, lq, f.read("lwhat").astype(np.float64), xbb)


def test_tensor_and_cuda_cores_agree():
    """Same filter, same streams: the two propagations differ only in rounding."""
    spec = workloads.make_model("growth_clg64", 1)
    _, ys = workloads.simulate(spec, 3, 1)
    N, M, L = 300, 256, 16
    a, _ = _mk(spec, N, M, L, 5, True)
    b, _ = _mk(spec, N, M, L, 5, False)
    for t in range(3):
        y = ys[t].astype(np.float32)
        ma, la = a.step(y)
        mb, lb = b.step(y)
        assert np.max(rel(ma, mb)) <= 1e-4
        assert abs(la - lb) <= 1e-4 * max(1.0, abs(lb))
    za, zb = a.read("z").astype(np.float64), b.read("z").astype(np.float64)
    same = np.all(a.read("anc") == b.read("anc"))
    assert same
    assert np.max(np.abs(za - zb)) <= 1e-4
    assert np.max(np.abs(za - zb)) > 0  # the paths really differ


def test_wide_full_size_sampled():
    """The full-size launch (N = 32768, M = 256, L = 16) on sampled groups."""
    spec = workloads.make_model("growth_clg64", 0)
    sz = spec.sizes
    N, M, L, seed = sz["N"], sz["M"], sz["L"], 0
    _, ys = workloads.simulate(spec, 3, 0)
    f, o = _mk(spec, N, M, L, seed, True)
    idx = np.sort(np.random.default_rng(1).choice(N, 96, replace=False))
    for t in range(1, 3):
        y = ys[t - 1].astype(np.float32)
        f.step(y)
        x, z, lq = state_from_gpu(f)
        ref = o.lookahead(t, y, idx, x, z, lq)
        lw = f.read("lw").astype(np.float64)
        assert np.all(np.isfinite(lw))
        assert np.max(rel(lw[idx], ref["lw"])) <= 1e-5
        check_lwhat(f.read("lwhat").astype(np.float64)[idx], ref["lwhat"], 1e-5)
        wout = f.read("wout").astype(np.float64)
        np.testing.assert_array_equal(f.read("anc"),
                                      oracle.sys_global(wout, word(seed, t, 0, oracle.P_OUTER)))


def test_wide_limits_refused():
    from paper_1203_2394_gb300 import dpf
    spec = workloads.make_model("growth_clg64", 0)
    m = dpf.Model.from_spec(spec, dpf.DPF_F32)
    with pytest.raises(dpf.DpfError) as e:
        dpf.Filter(m, 8, 56, 16, 512, 8)  # one inner particle a thread: M <= 256
    assert e.value.status == dpf.DPF_E_UNSUPPORTED


def test_wide_batch_equals_single_filters():
    """Filters of the wide variant in one batch (each its own launch of the wide step,
    with its own model, on the batch's stream; the outer stages batched): every member
    equals, bit for bit, the single filter with its seed, stepped and in a graph."""
    from paper_1203_2394_gb300 import dpf
    specs = [workloads.make_model("growth_clg64", s) for s in (0, 1)]
    models = [dpf.Model.from_spec(sp, dpf.DPF_F32) for sp in specs]
    Ns, Ms, L, seeds, T = [300, 157], [256, 128], 16, [31, 32], 4
    ys = np.stack([workloads.simulate(sp, T, 9 + f)[1] for f, sp in enumerate(specs)], axis=1).astype(np.float32)
    yd = torch.tensor(ys, device="cuda")
    b = dpf.Batch(models, [8, 8], Ns, Ms, L, seeds)
    singles = [dpf.Filter(models[f], 8, 56, Ns[f], Ms[f], L, seeds[f]) for f in range(2)]
    means = torch.zeros((T, 2, 64), dtype=torch.float64, device="cuda")
    for t in range(T // 2):
        b.step_device(yd[t].data_ptr(), means[t].data_ptr())
        if t == 0:  # the autotuner has only the one-launch-a-filter schedule to offer here
            report = b.autotune(reps=1)
            assert all(c["split"] for c in report["classes"])
    b.run_device(yd[T // 2:].data_ptr(), T - T // 2, means[T // 2:].data_ptr(), graph=True)
    for t in range(T):
        for f, s in enumerate(singles):
            ms, _ = s.step(ys[t, f])
            np.testing.assert_array_equal(means[t, f].cpu().numpy(), ms, err_msg=f"mean f={f} t={t}")
    for f, s in enumerate(singles):
        for name in ("anc", "lw", "lwhat", "x", "z", "lq"):
            np.testing.assert_array_equal(b.filter(f).read(name), s.read(name), err_msg=f"{name} f={f}")
        s.close()
    b.close()
