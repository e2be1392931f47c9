"""The batched form: many filters of mixed N, M and x/z split stepped together.

* Every member reproduces, bit for bit, the single filter created with its seed
  (same kernels, same random-number keys), whether the members of a launch read
  their own model constants or share one set.
* A graph-captured run equals step-by-step stepping, and one launch a filter (the
  autotuner's other schedule) equals one launch a class.
* Members of the d = 16 variants (splits 1/15 and 8/8, dy = 4) agree with the
  FP64 oracle, teacher-forced, within the FP32 tolerances: every selection and
  local resampling index equal or an explained flip, every group's inner state
  (z and lq) equal to the oracle's given the member's indices.
* After autotuning (which may change the launch shape, hence rounding) the
  results stay within those tolerances.
"""
import numpy as np
import pytest

from oracle import oracle
from paper_1203_2394_gb300 import workloads
from tests.gpu_util import check_inner_step, check_lwhat, check_selection, rel, state_from_gpu, word

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MEMBERS = [  # (d1, N, M)
    (1, 96, 16), (2, 130, 32), (4, 64, 64), (8, 200, 128), (2, 77, 256),
    (1, 150, 128), (8, 40, 32), (4, 300, 16), (2, 64, 64), (8, 90, 256),
]
L, T, SEED0 = 8, 5, 100


def _models(one_system=False):
    # one_system: every filter decomposes the same system, so the members of a class
    # share their model constants (the launch-parameter path of the batched kernel)
    from paper_1203_2394_gb300 import dpf
    specs = [workloads.make_model("lg16", 10 if one_system else 10 + f, d1=d1)
             for f, (d1, _, _) in enumerate(MEMBERS)]
    return specs, [dpf.Model.from_spec(s, dpf.DPF_F32) for s in specs]


def _ys(specs):
    # one observation stream per filter from its own model: ys[t, f, :]
    return np.stack([workloads.simulate(s, T, 7 + f)[1] for f, s in enumerate(specs)], axis=1)


def _batch(models):
    from paper_1203_2394_gb300 import dpf
    return dpf.Batch(models, [m[0] for m in MEMBERS], [m[1] for m in MEMBERS],
                     [m[2] for m in MEMBERS], L, [SEED0 + f for f in range(len(MEMBERS))])


@pytest.mark.parametrize("one_system", [False, True])
def test_members_equal_single_filters_bitwise(one_system):
    from paper_1203_2394_gb300 import dpf
    specs, models = _models(one_system)
    ys = _ys(specs).astype(np.float32)
    b = _batch(models)
    singles = [dpf.Filter(models[f], d1, 16 - d1, N, M, L, SEED0 + f)
               for f, (d1, N, M) in enumerate(MEMBERS)]
    yd = torch.tensor(ys, device="cuda")
    means = torch.zeros((len(MEMBERS), 16), dtype=torch.float64, device="cuda")
    for t in range(T):
        b.step_device(yd[t].data_ptr(), means.data_ptr())
        b.sync()
        for f, s in enumerate(singles):
            ms, _ = s.step(ys[t, f])
            m = b.filter(f)
            for name in ("lw", "lwhat", "anc", "sel", "x", "z", "lq"):
                np.testing.assert_array_equal(m.read(name), s.read(name), err_msg=f"{name} f={f} t={t}")
            np.testing.assert_array_equal(means[f].cpu().numpy(), ms)


def test_split_schedule_equals_fused():
    """One launch a filter (each filter's constants a launch parameter) gives the same
    bits as one launch a class (at the same inner particles per lane), stepped and in a
    graph."""
    specs, models = _models()
    ys = _ys(specs).astype(np.float32)
    yd = torch.tensor(ys, device="cuda")
    F = len(MEMBERS)
    runs = []
    for mode in ("fused", "split"):
        b = _batch(models)
        m = torch.zeros((T, F, 16), dtype=torch.float64, device="cuda")
        lz = torch.zeros((T, F), dtype=torch.float64, device="cuda")
        b.step_device(yd[0].data_ptr(), m[0].data_ptr(), lz[0].data_ptr())
        b.sync()
        if mode == "split":
            b.set_split(True)
        for t in range(1, T // 2):
            b.step_device(yd[t].data_ptr(), m[t].data_ptr(), lz[t].data_ptr())
        b.run_device(yd[T // 2:].data_ptr(), T - T // 2, m[T // 2:].data_ptr(), lz[T // 2:].data_ptr(), graph=True)
        runs.append((m, lz, [{k: b.filter(f).read(k) for k in ("z", "lq", "x", "anc", "lw")} for f in range(F)]))
        b.close()
    for m, lz, st in runs[1:]:
        assert torch.equal(m, runs[0][0]) and torch.equal(lz, runs[0][1])
        for f in range(F):
            for k in st[f]:
                np.testing.assert_array_equal(st[f][k], runs[0][2][f][k], err_msg=f"{k} f={f}")


def test_graph_run_equals_stepping():
    specs, models = _models()
    ys = _ys(specs).astype(np.float32)
    yd = torch.tensor(ys, device="cuda")
    b1, b2 = _batch(models), _batch(models)
    F = len(MEMBERS)
    m1 = torch.zeros((T, F, 16), dtype=torch.float64, device="cuda")
    l1 = torch.zeros((T, F), dtype=torch.float64, device="cuda")
    for t in range(T):
        b1.step_device(yd[t].data_ptr(), m1[t].data_ptr(), l1[t].data_ptr())
    b1.sync()
    m2 = torch.zeros_like(m1)
    l2 = torch.zeros_like(l1)
    b2.run_device(yd.data_ptr(), T, m2.data_ptr(), l2.data_ptr(), graph=True)
    assert torch.equal(m1, m2) and torch.equal(l1, l2)
    for f in range(F):
        np.testing.assert_array_equal(b1.filter(f).read("z"), b2.filter(f).read("z"))


@pytest.mark.parametrize("f", [0, 3])  # splits 1/15 and 8/8
def test_members_match_oracle_teacher_forced(f):
    specs, models = _models()
    ys = _ys(specs).astype(np.float32)
    yd = torch.tensor(ys, device="cuda")
    b = _batch(models)
    d1, N, M = MEMBERS[f]
    seed = SEED0 + f
    ora = oracle.Oracle(oracle.OracleModel.from_spec(specs[f], d1), N, M, L, seed, nthreads=8)
    b.filter(f).set_debug(True)
    prev = None
    for t in range(1, T + 1):
        b.step_device(yd[t - 1].data_ptr())
        b.sync()
        m = b.filter(f)
        x, z, lq = state_from_gpu(m)
        y = ys[t - 1, f]
        ref = ora.lookahead(t, y, np.arange(N), x, z, lq)
        assert np.max(rel(m.read("lw"), ref["lw"])) <= 1e-5
        check_lwhat(m.read("lwhat").astype(np.float64), ref["lwhat"], 1e-5)
        np.testing.assert_array_equal(
            m.read("anc"), oracle.sys_global(m.read("wout").astype(np.float64),
                                             word(seed, t, 0, oracle.P_OUTER)))
        if prev is not None:
            # the inner step of t-1 ran at the start of this call (lg16: x depends on z)
            pa, px, pz, plq, plwhat, pxbb = prev
            sel = m.read("sel")
            check_selection(seed, t - 1, pa, plwhat, sel)
            np.testing.assert_allclose(x, pxbb[pa, sel], rtol=0, atol=0)
            check_inner_step(ora, seed, t - 1, ys[t - 2, f], pa, px, pz, plq, x, z, lq, m.read("bidx"),
                             x_in_alpha=True)
        prev = (m.read("anc"), x, z, lq, m.read("lwhat").astype(np.float64),
                m.read("xbb").astype(np.float64))


def test_autotune_keeps_results_within_tolerance():
    from paper_1203_2394_gb300 import dpf
    specs, models = _models()
    ys = _ys(specs).astype(np.float32)
    yd = torch.tensor(ys, device="cuda")
    b = _batch(models)
    with pytest.raises(dpf.DpfError):  # nothing to time before the first step
        b.autotune(reps=1)
    single = [dpf.Filter(models[f], d1, 16 - d1, N, M, L, SEED0 + f) for f, (d1, N, M) in enumerate(MEMBERS)]
    b.step_device(yd[0].data_ptr())
    for s, f in zip(single, range(len(MEMBERS))):
        s.step(ys[0, f])
    report = b.autotune(reps=2)
    assert len(report["classes"]) >= 4
    for c in report["classes"]:
        assert c["chosen_ppl"] in [t["ppl"] for t in c["tried"]]
    b.step_device(yd[1].data_ptr())
    b.sync()
    for f, s in enumerate(single):
        s.step(ys[1, f])
        for name in ("lw", "lwhat"):
            assert np.max(rel(b.filter(f).read(name), s.read(name))) <= 1e-5, (name, f)


def test_full_size_batched_workload_sampled():
    """The benchmark's batched workload (512 filters of d = 16, mixed N, M and d1) in its
    graph-captured launch: sampled groups of a few members against the oracle's look-ahead
    from the member's own state, and every member's outer ancestors bit-exact."""
    from paper_1203_2394_gb300 import dpf
    rng = np.random.default_rng(0)
    F = 512
    d1s = [int(v) for v in rng.choice([1, 2, 4, 8], F)]
    Ns = [int(v) for v in rng.integers(1024, 65537, F)]
    Ms = [int(v) for v in rng.choice([16, 32, 64, 128, 256], F)]
    free, _ = torch.cuda.mem_get_info()
    need = sum(n * m * (16 - d + 1) * 4 * 2 for n, m, d in zip(Ns, Ms, d1s)) * 1.15
    if need > 0.9 * free:  # the bench runs the same proportional share
        F = max(1, int(F * 0.9 * free / need))
        d1s, Ns, Ms = d1s[:F], Ns[:F], Ms[:F]
    specs = [workloads.make_model("lg16", 1000 + f, d1=d1s[f]) for f in range(F)]
    models = [dpf.Model.from_spec(s, dpf.DPF_F32) for s in specs]
    T = 3
    ys = np.stack([workloads.simulate(s, T, 5 + f)[1] for f, s in enumerate(specs)], axis=1).astype(np.float32)
    b = dpf.Batch(models, d1s, Ns, Ms, 8, list(range(F)))
    yd = torch.tensor(ys, device="cuda")
    b.run_device(yd.data_ptr(), T, graph=True)
    # after call T the materialised state is that of step T-1: the look-ahead of step T
    # starts from it
    picks = sorted({0, int(np.argmax(Ns)), int(np.argmax(Ms)), d1s.index(8) if 8 in d1s else 1})
    states = {f: state_from_gpu(b.filter(f)) for f in picks}
    for f in picks:
        m = b.filter(f)
        x, z, lq = states[f]
        o = oracle.Oracle(oracle.OracleModel.from_spec(specs[f], d1s[f]), Ns[f], Ms[f], 8, f, nthreads=16)
        idx = np.sort(np.random.default_rng(f).choice(Ns[f], min(64, Ns[f]), replace=False))
        ref = o.lookahead(T, ys[T - 1, f], idx, x, z, lq)
        lw = m.read("lw").astype(np.float64)
        assert np.max(rel(lw[idx], ref["lw"])) <= 1e-5, (f, np.max(rel(lw[idx], ref["lw"])))
        check_lwhat(m.read("lwhat").astype(np.float64)[idx], ref["lwhat"], 1e-5)
    for f in range(F):
        m = b.filter(f)
        wout = m.read("wout").astype(np.float64)
        np.testing.assert_array_equal(m.read("anc"), oracle.sys_global(wout, word(f, T, 0, oracle.P_OUTER)))
