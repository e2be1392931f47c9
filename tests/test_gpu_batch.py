"""The batched form: many filters of mixed N, M and x/z split stepped together.

* Every member reproduces, bit for bit, the single filter created with its seed
  (same kernels, same random-number keys), whether the members of a launch read
  their own model constants or share one set.
* A graph-captured run equals step-by-step stepping.
* Members of the d = 16 variants (splits 1/15 and 8/8, dy = 4) agree with the
  FP64 oracle, teacher-forced, within the FP32 tolerances.
* After autotuning (which may change the launch shape, hence rounding) the
  results stay within those tolerances.
"""
import numpy as np
import pytest

from oracle import oracle
from paper_1203_2394_gb300 import workloads
from tests.gpu_util import check_lwhat, rel, state_from_gpu, word

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
            pa, px, pz, plq = prev
            fin = ora.finalize(t - 1, ys[t - 2, f], np.arange(N), pa, px, pz, plq, x)
            close = np.all(rel(z, fin["z"]) <= 1e-5, axis=(1, 2))
            assert close.mean() >= 0.95, close.mean()
        prev = (m.read("anc"), x, z, lq)


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
