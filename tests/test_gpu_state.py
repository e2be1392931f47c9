"""Checkpoints: a filter restored from dpf_get_state continues exactly as the original
(same seed), and states of other sizes, kinds of filter or models are refused."""
import numpy as np
import pytest

from paper_1203_2394_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("name,prec", [("growth_clg10", "f32"), ("lg4", "f64")])
def test_restore_continues_bit_for_bit(name, prec):
    from paper_1203_2394_gb300 import dpf
    spec = workloads.make_model(name, 0)
    p = dpf.DPF_F32 if prec == "f32" else dpf.DPF_F64
    dt = np.float32 if prec == "f32" else np.float64
    m = dpf.Model.from_spec(spec, p)
    N, M, L = 300, 64, 8
    _, ys = workloads.simulate(spec, 10, 0)
    a = dpf.Filter(m, spec.d1, spec.d2, N, M, L, seed=4)
    for t in range(5):
        a.step(ys[t].astype(dt))
    st = a.get_state()
    b = dpf.Filter(m, spec.d1, spec.d2, N, M, L, seed=4)
    b.set_state(st)
    for t in range(5, 9):
        ma, la = a.step(ys[t].astype(dt))
        mb, lb = b.step(ys[t].astype(dt))
        np.testing.assert_array_equal(ma, mb)
        assert la == lb
        for name_ in ("lw", "anc", "sel", "z", "lq", "x"):
            np.testing.assert_array_equal(a.read(name_), b.read(name_))


def test_state_of_other_sizes_refused():
    from paper_1203_2394_gb300 import dpf
    spec = workloads.make_model("lg4", 0)
    m = dpf.Model.from_spec(spec, dpf.DPF_F64)
    a = dpf.Filter(m, 2, 2, 64, 32, 4)
    b = dpf.Filter(m, 2, 2, 64, 64, 4)
    st = a.get_state()
    big = torch.zeros(b.state_bytes(), dtype=torch.uint8, device="cuda")
    big[:st.numel()] = st
    with pytest.raises(dpf.DpfError):
        b.set_state(big)
    with pytest.raises(dpf.DpfError):
        a.set_state(st[:100])


@pytest.mark.parametrize("kind", ["pf", "std"])
def test_restore_baselines_continue_bit_for_bit(kind):
    """The bootstrap particle filter and the DPF without look-ahead restore from their own
    checkpoints (the newest particles are the state they read next), and a state of another
    kind of filter with the same sizes is refused."""
    from paper_1203_2394_gb300 import dpf
    spec = workloads.make_model("growth_clg10", 0)
    m = dpf.Model.from_spec(spec, dpf.DPF_F32)
    _, ys = workloads.simulate(spec, 9, 0)
    make = (lambda: dpf.ParticleFilter(m, 2, 8, 3000, seed=6)) if kind == "pf" else \
        (lambda: dpf.StandardDPF(m, 2, 8, 500, 64, seed=6))
    a = make()
    for t in range(4):
        a.step(ys[t].astype(np.float32))
    st = a.get_state()
    b = make()
    b.set_state(st)
    for t in range(4, 8):
        ma, la = a.step(ys[t].astype(np.float32))
        mb, lb = b.step(ys[t].astype(np.float32))
        np.testing.assert_array_equal(ma, mb)
        assert la == lb
    if kind == "std":
        other = dpf.Filter(m, 2, 8, 500, 64, 1, seed=6)
        with pytest.raises(dpf.DpfError):
            other.set_state(st)


def test_restore_paper_model_and_refuse_the_other_decomposition():
    """The LA-DPF of the paper's model 1 restores from its checkpoint and continues exactly;
    the same sizes decomposed the other way (perm = (1, 0)) refuse that state."""
    from paper_1203_2394_gb300 import dpf
    _, ys = workloads.simulate_paper(1, 9, 0)
    pm = dpf.PaperModel(1)
    a = dpf.Filter(pm, 1, 1, 400, 32, 8, seed=6)
    for t in range(4):
        a.step(ys[t].astype(np.float32))
    st = a.get_state()
    b = dpf.Filter(pm, 1, 1, 400, 32, 8, seed=6)
    b.set_state(st)
    for t in range(4, 8):
        ma, la = a.step(ys[t].astype(np.float32))
        mb, lb = b.step(ys[t].astype(np.float32))
        np.testing.assert_array_equal(ma, mb)
        assert la == lb
    swapped = dpf.Filter(dpf.PaperModel(1, perm=(1, 0)), 1, 1, 400, 32, 8, seed=6)
    with pytest.raises(dpf.DpfError):
        swapped.set_state(st)
