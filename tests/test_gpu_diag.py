"""dpf_diag_inner: the minimum and mean over the groups of the inner effective sample
size of the materialised state, against the same sums in numpy on the state read back
(FP64 and FP32 filters); equal inner weights (the initial state) give exactly M."""
import numpy as np
import pytest

from paper_1203_2394_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ess(lq):
    W = np.exp(lq.astype(np.float64))
    return W.sum(1) ** 2 / (W * W).sum(1)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_inner_ess_diagnostic(prec):
    from paper_1203_2394_gb300 import dpf
    spec = workloads.make_model("lg4", 0)
    p = dpf.DPF_F64 if prec == "f64" else dpf.DPF_F32
    N, M, L = 1000, 64, 4
    f = dpf.Filter(dpf.Model.from_spec(spec, p), 2, 2, N, M, L, seed=4)
    _, ys = workloads.simulate(spec, 6, 0)
    f.step(ys[0])
    d = f.diag_inner()
    assert d["ess_inner_min"] == pytest.approx(M, rel=1e-12)
    assert d["ess_inner_mean"] == pytest.approx(M, rel=1e-12)
    for t in range(1, 6):
        f.step(ys[t])
        d = f.diag_inner()
        e = _ess(f.read("lq"))
        assert d["ess_inner_min"] == pytest.approx(e.min(), rel=1e-12)
        assert d["ess_inner_mean"] == pytest.approx(e.mean(), rel=1e-12)
        assert 1.0 <= d["ess_inner_min"] <= d["ess_inner_mean"] <= M
