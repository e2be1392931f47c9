"""The outer stage of a step (one cooperative launch: sums, a grid barrier, the scan and
scatter of the global systematic resampling, the statistics) at sizes where every CTA
walks several chunks of outer particles, and at a ragged small size.

Checked per step against quantities computed here from the filter's own outputs:
* the ancestors, bit for bit, against the oracle's integer global rule (oracle.sys_global)
  on the weights W_i the stage fed to it and the step's uniform word;
* W_i = exp(lw_i - max lw) to FP32 rounding;
* the evidence increment, the ESS and the filtered mean (returned by the step) against
  double-precision sums of the same W_i and per-particle mean parts.
"""
import numpy as np
import pytest

from oracle import oracle
from paper_1203_2394_gb300 import workloads
from tests.gpu_util import word

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("N", [1_048_576 + 37, 3001])
def test_outer_stage_many_chunks_per_cta(N):
    from paper_1203_2394_gb300 import dpf
    spec = workloads.make_model("lg4", 0)
    M, L, seed, T = 32, 4, 11, 3
    _, ys = workloads.simulate(spec, T, 3)
    f = dpf.Filter(dpf.Model.from_spec(spec, dpf.DPF_F32), spec.d1, spec.d2, N, M, L, seed)
    for t in range(1, T + 1):
        mean, _ = f.step(ys[t - 1].astype(np.float32))
        lw = f.read("lw").astype(np.float64)
        wout = f.read("wout").astype(np.float64)
        np.testing.assert_array_equal(f.read("anc"), oracle.sys_global(wout, word(seed, t, 0, oracle.P_OUTER)))
        # W = exp(lw - max) in FP32: the difference rounds to half an ulp of itself, the
        # exponential to about an ulp
        ref = np.exp(lw - lw.max())
        assert np.all(np.abs(wout - ref) <= (np.abs(lw - lw.max()) * 2.0 ** -23 + 2.0 ** -21) * ref + 1e-38)
        parts = np.concatenate([f.read("xm"), f.read("zm")]).astype(np.float64)  # (d, N), x first
        s1, s2 = wout.sum(), (wout ** 2).sum()
        mean_ref = parts @ wout / s1  # internal order; the model's permutation is the identity
        # FP32 partial sums (a few terms a thread, then warp and block trees) combined in double
        np.testing.assert_allclose(mean, mean_ref, rtol=1e-5, atol=1e-5 * np.abs(parts).max())
        d = f.diag()
        assert d["ess"] == pytest.approx(s1 * s1 / s2, rel=1e-5)
        assert d["logZ_step"] == pytest.approx(lw.max() + np.log(s1) - np.log(N), rel=0, abs=1e-5)
    f.close()


def test_batched_outer_stage_equals_single_filters():
    """The batched form runs the same stage in two launches (sums, then prefix, scatter and
    statistics) over each member's own CTAs with the single launch's partition: at the
    same sizes its members' ancestors, weights and means equal the single filters' bit
    for bit."""
    from paper_1203_2394_gb300 import dpf
    spec = workloads.make_model("lg4", 0)
    m = dpf.Model.from_spec(spec, dpf.DPF_F32)
    Ns, M, L, seeds, T = [1_048_576 + 37, 3001], 32, 4, [21, 22], 3
    ys = np.stack([workloads.simulate(spec, T, 7 + f)[1] for f in range(2)], axis=1).astype(np.float32)
    b = dpf.Batch([m, m], [spec.d1] * 2, Ns, [M] * 2, L, seeds)
    singles = [dpf.Filter(m, spec.d1, spec.d2, N, M, L, s) for N, s in zip(Ns, seeds)]
    yd = torch.tensor(ys, device="cuda")
    means = torch.zeros((2, spec.d), dtype=torch.float64, device="cuda")
    for t in range(T):
        b.step_device(yd[t].data_ptr(), means.data_ptr())
        b.sync()
        for f, s in enumerate(singles):
            ms, _ = s.step(ys[t, f])
            for name in ("anc", "lw", "wout"):
                np.testing.assert_array_equal(b.filter(f).read(name), s.read(name), err_msg=f"{name} f={f} t={t}")
            np.testing.assert_array_equal(means[f].cpu().numpy(), ms)
    for s in singles:
        s.close()
    b.close()
