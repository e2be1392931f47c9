"""Failure detection on the GPU without a fault: a wait that can never be satisfied (a
scan tile that publishes nothing) gives up after its bound and the call reports
DPF_E_TIMEOUT; the context stays usable and the next calls succeed."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_bounded_wait_reports_timeout_and_context_survives():
    from paper_1203_2394_gb300 import dpf
    t0 = time.perf_counter()
    with pytest.raises(dpf.DpfError) as e:
        dpf.check_bounded_wait()
    assert e.value.status == dpf.DPF_E_TIMEOUT
    assert time.perf_counter() - t0 < 60
    # the device and the library still work
    w = torch.rand(10000, dtype=torch.float64, device="cuda")
    idx = dpf.resample(w, rule=dpf.DPF_SYS_GLOBAL, u=torch.zeros(1, dtype=torch.int32, device="cuda"))
    assert idx.shape[0] == 10000
    assert int(idx.min()) >= 0 and int(idx.max()) < 10000
    assert np.all(np.diff(idx.cpu().numpy()) >= 0)


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_allocation_failure_returns_nomem_and_frees_everything():
    """A device allocation that fails part-way through dpf_create (or dpf_batch_create)
    makes the call return DPF_E_NOMEM and release everything it had allocated: the
    device's free memory afterwards equals the free memory before. The failure is made
    on the host (dpf_fail_allocation_after), not by exhausting the GPU."""
    from paper_1203_2394_gb300 import dpf, workloads
    spec = workloads.make_model("growth_clg10", 0)
    m = dpf.Model.from_spec(spec, dpf.DPF_F32)
    N, M, L = 4096, 128, 16
    dpf.Filter(m, 2, 8, N, M, L, 1).close()  # warm-up: the library's modules load once
    b = dpf.Batch([m, m], [2, 2], [512, 300], [64, 128], 8, [1, 2])
    b.close()
    before = _free_bytes()
    # dpf_create makes 25 device allocations: the first, some in between, the last
    for k in (1, 2, 7, 15, 25):
        dpf.fail_allocation_after(k)
        with pytest.raises(dpf.DpfError) as e:
            dpf.Filter(m, 2, 8, N, M, L, 1)
        assert e.value.status == dpf.DPF_E_NOMEM, (k, e.value)
        assert _free_bytes() == before, k
    # a batch: inside its first member's context, and in the batch's own allocations
    for k in (5, 54):
        dpf.fail_allocation_after(k)
        with pytest.raises(dpf.DpfError) as e:
            dpf.Batch([m, m], [2, 2], [512, 300], [64, 128], 8, [1, 2])
        assert e.value.status == dpf.DPF_E_NOMEM, (k, e.value)
        assert _free_bytes() == before, k
    dpf.fail_allocation_after(0)
    f = dpf.Filter(m, 2, 8, N, M, L, 1)  # and the library works normally afterwards
    _, ys = workloads.simulate(spec, 2, 0)
    mean, _ = f.step(ys[0].astype(np.float32))
    assert np.all(np.isfinite(mean))
    f.close()
    assert _free_bytes() == before


def test_step_with_a_nan_observation_reports_numeric():
    """A NaN observation makes every look-ahead weight NaN: the step kernel and the outer
    stage flag it (no resampling is applied), dpf_step returns DPF_E_NUMERIC through the
    statistics mirror, the asynchronous step reports it at dpf_sync, and a new filter on
    the same device works normally."""
    from paper_1203_2394_gb300 import dpf, workloads
    spec = workloads.make_model("growth_clg10", 0)
    m = dpf.Model.from_spec(spec, dpf.DPF_F32)
    _, ys = workloads.simulate(spec, 3, 0)
    bad = np.full(spec.dy, np.nan, dtype=np.float32)
    f = dpf.Filter(m, 2, 8, 256, 128, 16, 1)
    f.step(ys[0].astype(np.float32))
    with pytest.raises(dpf.DpfError) as e:
        f.step(bad)
    assert e.value.status == dpf.DPF_E_NUMERIC
    f.close()
    g = dpf.Filter(m, 2, 8, 256, 128, 16, 2)
    g.step(ys[0].astype(np.float32))
    yd = torch.tensor(bad, device="cuda")
    g.step_device(yd.data_ptr())
    with pytest.raises(dpf.DpfError) as e:
        g.sync()
    assert e.value.status == dpf.DPF_E_NUMERIC
    g.close()
    h = dpf.Filter(m, 2, 8, 256, 128, 16, 3)
    for t in range(3):
        mean, _ = h.step(ys[t].astype(np.float32))
        assert np.all(np.isfinite(mean))
    h.close()
