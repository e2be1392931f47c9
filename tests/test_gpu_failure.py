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
