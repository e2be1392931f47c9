"""The allocation-free resampler (dpf_resample_noalloc) against dpf_resample and,
bit for bit, against the oracle's global systematic rule (oracle.sys_global).

It exists for callers that cannot allocate device memory while they resample
(a loop that must not allocate after start-up, or a process whose framework
allocator holds the whole device); its scratch is a fixed per-device array.
This file runs last, so a failure here leaves the other tests' results intact.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _case(rng, n, dtype):
    w = (rng.exponential(size=n) ** 3).astype(dtype)
    w[rng.random(n) < 0.1] = 0
    if not w.any():
        w[0] = 1
    u = rng.integers(0, 2**32, 1, dtype=np.uint64).astype(np.uint32)
    return (torch.tensor(w, device="cuda"), torch.tensor(u.view(np.int32), device="cuda"))


def test_noalloc_matches_resample_twice_in_a_row():
    from paper_1203_2394_gb300 import dpf
    rng = np.random.default_rng(0)
    cases = [_case(rng, n, dt) for n, dt in [(1, np.float32), (2049, np.float32),
                                             (65536, np.float64), (1 << 20, np.float32),
                                             ((1 << 22), np.float32)]]
    for _ in range(2):  # the scratch keeps the last call's contents; each call must still agree
        for w, u in cases:
            ref = dpf.resample(w, u, dpf.DPF_SYS_GLOBAL, 1)
            got = dpf.resample_noalloc(w, u)
            assert torch.equal(got, ref), (w.numel(), w.dtype)


def test_noalloc_matches_the_oracle_bit_for_bit():
    """Independent of the library's other resampling path: the oracle's exact integer
    rule on the same weights (widened exactly to FP64) and the same uniform, at the
    largest accepted size and at a size that is not a multiple of the 2048-weight tile."""
    from oracle import oracle
    from paper_1203_2394_gb300 import dpf
    rng = np.random.default_rng(1)
    for n, dt in [(1 << 22, np.float32), (1_000_003, np.float64)]:
        w, u = _case(rng, n, dt)
        got = dpf.resample_noalloc(w, u).cpu().numpy()
        ref = oracle.sys_global(w.cpu().numpy().astype(np.float64), int(u.cpu().numpy().view(np.uint32)[0]))
        np.testing.assert_array_equal(got, ref, err_msg=f"n={n}")


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1203_2394_gb300 import dpf
    w = torch.ones((1 << 22) + 1, device="cuda")
    u = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(dpf.DpfError) as e:
        dpf.resample_noalloc(w, u)
    assert e.value.status == dpf.DPF_E_INVALID
