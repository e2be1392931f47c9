"""dpf_resample on the GPU is bit-exact against the oracle's integer rule."""
import numpy as np
import pytest

from oracle import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _weights(rng, n, kind):
    if kind == "random":
        return rng.exponential(size=n) ** 3
    if kind == "spiky":
        w = np.zeros(n); w[rng.integers(0, n, 3)] = [1.0, 1e-3, 1e-9]; return w
    if kind == "zeros":
        w = rng.random(n); w[rng.random(n) < 0.8] = 0
        if not w.any():
            w[n // 2] = 0.5
        return w
    if kind == "ties":
        return np.full(n, 0.25)
    if kind == "tiny":
        return rng.random(n) * 1e-30 + 1e-32
    if kind == "huge":
        return rng.random(n) * 1e30
    raise KeyError(kind)


def _u(rng, k):
    return rng.integers(0, 2**32, k, dtype=np.uint64).astype(np.uint32)


def _dev(a, dtype):
    return torch.tensor(a, dtype=dtype, device="cuda")


def _dev_u(u):
    return torch.tensor(u.view(np.int32), device="cuda")


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 1023, 2048, 2049, 65536, 262147])
@pytest.mark.parametrize("kind", ["random", "spiky", "zeros", "ties", "tiny", "huge"])
def test_global_bit_exact(n, kind, dtype):
    from paper_1203_2394_gb300 import dpf
    rng = np.random.default_rng(n * 13 + len(kind))
    w = _weights(rng, n, kind).astype(dtype)
    u = _u(rng, 1)
    got = dpf.resample(_dev(w, getattr(torch, dtype)), _dev_u(u), dpf.DPF_SYS_GLOBAL).cpu().numpy()
    ref = oracle.sys_global(w.astype(np.float64), int(u[0]))
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("seglen,nseg", [(1, 7), (7, 5), (32, 300), (100, 64), (128, 1000), (1024, 9)])
@pytest.mark.parametrize("kind", ["random", "spiky", "zeros", "ties"])
def test_local_bit_exact(seglen, nseg, kind, dtype):
    from paper_1203_2394_gb300 import dpf
    rng = np.random.default_rng(seglen * 31 + nseg + len(kind))
    w = np.concatenate([_weights(rng, seglen, kind) for _ in range(nseg)]).astype(dtype)
    u = _u(rng, nseg)
    got = dpf.resample(_dev(w, getattr(torch, dtype)), _dev_u(u), dpf.DPF_SYS_LOCAL, nseg)
    got = got.cpu().numpy().reshape(nseg, seglen)
    W = w.astype(np.float64).reshape(nseg, seglen)
    for s in range(nseg):
        np.testing.assert_array_equal(got[s], oracle.sys_local(W[s], seglen, int(u[s])))


def test_large_global_counts_invariants():
    from paper_1203_2394_gb300 import dpf
    n = (1 << 22) + 5
    rng = np.random.default_rng(1)
    w = (rng.exponential(size=n) ** 2).astype(np.float32)
    u = _u(rng, 1)
    got = dpf.resample(_dev(w, torch.float32), _dev_u(u), dpf.DPF_SYS_GLOBAL).cpu().numpy()
    assert np.all(np.diff(got) >= 0)
    counts = np.bincount(got, minlength=n)
    assert counts.sum() == n
    e = int(np.floor(np.log2(w.max())))
    c = np.floor(np.ldexp(w.astype(np.float64), 62 - 23 - e))
    frac = n * c / c.sum()
    assert np.all(counts >= np.floor(frac) - 1e-6) and np.all(counts <= np.ceil(frac) + 1e-6)


@pytest.mark.parametrize("rule", [0, 1])
def test_all_zero_weights_is_numeric_error(rule):
    from paper_1203_2394_gb300 import dpf
    w = torch.zeros(64, device="cuda")
    u = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(dpf.DpfError) as e:
        dpf.resample(w, u, rule, 1)
    assert e.value.status == dpf.DPF_E_NUMERIC


def test_negative_weight_is_numeric_error():
    from paper_1203_2394_gb300 import dpf
    w = torch.ones(100, device="cuda"); w[7] = -1
    u = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(dpf.DpfError) as e:
        dpf.resample(w, u, dpf.DPF_SYS_GLOBAL, 1)
    assert e.value.status == dpf.DPF_E_NUMERIC


def test_empty_and_bad_arguments():
    from paper_1203_2394_gb300 import dpf
    w = torch.ones(10, device="cuda")
    u = torch.zeros(2, dtype=torch.int32, device="cuda")
    with pytest.raises(dpf.DpfError) as e:
        dpf.resample(w, u, dpf.DPF_SYS_LOCAL, 3)  # 3 does not divide 10
    assert e.value.status == dpf.DPF_E_INVALID
    with pytest.raises(dpf.DpfError) as e:
        dpf.resample(torch.ones(2048, device="cuda"), u, dpf.DPF_SYS_LOCAL, 1)  # segment > 1024
    assert e.value.status == dpf.DPF_E_INVALID
    out = dpf.resample(torch.ones(0, device="cuda"), u, dpf.DPF_SYS_GLOBAL, 1)
    assert out.numel() == 0
