"""Exhaustive accuracy of the library's Box-Muller transform: every one of the
2^23 values each uniform can take, against the exact formula in FP64."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K = np.arange(1 << 23, dtype=np.uint64)
U = ((K.astype(np.float64)) + 0.5) * 2.0 ** -23


def _run(words, dtype):
    from paper_1203_2394_gb300 import dpf
    w = torch.tensor(words.astype(np.uint32).view(np.int32), device="cuda")
    out = dpf.box_muller(w, dtype).cpu().numpy().astype(np.float64)
    return out[0::2], out[1::2]


@pytest.mark.parametrize("dtype,tol", [("float32", 4e-6), ("float64", 1e-13)])
def test_radius_all_ua(dtype, tol):
    # u_b fixed at 1/8 + 2^-24 (angle near pi/4), u_a over all values
    kb = (1 << 20)
    words = np.empty(2 * K.size, np.uint64)
    words[0::2] = K << 9
    words[1::2] = kb << 9
    n0, n1 = _run(words, dtype)
    ub = (kb + 0.5) * 2.0 ** -23
    r = np.sqrt(-2 * np.log(U))
    e0 = np.abs(n0 - r * np.cos(2 * np.pi * ub))
    e1 = np.abs(n1 - r * np.sin(2 * np.pi * ub))
    assert max(e0.max(), e1.max()) <= tol, (e0.max(), e1.max(), int(np.argmax(e0)))


@pytest.mark.parametrize("dtype,tol", [("float32", 4e-6), ("float64", 1e-13)])
def test_angle_all_ub(dtype, tol):
    # u_a fixed at its smallest value (the largest radius, 5.77), u_b over all values
    words = np.empty(2 * K.size, np.uint64)
    words[0::2] = 0
    words[1::2] = K << 9
    n0, n1 = _run(words, dtype)
    r = np.sqrt(-2 * np.log(2.0 ** -24))
    e0 = np.abs(n0 - r * np.cos(2 * np.pi * U))
    e1 = np.abs(n1 - r * np.sin(2 * np.pi * U))
    assert max(e0.max(), e1.max()) <= tol, (e0.max(), e1.max())


def test_low_bits_ignored():
    rng = np.random.default_rng(0)
    w = rng.integers(0, 2**32, 2 * 4096, dtype=np.uint64)
    a = _run(w, "float32")
    b = _run(w | 0x1FF, "float32")
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
