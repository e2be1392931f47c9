"""Helpers shared by the GPU parity tests (layout conversion, keys, tolerances)."""
import numpy as np

from oracle import oracle


def state_from_gpu(f):
    """The filter's newest materialised state in the oracle's layout (float64)."""
    x = f.read("x").astype(np.float64)
    z = f.read("z").transpose(1, 2, 0).astype(np.float64)
    lq = f.read("lq").astype(np.float64)
    return np.ascontiguousarray(x), np.ascontiguousarray(z), np.ascontiguousarray(lq)


def key(seed):
    return (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def word(seed, t, i, purpose, sub=0):
    return int(oracle.philox((t, i, (purpose << 24) | sub, 0), key(seed))[0])


def rel(a, ref):
    """|a - ref| / max(1, |ref|), elementwise."""
    a = np.asarray(a, np.float64); ref = np.asarray(ref, np.float64)
    return np.abs(a - ref) / np.maximum(1.0, np.abs(ref))


def check_lwhat(gpu, ref, tol, floor=40.0):
    """Per-draw log weights: entries within `floor` nats of their group's maximum
    must agree within tol; the others must be negligible on both sides."""
    gmax = ref.max(axis=1, keepdims=True)
    live = ref >= gmax - floor
    assert np.all(rel(gpu[live], ref[live]) <= tol), np.max(rel(gpu[live], ref[live]))
    dead = ~live
    if dead.any():
        assert np.all(gpu[dead] <= gmax.repeat(gpu.shape[1], 1)[dead] - floor / 2)
