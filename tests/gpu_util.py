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


def check_fallback(fb, z, lq, got, fin, frac=0.25, tol=1e-5):
    """The learned inner update with the per-group fallback: the GPU's flags `fb` agree
    with the oracle's rule on the oracle's learned weights (ESS < frac M), except for
    groups whose ESS lies within 1e-4 M of the threshold (the GPU decides in FP32); the
    groups that fell back match the oracle's plain update `fin`, the others its learned
    update `got`. Returns the number of groups that fell back."""
    from oracle import learned
    fb = np.asarray(fb).astype(bool)
    M = lq.shape[1]
    ess = learned.inner_ess(got["lq"])
    near = np.abs(ess - frac * M) <= 1e-4 * M
    bad = (fb != (ess < frac * M)) & ~near
    assert not bad.any(), (np.nonzero(bad)[0][:10], ess[bad][:10])
    zr = np.where(fb[:, None, None], fin["z"], got["z"])
    lqr = np.where(fb[:, None], fin["lq"], got["lq"])
    np.testing.assert_allclose(z, zr, rtol=0, atol=tol)
    assert np.max(rel(lq, lqr)) <= tol, np.max(rel(lq, lqr))
    return int(fb.sum())
