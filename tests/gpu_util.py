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


# ---- resampling decisions that differ between the FP32 GPU path and the FP64 oracle ----
#
# Both sides take the same exact integer rule (systematic resampling on weights quantised
# as c_i = floor(W_i 2^(S - e)), e = floor(log2 max W)), each on its own weights. Given the
# same uniform, an index can differ only where a systematic point P_j lies closer to a
# cumulative-weight boundary F_k = cum_k / C than the two sides' cumulative weights differ.
# For weights W'_i = W_i (1 + rho_i) and floors that each lose less than one unit,
#   |F'_k - F_k| <= 2 sum_i W_i rho_i / sum_i W_i + 2 n / C,
# which is the bound a differing index must meet (fp32_cum_bound).

FP32_EPS = 2.0 ** -24      # unit roundoff of binary32
EX2_REL = 2.0 ** -21       # ex2.approx.f32: relative error 2 ulp, taken twice over


def fp32_weight_relerr(v_log2, extra_abs=0.0):
    """Relative error bound of a weight 2^v evaluated as ex2.approx((a - amax) * log2 e) in
    FP32: the difference and the product are each rounded (and log2 e itself), so the
    exponent is off by at most 2.5 u |v|; the exponential adds EX2_REL. extra_abs: an
    absolute error bound (in nats) of the log-weight a itself, when the GPU computed it."""
    v = np.abs(np.asarray(v_log2, np.float64))
    return np.log(2.0) * 2.5 * FP32_EPS * v + EX2_REL + np.asarray(extra_abs, np.float64)


def _quantised_cum(W, S):
    W = np.asarray(W, np.float64)
    e = np.frexp(W.max())[1] - 1
    c = np.floor(np.ldexp(W, S - e)).astype(np.int64)
    return np.cumsum(c)


def fp32_cum_bound(W, rho, n_quant):
    """The bound on |F'_k - F_k| above: W the oracle's weights, rho their relative error
    bounds, n_quant the count of quantised terms (n) divided by C is added twice."""
    W = np.asarray(W, np.float64)
    return 2.0 * float(np.sum(W * rho) / np.sum(W)) + n_quant


def explain_flips(W, got, ref, u, n_out, rho, rule="local"):
    """Every index in `got` (GPU) that differs from `ref` (oracle) must be explained.
    W: the oracle's FP64 weights (n); u: the uniform word; n_out: number of draws; rho: the
    weights' relative error bounds (scalar or n). rule 'local' (S = 31 - ceil log2 n; b = 16,
    or b = 32 for a single draw) or 'global' (S = 62 - ceil log2 n, b = 32).
    Checks that ref is the integer rule on W, then that every differing j has its point
    P_j within the bound of the boundary between the two choices: got > ref needs
    F_{got-1} - P_j <= tol, got < ref needs P_j - F_got <= tol.
    Returns (number of differing indices, largest such distance, tol)."""
    W = np.asarray(W, np.float64)
    got = np.asarray(got).astype(np.int64)
    ref = np.asarray(ref).astype(np.int64)
    n = len(W)
    B = int(np.ceil(np.log2(n))) if n > 1 else 0
    S = (62 if rule == "global" else 31) - B
    b = 32 if (rule == "global" or n_out == 1) else 16
    ub = int(u) if b == 32 else int(u) >> 16
    cum = _quantised_cum(W, S)
    C = int(cum[-1])
    # the oracle's indices are the rule on its own quantised weights (exact integers)
    lhs = [int(ci) * n_out * (1 << b) for ci in cum]
    for j in range(n_out):
        rhs = (j * (1 << b) + ub) * C
        k = int(ref[j])
        assert lhs[k] > rhs and (k == 0 or lhs[k - 1] <= rhs), ("oracle index off the rule", j, k)
    tol = fp32_cum_bound(W, rho, 2.0 * n / C)
    F = cum.astype(np.float64) / C
    diff = np.nonzero(got != ref)[0]
    worst = 0.0
    for j in diff:
        g, r = int(got[j]), int(ref[j])
        assert 0 <= g < n, ("index out of range", j, g)
        P = (j * 2.0 ** b + ub) / (n_out * 2.0 ** b)
        d = F[g - 1] - P if g > r else P - F[g]
        worst = max(worst, d)
        assert d <= tol, ("unexplained index flip", int(j), g, r, d, tol)
    return len(diff), worst, tol


LOG2E = 1.0 / np.log(2.0)


def check_selection(seed, t, pa, plwhat, sel, idx=None):
    """Step 4's choice of x_t among the ancestor's L look-ahead draws (one systematic draw
    on exp(lwhat), key (t, i, SEL)), made by the GPU from its own FP32 lwhat (plwhat, read
    back): the oracle's rule on the same values must agree except at explained flips.
    pa, sel: ancestors and selections of the outer particles idx (default: all).
    Returns (flips, largest distance)."""
    idx = np.arange(len(pa)) if idx is None else np.asarray(idx)
    flips, worst = 0, 0.0
    for q in range(len(pa)):
        lw = plwhat[pa[q]]
        W = np.exp(lw - lw.max())
        u = word(seed, t, int(idx[q]), oracle.P_SEL)
        ref = oracle.sys_local(W, 1, u)
        if int(ref[0]) != int(sel[q]):
            n, d, _ = explain_flips(W, [sel[q]], ref, u, 1, fp32_weight_relerr((lw - lw.max()) * LOG2E))
            flips += n
            worst = max(worst, d)
    return flips, worst


def check_inner_step(o, seed, t, y, pa, px, pz, plq, x, z, lq, bidx, z_tol=1e-5, lq_tol=1e-5,
                     x_in_alpha=False):
    """Step 4 of step t for every outer particle (local resampling by alpha, propagation,
    measurement update), run by the GPU from the state (px, pz, plq) with ancestors pa
    and new x: every local resampling index it took (bidx, from the debug read-back)
    equals the oracle's or is an explained flip, and its inner state (z, lq) matches the
    oracle's given the GPU's indices in every group, flipped or not.
    x_in_alpha: alpha carries log p(x_t | x, z) computed by the GPU in FP32 (the x
    transition depends on z); its FP32 error is bounded by 2^-18 (1 + |alpha - lq|), a
    64-fold margin over four unit roundoffs of the quadratic form.
    Returns (groups with a flip, flipped indices, largest distance)."""
    N, M = bidx.shape
    idx = np.arange(N)
    own = o.finalize(t, y, idx, pa, px, pz, plq, x)
    rep = o.finalize(t, y, idx, pa, px, pz, plq, x, bidx=bidx)
    groups, flips, worst = 0, 0, 0.0
    for i in np.nonzero(np.any(bidx != own["bidx"], axis=1))[0]:
        al = own["alpha"][i]
        v = (al - al.max()) * LOG2E
        extra = 2.0 ** -18 * (1.0 + np.abs(al - plq[pa[i]])) if x_in_alpha else 0.0
        n, d, _ = explain_flips(np.exp(al - al.max()), bidx[i], own["bidx"][i],
                                word(seed, t, i, oracle.P_INNER), M, fp32_weight_relerr(v, extra))
        groups += 1
        flips += n
        worst = max(worst, d)
    assert np.max(rel(z, rep["z"])) <= z_tol, ("z", np.max(rel(z, rep["z"])))
    assert np.max(rel(lq, rep["lq"])) <= lq_tol, ("lq", np.max(rel(lq, rep["lq"])))
    return groups, flips, worst
