"""The DPF without look-ahead on the GPU (dpf_create_std) against its oracle.

* Teacher-forced, call by call (lg4 in FP64, the growth model in FP32), from the GPU's
  state and ancestors of call t-1: every mixture component and local resampling index
  the GPU took equals the oracle's or is an explained flip (tests/gpu_util.explain_flips);
  with the GPU's components replayed the oracle draws the same x_t; with the GPU's x_t
  and indices replayed it gives the same inner particles, inner and outer log-weights, in
  every group (FP64: 1e-11; FP32: 1e-5, relative with floor 1, but 1e-4 on the inner
  log-weights lq, see LQ_TOL). x_t enters the replay as the GPU drew it: the growth
  observation's d ell / d x ~ (x / 10) |residual| would turn x_t's own FP32 rounding
  (about 1e-6 |x|) into inner log-weight differences near 1e-4, which is the draw's
  rounding, not an error of the weights. The outer ancestors equal
  the oracle's systematic resampling of the GPU's weights bit for bit. The same in FP64
  with the Gaussian approximation of the mixture prior of x_t.
* FP64 tracks the Kalman filter on lg4.
* The comparison workload's size (N = 65536, M = 128, FP32): sampled groups of one call.
"""
import numpy as np
import pytest

from oracle import oracle, std_dpf
from paper_1203_2394_gb300 import workloads
from tests.gpu_util import LOG2E, explain_flips, fp32_weight_relerr, rel, state_from_gpu, word
from tests.kalman import kalman

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _filter(name, prec, N, M, seed):
    from paper_1203_2394_gb300 import dpf
    spec = workloads.make_model(name, 0)
    p = dpf.DPF_F64 if prec == "f64" else dpf.DPF_F32
    return spec, dpf.StandardDPF(dpf.Model.from_spec(spec, p), spec.d1, spec.d2, N, M, seed)


# The inner log-weights of this filter, lq = ell - LSE ell, are normalised by one FP32
# log-sum-exp a group whose terms hold the growth observation's x^2 / 20 (about 30 at
# |x| = 24): the normaliser's rounding shifts a whole group's lq by a few 1e-5 (7.6e-5 at
# most on these trajectories), so lq is held to 1e-4 (relative, floor 1); x_t, z and the
# outer log-weight keep 1e-5.
LQ_TOL = 1e-4


def _check_call(om, seed, t, y, x, z, lq, anc, lib, gx, gz, glq, glw, comp, bidx, tol, gauss=False,
                dest=None):
    """One call of the DPF without look-ahead for the destinations dest (all by default):
    the GPU's components and local indices equal the oracle's or are explained flips;
    x_t with the components replayed, then z, lq and log w with x_t and the indices
    replayed, within tol."""
    n = len(gx)
    dest = np.arange(n) if dest is None else np.asarray(dest)
    kw = dict(dest=dest, gauss=gauss)
    own = std_dpf.std_step(om, seed, t, y, x, z, lq, anc, lib, **kw)
    M = lq.shape[1]
    if not gauss:
        for r in np.nonzero(comp != own[5])[0]:
            a = int(dest[r]) if anc is None else int(anc[r])
            v = (lq[a] - lq[a].max()) * LOG2E
            explain_flips(np.exp(lq[a] - lq[a].max()), [comp[r]], [own[5][r]],
                          word(seed, t, int(dest[r]), oracle.P_LA_J), 1, fp32_weight_relerr(v))
    cin = None if gauss else comp
    r1 = std_dpf.std_step(om, seed, t, y, x, z, lq, anc, lib, comp_in=cin, **kw)
    assert np.max(rel(gx, r1[0])) <= tol, ("x", np.max(rel(gx, r1[0])))
    r2 = std_dpf.std_step(om, seed, t, y, x, z, lq, anc, lib, comp_in=cin, x_in=gx, return_q=True, **kw)
    for r in np.nonzero(np.any(bidx != r2[4], axis=1))[0]:
        q = r2[6][r]
        a = int(dest[r]) if anc is None else int(anc[r])
        explain_flips(np.exp(q - q.max()), bidx[r], r2[4][r], word(seed, t, int(dest[r]), oracle.P_INNER), M,
                      fp32_weight_relerr((q - q.max()) * LOG2E, 2.0 ** -18 * (1.0 + np.abs(q - lq[a]))))
    r3 = std_dpf.std_step(om, seed, t, y, x, z, lq, anc, lib, comp_in=cin, x_in=gx, bidx_in=bidx, **kw)
    for name, g, e, tl in (("z", gz, r3[1], tol), ("lq", glq, r3[2], max(tol, LQ_TOL) if tol > 1e-8 else tol),
                           ("lw", glw, r3[3], tol)):
        assert np.max(rel(g, e)) <= tl, (name, t, np.max(rel(g, e)))


@pytest.mark.parametrize("name,prec,M,gauss", [("lg4", "f64", 32, False), ("lg4", "f64", 32, True),
                                                ("growth_clg10", "f32", 64, False)])
def test_std_teacher_forced(name, prec, M, gauss):
    N, seed = 400, 9
    spec, f = _filter(name, prec, N, M, seed)
    if gauss:
        f.set_gaussian_approx(True)
    f.set_debug(True)
    om = oracle.OracleModel.from_spec(spec)
    lib = oracle.load()
    dt = np.float64 if prec == "f64" else np.float32
    tol = 1e-11 if prec == "f64" else 1e-5
    x, z, lq = state_from_gpu(f)
    ox, oz, olq = oracle.Oracle(om, N, M, 1, seed, lib=lib).init()
    assert np.max(rel(x, ox)) <= tol and np.max(rel(z, oz)) <= tol
    _, ys = workloads.simulate(spec, 5, 1)
    anc = None
    for t in range(1, 5):
        y = ys[t - 1].astype(dt)
        mean, _ = f.step(y)
        gx, gz, glq = state_from_gpu(f)
        glw = f.read("lw").astype(np.float64)
        _check_call(om, seed, t, y.astype(np.float64), x, z, lq, anc, lib, gx, gz, glq, glw,
                    f.read("jla")[:, 0], f.read("bidx"), tol, gauss)
        W = np.exp(glw - glw.max())
        W /= W.sum()
        zmean = np.einsum("nm,nmc->nc", np.exp(glq), gz)
        assert np.max(rel(mean, np.concatenate([W @ gx, W @ zmean]))) <= (1e-10 if prec == "f64" else 1e-4)
        anc = f.read("anc")
        wout = f.read("wout").astype(np.float64)
        np.testing.assert_array_equal(anc, oracle.sys_global(wout, word(seed, t, 0, oracle.P_OUTER), lib))
        x, z, lq = gx, gz, glq


def test_std_f64_tracks_kalman():
    spec, f = _filter("lg4", "f64", 20000, 32, 3)
    _, ys = workloads.simulate(spec, 15, 2)
    km, kP, _ = kalman(spec.A, spec.Q, spec.H, spec.R, spec.m0, spec.P0, ys)
    means = np.array([f.step(ys[t])[0] for t in range(15)])
    sd = np.sqrt(np.stack([np.diag(P) for P in kP]))
    err = np.max(np.abs(means - km) / sd)
    assert err < 0.15, err


def test_std_comparison_size_sampled():
    N, M, seed = 65536, 128, 5
    spec, f = _filter("growth_clg10", "f32", N, M, seed)
    om = oracle.OracleModel.from_spec(spec)
    lib = oracle.load()
    _, ys = workloads.simulate(spec, 2, 0)
    f.set_debug(True)
    f.step(ys[0].astype(np.float32))
    x, z, lq = state_from_gpu(f)
    anc = f.read("anc")
    f.step(ys[1].astype(np.float32))
    gx, gz, glq = state_from_gpu(f)
    glw = f.read("lw").astype(np.float64)
    idx = np.sort(np.random.default_rng(2).choice(N, 32, replace=False))
    _check_call(om, seed, 2, ys[1].astype(np.float32).astype(np.float64), x, z, lq, anc[idx], lib, gx[idx],
                gz[idx], glq[idx], glw[idx], f.read("jla")[idx, 0], f.read("bidx")[idx], 1e-5, dest=idx)
