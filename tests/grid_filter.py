"""The exact filter of a two-dimensional state-space model by numerical integration on a grid
(a point-mass filter): the Bayes recursion
  p(s_t | y_1:t) proportional to p(y_t | s_t) sum_s' p(s_t | s') p(s' | y_1:t-1) dA
with the transition and likelihood densities written out, so that it shares nothing with
the particle filters it checks. Each source point spreads its mass as the transition's
Gaussian over the target points within 5.5 standard deviations of its mean; sources of
negligible mass are skipped. It is pinned itself to the Kalman filter on a linear model
(tests/test_oracle_nl.py); model1_posterior_means is the paper's model 1 (Table 1)."""
import numpy as np


def posterior_means(ys, xg, zg, mean_fn, obs_fn, Q, r_var=1.0, p0_sd=1.0, cut=1e-12, chunk=256):
    """For s = (x, z) with s_t = mean_fn(x, z, t - 1) + N(0, Q), y_t = obs_fn(x, z) + N(0, r_var)
    and s_0 ~ N(0, p0_sd^2 I): posterior means (T, 2) and standard deviations (T, 2) on the
    uniform grid xg x zg, the log-evidence increments log p(y_t | y_1:t-1) (T,), and the
    largest posterior mass found on the grid's boundary."""
    nx, nz = len(xg), len(zg)
    dx, dz = xg[1] - xg[0], zg[1] - zg[0]
    X, Z = np.meshgrid(xg, zg, indexing="ij")
    px, pz = X.ravel(), Z.ravel()
    dA = dx * dz
    Q = np.asarray(Q, float)
    Qi = np.linalg.inv(Q)
    lnorm = -np.log(2 * np.pi) - 0.5 * np.log(np.linalg.det(Q))
    wx, wz = int(np.ceil(5.5 * np.sqrt(Q[0, 0]) / dx)), int(np.ceil(5.5 * np.sqrt(Q[1, 1]) / dz))
    ox, oz = np.arange(-wx, wx + 1), np.arange(-wz, wz + 1)
    p = np.exp(-0.5 * (px ** 2 + pz ** 2) / p0_sd ** 2) / (2 * np.pi * p0_sd ** 2)
    edge = np.zeros(X.shape, bool)
    edge[0, :] = edge[-1, :] = edge[:, 0] = edge[:, -1] = True
    edge = edge.ravel()
    means, sds, lz, bmax = [], [], [], 0.0
    for t, y in enumerate(np.ravel(ys), start=1):
        w = p * dA
        src = np.nonzero(w > cut * w.max())[0]
        fx, fz = mean_fn(px[src], pz[src], t - 1)
        pred = np.zeros(nx * nz)
        for c in range(0, len(src), chunk):
            sl = slice(c, c + chunk)
            ix = np.rint((fx[sl] - xg[0]) / dx).astype(np.int64)[:, None] + ox  # (S, Wx)
            iz = np.rint((fz[sl] - zg[0]) / dz).astype(np.int64)[:, None] + oz  # (S, Wz)
            rx = (xg[0] + ix * dx) - fx[sl, None]
            rz = (zg[0] + iz * dz) - fz[sl, None]
            q = (Qi[0, 0] * (rx * rx)[:, :, None] + 2 * Qi[0, 1] * rx[:, :, None] * rz[:, None, :]
                 + Qi[1, 1] * (rz * rz)[:, None, :])
            val = w[src[sl], None, None] * np.exp(lnorm - 0.5 * q)
            ok = ((ix >= 0) & (ix < nx))[:, :, None] & ((iz >= 0) & (iz < nz))[:, None, :]
            flat = ix[:, :, None] * nz + iz[:, None, :]
            pred += np.bincount(flat[ok], val[ok], minlength=nx * nz)
        r = y - obs_fn(px, pz)
        p = pred * np.exp(-0.5 * r * r / r_var) / np.sqrt(2 * np.pi * r_var)
        ev = p.sum() * dA  # the predictive density of y_t, pred normalised to one below
        lz.append(np.log(ev / (pred.sum() * dA)))
        p /= ev
        m = np.array([px @ p, pz @ p]) * dA
        v = np.array([(px - m[0]) ** 2 @ p, (pz - m[1]) ** 2 @ p]) * dA
        means.append(m)
        sds.append(np.sqrt(v))
        bmax = max(bmax, p[edge].max() * dA)
    return np.array(means), np.array(sds), np.array(lz), bmax


def model1_posterior_means(ys, xg, zg, cut=1e-12, chunk=256):
    """The paper's model 1 (Table 1): x' = x + z / (1 + z^2), z' = x + 0.5 z + 25 z / (1 + z^2)
    + 8 cos(1.2 t), noise covariance [[1, 0.1], [0.1, 1]], y = atan(x) + z^2 / 20 + N(0, 1),
    s_0 ~ N(0, I)."""
    def mean_fn(x, z, s):
        return x + z / (1 + z ** 2), x + 0.5 * z + 25 * z / (1 + z ** 2) + 8 * np.cos(1.2 * s)

    def obs_fn(x, z):
        return np.arctan(x) + z ** 2 / 20

    return posterior_means(ys, xg, zg, mean_fn, obs_fn, [[1.0, 0.1], [0.1, 1.0]], cut=cut, chunk=chunk)
