"""Closed forms for linear-Gaussian state-space models (test pins).

``kalman`` is the textbook Kalman filter; ``dense_posterior`` conditions the
joint Gaussian of (s_0..s_T, y_1..y_T) directly, which pins the filter itself.
"""
import numpy as np


def kalman(A, Q, H, R, m0, P0, ys):
    """Filtered means E[s_t | y_1..t], covariances, and log p(y_t | y_1..t-1) per step."""
    m, P = np.array(m0, float), np.array(P0, float)
    means, covs, lls = [], [], []
    for y in ys:
        m = A @ m
        P = A @ P @ A.T + Q
        S = H @ P @ H.T + R
        r = y - H @ m
        Sinv_r = np.linalg.solve(S, r)
        sign, logdet = np.linalg.slogdet(S)
        lls.append(-0.5 * (r @ Sinv_r) - 0.5 * logdet - 0.5 * len(y) * np.log(2 * np.pi))
        K = P @ H.T @ np.linalg.inv(S)
        m = m + K @ r
        P = P - K @ S @ K.T
        P = 0.5 * (P + P.T)
        means.append(m.copy())
        covs.append(P.copy())
    return np.array(means), np.array(covs), np.array(lls)


def dense_posterior(A, Q, H, R, m0, P0, ys):
    """E[s_t | y_1..t] and log p(y_1..T) from the joint Gaussian, by direct conditioning."""
    T, dy = ys.shape
    d = A.shape[0]
    # s_t = A^t s_0 + sum_{u=1..t} A^{t-u} v_u ; stack (s_1..s_T) and y
    nS = (T + 1) * d
    mean_s = np.zeros(nS)
    Phi = np.zeros((nS, nS))  # maps (s_0, v_1..v_T) to (s_0..s_T)
    mean_s[:d] = m0
    for t in range(T + 1):
        for u in range(t + 1):
            Phi[t * d:(t + 1) * d, u * d:(u + 1) * d] = np.linalg.matrix_power(A, t - u)
    Cov_in = np.zeros((nS, nS))
    Cov_in[:d, :d] = P0
    for u in range(1, T + 1):
        Cov_in[u * d:(u + 1) * d, u * d:(u + 1) * d] = Q
    mu_in = np.zeros(nS)
    mu_in[:d] = m0
    mu_s = Phi @ mu_in
    Cs = Phi @ Cov_in @ Phi.T
    Hb = np.zeros((T * dy, nS))
    for t in range(1, T + 1):
        Hb[(t - 1) * dy:t * dy, t * d:(t + 1) * d] = H
    mu_y = Hb @ mu_s
    Cy = Hb @ Cs @ Hb.T + np.kron(np.eye(T), R)
    Csy = Cs @ Hb.T
    yv = ys.reshape(-1)
    means = []
    for t in range(1, T + 1):
        k = t * dy
        gain = Csy[t * d:(t + 1) * d, :k] @ np.linalg.inv(Cy[:k, :k])
        means.append(mu_s[t * d:(t + 1) * d] + gain @ (yv[:k] - mu_y[:k]))
    from scipy.stats import multivariate_normal
    ll = multivariate_normal(mean=mu_y, cov=Cy).logpdf(yv)
    return np.array(means), float(ll)
