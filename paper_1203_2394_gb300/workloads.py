"""Seeded synthetic workloads: model matrices, true trajectories, observations.

This module only draws inputs (numpy ``Generator(PCG64(seed))``); it holds none
of the filter's arithmetic. It serves both the CUDA path and the CPU oracle.

The paper evaluates on synthetic state-space models only (Table 1); the
workloads here follow the same recipe: random transition matrices rescaled to a
stated spectral radius, Gaussian noise, a true trajectory simulated from
``s_0 ~ N(m0, P0)`` and observations ``y_1..y_T`` of it.

Named workloads (sizes are the filter's, model sizes in the spec):

* ``lg4``: linear-Gaussian, d = 4 split x = 2 / z = 2, A random with spectral
  radius 0.9, Q = 0.1 I, y = H s + N(0, 0.5 I) with H 2x4 standard normal,
  T = 50, N = 256, M = 32, L = 8, FP64 (the Kalman-checked case).
* ``growth_clg10``: x of dim 2 with the growth map
  x' = 0.5 x + 25 x/(1+x^2) + 8 cos(1.2 t) + N(0, 1) per coordinate; z of dim 8
  linear-Gaussian with spectral radius 0.9 and Q_z = 0.1 I; y = x.^2/20 + C z +
  N(0, I) with C 2x8 of N(0, 1/8) entries; T = 200, N = 65536, M = 128, L = 16, FP32.
* ``lg16``: linear-Gaussian, d = 16, A spectral radius 0.9, Q = 0.1 I, dy = 4,
  H of N(0, 1/16) entries, R = 0.5 I; the x/z split d1 is chosen per filter.
* ``growth_clg64``: the growth_clg10 recipe widened: x of dim 8 (the growth map per
  coordinate, Q_x = I), z of dim 56 with a dense A_zz of spectral radius 0.95 and
  Q_z = 0.1 I, y = x.^2/20 + C z + N(0, I) with C 8x56 of N(0, 1/56) entries;
  T = 500, N = 32768, M = 256, L = 16, FP32.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class ModelSpec:
    name: str
    d: int
    d1: int
    dy: int
    A: np.ndarray
    Q: np.ndarray
    H: np.ndarray
    R: np.ndarray
    m0: np.ndarray
    P0: np.ndarray
    growth: tuple | None = None  # (a, b, c, w): a x + b x/(1+x^2) + c cos(w t) on the x block
    qc: float | None = None      # y += qc * x.^2 on the x block (dy == d1)
    sizes: dict = field(default_factory=dict)

    @property
    def d2(self) -> int:
        return self.d - self.d1

    def perm(self, d1: int | None = None):
        """Coordinate order with the x block first (identity: x = the first d1 coordinates)."""
        return list(range(self.d))

    def mean_fn(self, s: np.ndarray, t: int, d1: int | None = None) -> np.ndarray:
        """E[s_{t+1} | s_t = s] for the simulator (vectorised over leading axes)."""
        d1 = self.d1 if d1 is None else d1
        out = s @ self.A.T
        if self.growth is not None:
            a, b, c, w = self.growth
            x = s[..., :d1]
            out[..., :d1] += a * x + b * x / (1.0 + x * x) + c * np.cos(w * t)
        return out

    def obs_fn(self, s: np.ndarray, d1: int | None = None) -> np.ndarray:
        d1 = self.d1 if d1 is None else d1
        out = s @ self.H.T
        if self.qc is not None:
            out[..., :d1] += self.qc * s[..., :d1] ** 2
        return out


def random_spectral(rng: np.random.Generator, d: int, rho: float) -> np.ndarray:
    """A = G rho / rho(G) with G ~ N(0,1)^{d x d}."""
    G = rng.standard_normal((d, d))
    return G * (rho / np.max(np.abs(np.linalg.eigvals(G))))


def make_model(name: str, seed: int = 0, d1: int | None = None) -> ModelSpec:
    rng = np.random.Generator(np.random.PCG64(seed))
    if name == "lg4":
        d, dd1, dy = 4, 2, 2
        A = random_spectral(rng, d, 0.9)
        H = rng.standard_normal((dy, d))
        return ModelSpec(name, d, dd1, dy, A, 0.1 * np.eye(d), H, 0.5 * np.eye(dy), np.zeros(d),
                         np.eye(d), sizes=dict(T=50, N=256, M=32, L=8, dtype="f64"))
    if name == "growth_clg10":
        dd1, d2, dy = 2, 8, 2
        d = dd1 + d2
        A = np.zeros((d, d))
        A[dd1:, dd1:] = random_spectral(rng, d2, 0.9)
        Q = np.zeros((d, d))
        Q[:dd1, :dd1] = np.eye(dd1)
        Q[dd1:, dd1:] = 0.1 * np.eye(d2)
        H = np.zeros((dy, d))
        H[:, dd1:] = rng.standard_normal((dy, d2)) / np.sqrt(d2)
        return ModelSpec(name, d, dd1, dy, A, Q, H, np.eye(dy), np.zeros(d), np.eye(d),
                         growth=(0.5, 25.0, 8.0, 1.2), qc=1.0 / 20.0,
                         sizes=dict(T=200, N=65536, M=128, L=16, dtype="f32"))
    if name == "growth_clg64":
        dd1, d2, dy = 8, 56, 8
        d = dd1 + d2
        A = np.zeros((d, d))
        A[dd1:, dd1:] = random_spectral(rng, d2, 0.95)
        Q = np.zeros((d, d))
        Q[:dd1, :dd1] = np.eye(dd1)
        Q[dd1:, dd1:] = 0.1 * np.eye(d2)
        H = np.zeros((dy, d))
        H[:, dd1:] = rng.standard_normal((dy, d2)) / np.sqrt(d2)
        return ModelSpec(name, d, dd1, dy, A, Q, H, np.eye(dy), np.zeros(d), np.eye(d),
                         growth=(0.5, 25.0, 8.0, 1.2), qc=1.0 / 20.0,
                         sizes=dict(T=500, N=32768, M=256, L=16, dtype="f32"))
    if name == "lg16":
        d, dy = 16, 4
        A = random_spectral(rng, d, 0.9)
        H = rng.standard_normal((dy, d)) / np.sqrt(d)
        return ModelSpec(name, d, 2 if d1 is None else d1, dy, A, 0.1 * np.eye(d), H,
                         0.5 * np.eye(dy), np.zeros(d), np.eye(d),
                         sizes=dict(T=100, dtype="f32"))
    raise KeyError(name)


def simulate(spec: ModelSpec, T: int, seed: int = 0):
    """True states s_0..s_T and observations y_1..y_T (ys[t-1] is y_t)."""
    rng = np.random.Generator(np.random.PCG64(seed + 1_000_003))
    d, dy = spec.d, spec.dy
    Lq = np.linalg.cholesky(spec.Q)
    Lr = np.linalg.cholesky(spec.R)
    s = np.zeros((T + 1, d))
    s[0] = spec.m0 + np.linalg.cholesky(spec.P0) @ rng.standard_normal(d)
    ys = np.zeros((T, dy))
    for t in range(1, T + 1):
        s[t] = spec.mean_fn(s[t - 1], t - 1) + Lq @ rng.standard_normal(d)
        ys[t - 1] = spec.obs_fn(s[t]) + Lr @ rng.standard_normal(dy)
    return s, ys


def simulate_paper(kind: int, T: int, seed: int = 0):
    """A trajectory of the paper's benchmark model 1 or 2 (Table 1): true states s_0..s_T
    as (T + 1, d) with the x coordinates first, and observations y_1..y_T as (T, 1). The
    sine and cosine take the step the transition leaves; s_0 ~ N(0, I)."""
    rng = np.random.Generator(np.random.PCG64(seed + 2_000_003))
    d = 2 if kind == 1 else 4
    if kind == 1:
        Lv = np.linalg.cholesky(np.array([[1.0, 0.1], [0.1, 1.0]]))
    else:
        Sv = np.eye(4)
        Sv[2:, 2:] = [[1.0, 0.1], [0.1, 10.0]]
        Lv = np.linalg.cholesky(Sv)
    s = np.zeros((T + 1, d))
    s[0] = rng.standard_normal(d)
    ys = np.zeros((T, 1))
    for t in range(1, T + 1):
        v = Lv @ rng.standard_normal(d)
        p, u = s[t - 1], t - 1
        if kind == 1:
            x, z = p
            s[t] = [x + z / (1 + z * z) + v[0],
                    x + 0.5 * z + 25 * z / (1 + z * z) + 8 * np.cos(1.2 * u) + v[1]]
            y = np.arctan(s[t, 0]) + s[t, 1] ** 2 / 20
        else:
            x1, x2, z1, z2 = p
            z1n = z1 + z2 / (1 + z2 * z2) + v[2]
            s[t] = [0.5 * x1 + 8 * np.sin(u) + v[0], 0.4 * x1 + 0.5 * x2 + v[1], z1n,
                    z1n + 0.5 * z2 + 25 * z2 / (1 + z2 * z2) + 8 * np.cos(1.2 * u) + v[3]]
            y = (s[t, 0] + s[t, 1]) / (1 + s[t, 0] ** 2) + np.arctan(s[t, 2]) + s[t, 3] ** 2 / 20
        ys[t - 1, 0] = y + rng.standard_normal()
    return s, ys


def proposal_dims(spec, d1: int | None = None, components: int = 4, hidden: int = 256):
    """Sizes of the learned inner proposal for a model: inputs (x_{t-1}, x_t, z_{t-1}, y_t),
    hidden width, and the mixture head (logits, means, log standard deviations)."""
    d1 = spec.d1 if d1 is None else d1
    d2 = spec.d - d1
    return dict(din=2 * d1 + d2 + spec.dy, hidden=hidden, components=components,
                dout=components * (1 + 2 * d2), d2=d2)


def init_mlp_weights(din: int, hidden: int, dout: int, seed: int = 0, layers: int = 3):
    """Seeded initial weights of an MLP with `layers` hidden ReLU layers of width `hidden`:
    He-normal weights, zero biases; the head starts at a tenth of that scale. Returns a
    dict of float64 arrays W1, b1, ..., W{layers+1}, b{layers+1} (W_l is out x in)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = [din] + [hidden] * layers + [dout]
    w = {}
    for l in range(1, len(sizes)):
        fan_in = sizes[l - 1]
        scale = np.sqrt(2.0 / fan_in) * (0.1 if l == len(sizes) - 1 else 1.0)
        w[f"W{l}"] = rng.standard_normal((sizes[l], fan_in)) * scale
        w[f"b{l}"] = np.zeros(sizes[l])
    return w
