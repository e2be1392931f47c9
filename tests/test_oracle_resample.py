"""Pins of the oracle's systematic resampling (CPU only).

On dyadic weights with a power-of-two n every quantity is exact in binary64,
so the integer rule must equal numpy's ``cumsum`` + ``searchsorted`` applied to
the systematic points (k + U) C / n. Invariants: offspring counts sum to n and
lie in {floor(n c_i / C), ceil(n c_i / C)}; zero weights are never chosen; the
output is non-decreasing. A hand-worked fixture checks small cases.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "resample_worked.json")


def _dyadic(rng, n, kind):
    if kind == "random":
        w = rng.integers(0, 1 << 20, n).astype(np.float64)
    elif kind == "spiky":
        w = np.zeros(n); w[rng.integers(0, n, 3)] = [1 << 30, 1 << 10, 1]
    elif kind == "zeros":
        w = rng.integers(0, 16, n).astype(np.float64); w[rng.random(n) < 0.7] = 0
        if w.sum() == 0:
            w[0] = 1
    else:  # ties
        w = np.full(n, 3.0)
    return w * 2.0 ** -7


def _reference(w, n_out, U):
    cum = np.cumsum(w)
    pts = (np.arange(n_out) + U) * cum[-1] / n_out
    return np.searchsorted(cum, pts, side="right")


@pytest.mark.parametrize("n", [1, 2, 32, 1024, 65536])
@pytest.mark.parametrize("kind", ["random", "spiky", "zeros", "ties"])
def test_global_matches_searchsorted_on_dyadic(oracle_lib, n, kind):
    rng = np.random.default_rng(n + len(kind))
    w = _dyadic(rng, n, kind)
    for u in [0, 1, 0x80000000, 0xFFFFFFFF, int(rng.integers(0, 2**32))]:
        got = oracle.sys_global(w, u, oracle_lib)
        np.testing.assert_array_equal(got, _reference(w, n, u / 2**32))


@pytest.mark.parametrize("n", [1, 2, 16, 128, 1024])
@pytest.mark.parametrize("kind", ["random", "spiky", "zeros", "ties"])
def test_local_matches_searchsorted_on_dyadic(oracle_lib, n, kind):
    rng = np.random.default_rng(n * 7 + len(kind))
    w = _dyadic(rng, n, kind)
    # keep the quantisation exact: the local rule keeps 31 - ceil(log2 n) bits
    w = np.floor(w / w.max() * 2.0 ** 12) + (w > 0)
    for u in [0, 65535, 0x80000000, 0xFFFFFFFF, int(rng.integers(0, 2**32))]:
        got = oracle.sys_local(w, n, u, oracle_lib)
        np.testing.assert_array_equal(got, _reference(w, n, (u >> 16) / 2**16))
        one = oracle.sys_local(w, 1, u, oracle_lib)
        np.testing.assert_array_equal(one, _reference(w, 1, u / 2**32))


@pytest.mark.parametrize("seed", range(5))
def test_counts_floor_ceil_and_zeros(oracle_lib, seed):
    rng = np.random.default_rng(seed)
    n = 1000 + seed * 37
    w = rng.exponential(size=n) ** 3
    w[rng.random(n) < 0.2] = 0
    idx = oracle.sys_global(w, int(rng.integers(0, 2**32)), oracle_lib)
    counts = np.bincount(idx, minlength=n)
    assert counts.sum() == n
    assert np.all(np.diff(idx) >= 0)
    assert np.all(counts[w == 0] == 0)
    e = int(np.floor(np.log2(w.max())))
    c = np.floor(np.ldexp(w, 62 - int(np.ceil(np.log2(n))) - e)).astype(object)
    C = sum(c)
    lo = [ci * n // C for ci in c]
    assert all(lo[i] <= counts[i] <= lo[i] + 1 for i in range(n))


def test_unbiased_offspring_counts(oracle_lib):
    """E[count_i] = n w_i / sum w over a uniform U (many u values)."""
    rng = np.random.default_rng(3)
    n = 50
    w = rng.random(n) ** 2
    acc = np.zeros(n)
    reps = 4000
    for u in rng.integers(0, 2**32, reps):
        acc += np.bincount(oracle.sys_global(w, int(u), oracle_lib), minlength=n)
    expected = n * w / w.sum()
    assert np.allclose(acc / reps, expected, atol=4 * 0.5 / np.sqrt(reps))


def test_worked_fixture(oracle_lib):
    cases = json.load(open(GOLD))["cases"]
    for c in cases:
        w = np.array(c["w"], float)
        if c["rule"] == "global":
            got = oracle.sys_global(w, c["u"], oracle_lib)
        elif c["rule"] == "local":
            got = oracle.sys_local(w, len(w), c["u"], oracle_lib)
        else:
            got = oracle.sys_local(w, 1, c["u"], oracle_lib)
        assert list(got) == c["idx"], c["_why"]


def test_all_zero_is_numeric_error(oracle_lib):
    with pytest.raises(RuntimeError):
        oracle.sys_global(np.zeros(8), 0, oracle_lib)
    with pytest.raises(RuntimeError):
        oracle.sys_local(np.zeros(8), 8, 0, oracle_lib)
