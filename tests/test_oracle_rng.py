"""Pins of the oracle's random-number generator (CPU only).

* Philox4x32-10 words agree with cuRAND's host Philox4_32_10 generator, an
  independent implementation of the same published generator (Salmon et al.,
  SC'11). cuRAND's host generator lays counter (x, 0, s, 0) at output word
  4 (x 65536 + s); the key is the 64-bit seed.
* The Box-Muller normals have the standard normal law (KS test, moments) and
  the uniform mapping hits its exact end points.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

from oracle import oracle


def _curand():
    for name in ("libcurand.so", "libcurand.so.10"):
        for cand in (name, os.path.join("/usr/local/cuda/lib64", name)):
            try:
                return ctypes.CDLL(cand)
            except OSError:
                continue
    return None


@pytest.mark.parametrize("seed", [0, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 42])
def test_philox_matches_curand_host(oracle_lib, seed):
    cur = _curand()
    if cur is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert cur.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    assert cur.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    n = 4 * 65536 * 3
    words = np.zeros(n, np.uint32)
    assert cur.curandGenerate(gen, words.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    cur.curandDestroyGenerator(gen)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    rng = np.random.default_rng(seed & 0xFFFF)
    picks = [(0, 0), (0, 1), (1, 0), (2, 65535)] + [
        (int(x), int(s)) for x, s in zip(rng.integers(0, 3, 40), rng.integers(0, 65536, 40))]
    for x, s in picks:
        got = oracle.philox((x, 0, s, 0), key, oracle_lib)
        off = 4 * (x * 65536 + s)
        np.testing.assert_array_equal(got, words[off:off + 4], err_msg=f"ctr=({x},0,{s},0)")


def test_philox_all_counter_words_matter(oracle_lib):
    base = oracle.philox((1, 2, 3, 4), (5, 6), oracle_lib)
    for pos in range(4):
        c = [1, 2, 3, 4]
        c[pos] ^= 1
        assert not np.array_equal(oracle.philox(c, (5, 6), oracle_lib), base)
    for pos in range(2):
        k = [5, 6]
        k[pos] ^= 1
        assert not np.array_equal(oracle.philox((1, 2, 3, 4), k, oracle_lib), base)


def test_uniform_endpoints(oracle_lib):
    assert oracle_lib.ora_u01(0) == 2.0 ** -24
    assert oracle_lib.ora_u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert oracle_lib.ora_u01(0x80000000) == 0.5 + 2.0 ** -24


def test_box_muller_law(oracle_lib):
    from scipy import stats
    vals = []
    for i in range(400):
        vals.append(oracle.normals(7, 0, 3, i, oracle.P_PROP, 0, 501, oracle_lib))
    v = np.concatenate(vals)
    assert abs(v.mean()) < 5 / np.sqrt(v.size)
    assert abs(v.var() - 1) < 5 * np.sqrt(2 / v.size)
    assert stats.kstest(v, "norm").pvalue > 1e-4
    # pairs are independent: correlation of (n0, n1)
    n0, n1 = v[0:-1:2], v[1::2]
    assert abs(np.corrcoef(n0[: len(n1)], n1[: len(n0)])[0, 1]) < 5 / np.sqrt(len(n1))


def test_box_muller_formula_single(oracle_lib):
    wa, wb = 0x12345678, 0x9ABCDEF0
    a = ctypes.c_double(); b = ctypes.c_double()
    oracle_lib.ora_box_muller(wa, wb, ctypes.byref(a), ctypes.byref(b))
    ua = ((wa >> 9) + 0.5) * 2.0 ** -23
    ub = ((wb >> 9) + 0.5) * 2.0 ** -23
    r = np.sqrt(-2 * np.log(ua))
    assert a.value == pytest.approx(r * np.cos(2 * np.pi * ub), rel=1e-14, abs=1e-14)
    assert b.value == pytest.approx(r * np.sin(2 * np.pi * ub), rel=1e-14, abs=1e-14)
