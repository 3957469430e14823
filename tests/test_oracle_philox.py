"""Pins of the oracle's DRM generator (Philox4x32-10 + Box-Muller)."""
import os

import numpy as np
import pytest

from oracle import philox

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        c = [int(x, 16) for x in r[:4]]
        k = [int(x, 16) for x in r[4:6]]
        want = [int(x, 16) for x in r[6:10]]
        got = philox.philox4x32_10(*[np.array([x], dtype=np.uint64) for x in c], *k)
        assert [int(g[0]) for g in got] == want


def test_uniform_ranges_exact():
    w = [np.array([0, 0xFFFFFFFF], dtype=np.uint64)] * 4
    u1, u2 = philox.uniforms(*w)
    assert u1[0] == 2.0 ** -53 and u1[1] == 1.0
    assert u2[0] == 0.0 and u2[1] == 1.0 - 2.0 ** -53


def test_ln_series_matches_log():
    rng = np.random.default_rng(0)
    u = np.concatenate([rng.random(20000), [1.0, 2.0 ** -53, 0.5, 1 - 2.0 ** -53, 0.7071067811865476]])
    u = u[u > 0]
    got = philox.ln_series(u)
    ref = np.log(u)
    err = np.abs(got - ref)
    assert np.all(err <= 4 * np.finfo(float).eps * np.maximum(np.abs(ref), 1e-300) + 1e-300)
    assert philox.ln_series(np.array([1.0]))[0] == 0.0


def test_sincos_matches_libm():
    rng = np.random.default_rng(1)
    u = np.concatenate([rng.random(20000), np.arange(8) / 8.0, [1 - 2.0 ** -53]])
    s, c = philox.sincos_2pi(u)
    assert np.max(np.abs(s - np.sin(2 * np.pi * u))) < 2e-15
    assert np.max(np.abs(c - np.cos(2 * np.pi * u))) < 2e-15
    # exact octant endpoints
    s0, c0 = philox.sincos_2pi(np.array([0.0, 0.25, 0.5, 0.75]))
    assert np.allclose(s0, [0, 1, 0, -1], atol=1e-16) and np.allclose(c0, [1, 0, -1, 0], atol=1e-16)


def test_gaussian_distribution():
    from scipy import stats
    z = philox.gaussian_matrix(2024, philox.KIND_X, 3, 1000, 200).ravel()
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # the two Box-Muller outputs of one counter are uncorrelated
    Z = philox.gaussian_matrix(7, philox.KIND_Y, 0, 100000, 2)
    assert abs(np.corrcoef(Z[:, 0], Z[:, 1])[0, 1]) < 5 / np.sqrt(100000)


def test_width_independent_and_streams_distinct():
    a = philox.gaussian_matrix(5, philox.KIND_X, 2, 7, 9)
    b = philox.gaussian_matrix(5, philox.KIND_X, 2, 7, 4)
    assert np.array_equal(a[:, :4], b)
    c = philox.gaussian_matrix(5, philox.KIND_Y, 2, 7, 9)
    d = philox.gaussian_matrix(5, philox.KIND_X, 3, 7, 9)
    e = philox.gaussian_matrix(6, philox.KIND_X, 2, 7, 9)
    for other in (c, d, e):
        assert not np.any(a == other)


@pytest.mark.parametrize("seed", [0, 1, 2 ** 63 + 12345])
def test_gaussian_deterministic(seed):
    a = philox.gaussian_matrix(seed, philox.KIND_XT, 11, 13, 6)
    b = philox.gaussian_matrix(seed, philox.KIND_XT, 11, 13, 6)
    assert np.array_equal(a, b) and np.all(np.isfinite(a))
