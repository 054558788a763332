"""Pins for the oracle's counter-based generator and samplers."""
import math
import os

import numpy as np

from oracle import prng

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vectors():
    rows = [l.split() for l in open(os.path.join(GOLD, "splitmix64_vectors.txt"))
            if l.strip() and not l.startswith("#")]
    for r in rows:
        seed, want = int(r[0]), [int(x) for x in r[1:]]
        got = [int(prng.mix64(np.uint64((seed + (i + 1) * prng.GAMMA) % 2 ** 64))) for i in range(5)]
        assert got == want


def test_draws_are_counter_addressable():
    a = prng.draws(42, 7, 0, 100)
    b = prng.draws(42, 7, 60, 40)
    assert (a[60:] == b).all()
    assert not (prng.draws(42, 8, 0, 100) == a).any()
    assert not (prng.draws(43, 7, 0, 100) == a).any()


def test_cdt_table_against_float_cdf():
    T = prng.cdt_table()
    assert len(T) == 20 and T[-1] == 1 << 63 and T == sorted(T)
    rho = [math.exp(-m * m / (2 * 3.2 * 3.2)) for m in range(20)]
    w = [rho[0]] + [2 * r for r in rho[1:]]
    z = sum(w)
    acc = 0.0
    for m in range(19):
        acc += w[m]
        assert abs(T[m] / 2 ** 63 - acc / z) < 1e-12


def test_gaussian_moments_and_support():
    e = prng.gaussian(5, 99, 400000)
    assert np.abs(e).max() <= 19
    assert abs(e.mean()) < 0.03
    assert abs(e.var() / (3.2 ** 2) - 1) < 0.02
    # discrete Gaussian: Pr(0) = 1/Z
    z = 1 + 2 * sum(math.exp(-m * m / 20.48) for m in range(1, 20))
    assert abs((e == 0).mean() - 1 / z) < 0.003


def test_ternary_and_uniform_distribution():
    s = prng.ternary(11, 300000)
    assert set(np.unique(s)) == {-1, 0, 1}
    for v in (-1, 0, 1):
        assert abs((s == v).mean() - 1 / 3) < 0.005
    q = 1125899906842177
    u = prng.uniform(3, 2, [q, 65537], 100000)
    assert u.shape == (2, 100000) and (u[0] < q).all() and (u[1] < 65537).all()
    assert abs(u[0].astype(np.float64).mean() / q - 0.5) < 0.005
