"""Pins for the oracle's slot encoder: evaluation semantics, slot-wise product/sum and the
rotation identities that DensePack relies on (Sec. 1, Sec. 3.2 Fig. 1b)."""
import numpy as np
import pytest

from oracle import bfv, encoder, params, ring


@pytest.fixture(scope="module")
def small():
    return params.Params(log_n=5, n_q=2, n_p=1, alpha=1)


def horner(poly, x, t):
    v = 0
    for c in reversed([int(c) for c in poly]):
        v = (v * x + c) % t
    return v


def test_encoding_evaluates_at_the_slot_roots(small):
    prm, t = small, small.t
    rng = np.random.default_rng(0)
    v = rng.integers(0, t, prm.n)
    m = encoder.encode(v, prm)
    e = encoder.slot_exponents(prm.n)
    for slot in range(prm.n):
        assert horner(m, pow(prm.zeta, int(e[slot]), t), t) == v[slot]


def test_round_trip_full_size():
    prm = params.cfg_small_layer()
    v = np.random.default_rng(1).integers(0, prm.t, prm.n)
    assert (encoder.decode(encoder.encode(v, prm), prm) == v).all()


def test_slotwise_product_and_sum(small):
    prm, t = small, small.t
    rng = np.random.default_rng(2)
    a, b = rng.integers(0, t, prm.n), rng.integers(0, t, prm.n)
    ma, mb = encoder.encode(a, prm), encoder.encode(b, prm)
    prod = ring.polymul_schoolbook(ma, mb, t)
    assert (encoder.decode(prod, prm) == (a * b) % t).all()
    assert (encoder.decode(ring.vadd(ma, mb, t), prm) == (a + b) % t).all()


def test_rotation_shifts_rows_left_and_swap(small):
    prm, t, n = small, small.t, small.n
    v = np.arange(n) + 100
    m = encoder.encode(v, prm)
    half = n // 2
    for k in (1, 3, half - 1):
        g = bfv.galois_element(k, n)
        mg = bfv.automorphism(m[None, :], g, [t])[0]
        got = encoder.decode(mg, prm)
        assert (got[:half] == np.roll(v[:half], -k)).all()
        assert (got[half:] == np.roll(v[half:], -k)).all()
    mg = bfv.automorphism(m[None, :], 2 * n - 1, [t])[0]
    got = encoder.decode(mg, prm)
    assert (got[:half] == v[half:]).all() and (got[half:] == v[:half]).all()


def test_constant_vector_is_constant_polynomial(small):
    prm = small
    for w in (0, 1, 7, -8):
        m = encoder.encode([w] * prm.n, prm)
        assert int(m[0]) == w % prm.t and not m[1:].any()
        assert encoder.lift_centered(m, prm)[0] == w
