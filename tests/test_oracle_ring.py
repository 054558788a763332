"""Pins for the oracle's ring arithmetic (oracle/ring.c) against closed forms and Python's
own integer arithmetic.  CPU only."""
import numpy as np
import pytest

from oracle import params, ring

Q50 = params.ntt_primes(50, 2, 8192)
P60 = params.ntt_primes(60, 1, 8192)


def kronecker_negacyclic(a, b, q):
    """a*b mod (X^n+1, q) through one big-integer product (Kronecker substitution)."""
    n = len(a)
    k = 2 * 64 + 16
    A = sum(int(x) << (k * i) for i, x in enumerate(a))
    B = sum(int(x) << (k * i) for i, x in enumerate(b))
    C = A * B
    mask = (1 << k) - 1
    full = [(C >> (k * i)) & mask for i in range(2 * n)]
    return [(full[i] - full[i + n]) % q for i in range(n)]


@pytest.mark.parametrize("n", [1, 2, 8, 32, 64])
@pytest.mark.parametrize("q", Q50 + P60)
def test_schoolbook_matches_kronecker(n, q):
    rng = np.random.default_rng(n)
    a = rng.integers(0, q, n, dtype=np.uint64)
    b = rng.integers(0, q, n, dtype=np.uint64)
    assert list(ring.polymul_schoolbook(a, b, q)) == kronecker_negacyclic(a, b, q)


def test_monomials_wrap_with_sign():
    n, q = 16, Q50[0]
    for i in range(n):
        for j in range(n):
            a = np.zeros(n, np.uint64); a[i] = 1
            b = np.zeros(n, np.uint64); b[j] = 1
            c = ring.polymul_schoolbook(a, b, q)
            want = np.zeros(n, np.uint64)
            want[(i + j) % n] = 1 if i + j < n else q - 1
            assert (c == want).all()


@pytest.mark.parametrize("n", [2, 4, 16, 128, 1024])
def test_fast_product_equals_schoolbook(n):
    rng = np.random.default_rng(7 + n)
    for q in (Q50[0], P60[0]):
        psi = params.root_2n(q, 8192) if n == 8192 else params.root_2n(q, n)
        a = rng.integers(0, q, n, dtype=np.uint64)
        b = rng.integers(0, q, n, dtype=np.uint64)
        assert (ring.polymul(a, b, q, psi) == ring.polymul_schoolbook(a, b, q)).all()


def test_fast_product_full_size_sampled_coefficients():
    n = 8192
    rng = np.random.default_rng(3)
    for q in (Q50[1], P60[0]):
        psi = params.root_2n(q, n)
        a = rng.integers(0, q, n, dtype=np.uint64)
        b = rng.integers(0, q, n, dtype=np.uint64)
        c = ring.polymul(a, b, q, psi)
        for k in [0, 1, 2, 4095, 4096, 8190, 8191] + list(rng.integers(0, n, 5)):
            assert int(c[k]) == ring.polymul_coeff(a, b, q, int(k))


def test_evaluation_is_value_at_odd_powers():
    n, q = 64, Q50[0]
    psi = params.root_2n(q, n)
    rng = np.random.default_rng(1)
    a = rng.integers(0, q, n, dtype=np.uint64)
    ev = ring.neg_eval(a, q, psi)
    for k in range(n):
        x = pow(psi, 2 * k + 1, q)
        val = 0
        for coef in reversed([int(c) for c in a]):      # Horner
            val = (val * x + coef) % q
        assert int(ev[k]) == val
    assert (ring.neg_interp(ev, q, psi) == a).all()


def test_product_is_pointwise_at_roots_of_x_n_plus_1():
    n, q = 256, P60[0]
    psi = params.root_2n(q, n)
    rng = np.random.default_rng(2)
    a = rng.integers(0, q, n, dtype=np.uint64)
    b = rng.integers(0, q, n, dtype=np.uint64)
    c = ring.polymul(a, b, q, psi)
    for k in (0, 1, 77, 255):
        x = pow(psi, 2 * k + 1, q)
        ev = lambda p: sum(int(cf) * pow(x, i, q) for i, cf in enumerate(p)) % q
        assert ev(c) == ev(a) * ev(b) % q


def test_elementwise_ops_against_python_ints():
    rng = np.random.default_rng(5)
    for q in (Q50[0], P60[0], 65537):
        a = rng.integers(0, q, 1000, dtype=np.uint64)
        b = rng.integers(0, q, 1000, dtype=np.uint64)
        s = int(rng.integers(0, q))
        A, B = [int(x) for x in a], [int(x) for x in b]
        assert [int(x) for x in ring.vadd(a, b, q)] == [(x + y) % q for x, y in zip(A, B)]
        assert [int(x) for x in ring.vsub(a, b, q)] == [(x - y) % q for x, y in zip(A, B)]
        assert [int(x) for x in ring.vmul(a, b, q)] == [(x * y) % q for x, y in zip(A, B)]
        assert [int(x) for x in ring.vmul_scalar(a, s, q)] == [(x * s) % q for x in A]
        assert [int(x) for x in ring.vmac_scalar(b, a, s, q)] == [(y + x * s) % q for x, y in zip(A, B)]
    sig = np.array([-(2 ** 63), -5, -1, 0, 1, 2 ** 63 - 1], dtype=np.int64)
    q = Q50[0]
    assert [int(x) for x in ring.from_signed(sig, q)] == [int(v) % q for v in sig]


def test_uniform_map_against_python_ints():
    rng = np.random.default_rng(9)
    hi = rng.integers(0, 2 ** 63, 500, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    lo = rng.integers(0, 2 ** 63, 500, dtype=np.uint64)
    for q in (Q50[0], P60[0]):
        got = ring.uniform_mod(hi, lo, q)
        want = [((int(h) << 64 | int(l)) * q) >> 128 for h, l in zip(hi, lo)]
        assert [int(x) for x in got] == want
