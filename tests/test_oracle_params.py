"""Pins for the oracle's parameter generation: primes, roots and the paper's plaintext moduli."""
import os

import pytest

from oracle import params

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def fermat_witness_composite(n):
    """True when a Fermat witness among small bases proves n composite."""
    return any(pow(a, n - 1, n) != 1 for a in (2, 3, 5, 7, 11))


def trial_factor(n, limit=20000):
    for p in range(2, limit):
        if n % p == 0 and n != p:
            return p
    return None


def test_miller_rabin_on_known_values():
    assert params.is_prime(2) and params.is_prime(3) and not params.is_prime(1)
    assert params.is_prime(65537) and params.is_prime((1 << 61) - 1)
    assert not params.is_prime(3215031751)          # strong pseudoprime to bases 2, 3, 5, 7
    assert not params.is_prime(561) and not params.is_prime((1 << 61) - 3)
    assert not params.is_prime(4294967297)          # 641 * 6700417


@pytest.mark.parametrize("log_n,bits,count", [(13, 50, 3), (13, 60, 1), (15, 50, 12), (15, 60, 3),
                                              (16, 50, 24), (16, 60, 6)])
def test_ntt_primes_are_the_largest_ones(log_n, bits, count):
    n = 1 << log_n
    ps = params.ntt_primes(bits, count, n)
    assert ps == sorted(ps, reverse=True) and len(set(ps)) == count
    for p in ps:
        assert p < 2 ** bits and p % (2 * n) == 1
        assert not fermat_witness_composite(p) and trial_factor(p) is None
    # every skipped candidate between 2^bits and the last prime is composite
    cand = ((2 ** bits - 2) // (2 * n)) * (2 * n) + 1
    while cand > ps[-1]:
        if cand not in ps:
            assert fermat_witness_composite(cand) or trial_factor(cand) is not None
        cand -= 2 * n


def test_roots_are_primitive_2n_th():
    prm = params.cfg_small_layer()
    for q in prm.qp:
        psi = prm.psi[q]
        assert pow(psi, prm.n, q) == q - 1 and pow(psi, 2 * prm.n, q) == 1
    # for t = 65537 the smallest non-residue is 3, so zeta = 3^(65536 / 2N)
    assert prm.zeta == pow(3, 65536 // (2 * prm.n), 65537) == 81


def test_delta_and_moduli_products():
    prm = params.cfg_small_layer()
    Q = prm.q[0] * prm.q[1] * prm.q[2]
    assert prm.Q() == Q and prm.delta() == Q // 65537 and Q % 65537 != 0
    assert prm.dnum == 3 and prm.digit(2) == [2]
    p15 = params.cfg_n15()
    assert p15.dnum == 4 and p15.digit(3) == [9, 10, 11]


def test_paper_plaintext_moduli_support_slots():
    """Every t of the paper's settings is prime and 1 mod 2N: slot packing applies."""
    rows = [l.split() for l in open(os.path.join(GOLD, "paper_plaintext_moduli.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 6
    for r in rows:
        n, t = int(r[0]), int(r[1])
        assert params.is_prime(t) and t % (2 * n) == 1
