"""The index map the kernels use for the automorphism in the NTT domain, restated here and
checked against the oracle (CPU, no GPU).

The library's forward NTT leaves position p holding a(psi^(2 brv(p) + 1)).  X -> X^g then
moves the value at odd power e to e g mod 2N, so the rotated polynomial's position p reads the
input's position perm_g(p) = brv(((2 brv(p) + 1) g mod 2N - 1) / 2) (perm_of / perm_src in the
CUDA sources).  The fused tap kernel and the automorphism kernel (which stages 2048-residue
chunks in shared memory) rely on perm_g mapping every aligned block of 2^k positions onto one
aligned block of 2^k positions.

Also restated: the forward NTT row pass's reordered twiddle table (ntt.cu k_row_table) and the
index the row pass reads it at."""
import numpy as np
import pytest

from oracle import bfv, params, ring


def brv(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


def perm(p, g, log_n):
    n2 = 2 << log_n
    e = (2 * brv(p, log_n) + 1) * g % n2
    return brv((e - 1) // 2, log_n)


def galois_elements(log_n):
    n = 1 << log_n
    return [pow(5, k, 2 * n) for k in (1, 2, 3, 7, n // 2 - 1)] + [2 * n - 1]


@pytest.mark.parametrize("log_n", [4, 6, 9])
def test_perm_matches_the_oracle_automorphism_in_the_ntt_domain(log_n):
    prm = params.Params(log_n=log_n, n_q=1, n_p=1, alpha=1)
    q, n = prm.q[0], prm.n
    rng = np.random.default_rng(log_n)
    a = rng.integers(0, q, n, dtype=np.uint64)
    order = [brv(p, log_n) for p in range(n)]
    x = ring.neg_eval(a, q, prm.psi[q])[order]           # NTT order: position p
    for g in galois_elements(log_n):
        b = bfv.automorphism(a[None, :], g, [q])[0]
        y = ring.neg_eval(b, q, prm.psi[q])[order]
        assert (y == x[[perm(p, g, log_n) for p in range(n)]]).all(), g


@pytest.mark.parametrize("log_n", [4, 7, 10])
def test_perm_maps_aligned_blocks_onto_aligned_blocks(log_n):
    n = 1 << log_n
    for g in galois_elements(log_n):
        pm = [perm(p, g, log_n) for p in range(n)]
        assert sorted(pm) == list(range(n))                  # a permutation
        for k in range(log_n + 1):
            size = 1 << k
            for a0 in range(0, n, size):
                blocks = {pm[p] // size for p in range(a0, a0 + size)}
                assert len(blocks) == 1, (g, k, a0)


def row_table(log_n, s1, kmax):
    """Position in the reordered table of every standard entry e >= 2^s1: stage s, offset
    o = base 2^ee + j with ee = (s - s1) mod kmax, moved to 2^s + j 2^(s - ee) + base."""
    n = 1 << log_n
    dst = list(range(n))
    for e in range(1 << s1, n):
        s = e.bit_length() - 1
        o, ee = e - (1 << s), (s - s1) % kmax
        b, j = o >> ee, o & ((1 << ee) - 1)
        dst[e] = (1 << s) + (j << (s - ee)) + b
    return dst


@pytest.mark.parametrize("log_n,s1,kmax", [(6, 3, 3), (9, 4, 3), (13, 6, 3), (15, 7, 3), (15, 6, 3),
                                           (15, 7, 2), (16, 8, 3), (16, 5, 2)])
def test_row_pass_reads_the_reordered_twiddles_it_needs(log_n, s1, kmax):
    """The table is a permutation inside every stage, and the forward row pass's index for
    stage s = s1 + e0 + ee of round (e0, K), group base and pair index j,
    2^s + j 2^(s1 + e0) + base, lands on the standard entry 2^s + base 2^ee + j."""
    n = 1 << log_n
    dst = row_table(log_n, s1, kmax)
    assert sorted(dst) == list(range(n))
    for s in range(s1, log_n):
        assert {dst[e] >> s for e in range(1 << s, 2 << s)} == {1}   # stays in its stage
    table = [None] * n
    for e in range(n):
        table[dst[e]] = e                                             # entry e's new position
    s2 = log_n - s1
    for e0 in range(0, s2, kmax):
        K = min(kmax, s2 - e0)
        for ee in range(K):
            s = s1 + e0 + ee
            for base in range(1 << (s1 + e0)):
                for j in range(1 << ee):
                    got = table[(1 << s) + (j << (s1 + e0)) + base]
                    assert got == (1 << s) + (base << ee) + j, (s, base, j)
