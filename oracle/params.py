"""RNS-BFV parameters for the oracle: primes, roots of unity and CRT constants.

Test infrastructure (independent CPU oracle).

The paper fixes only (t, Q, N) for BFV (Sec. 2.1) and the security target; the readings used
here for the unstated parts:
  * the ciphertext primes q_0 > q_1 > ... are the largest primes below 2^q_bits with
    q = 1 (mod 2N); the special primes p_0 > p_1 > ... the largest below 2^p_bits with the
    same congruence (needed for negacyclic transforms of length N);
  * a key-switching digit holds `alpha` consecutive q's; dnum = ceil(L / alpha);
  * the batching root zeta mod t is x^((t-1)/2N) for the smallest quadratic non-residue x
    mod t (for t = 65537 this is 3^(65536/2N)); it fixes which polynomial encodes a slot
    vector.
"""
from dataclasses import dataclass, field
from typing import List


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin, exact for n < 3.3e24 with the first twelve prime bases."""
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for p in small:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def ntt_primes(bits: int, count: int, n: int) -> List[int]:
    """The `count` largest primes below 2^bits congruent to 1 mod 2n, descending."""
    m = 2 * n
    p = ((2 ** bits - 2) // m) * m + 1
    out = []
    while len(out) < count:
        if p < 2:
            raise ValueError("not enough primes")
        if is_prime(p):
            out.append(p)
        p -= m
    return out


def nonresidue(q: int) -> int:
    x = 2
    while pow(x, (q - 1) // 2, q) != q - 1:
        x += 1
    return x


def root_2n(q: int, n: int) -> int:
    """A primitive 2n-th root of unity mod q (requires 2n | q-1)."""
    assert (q - 1) % (2 * n) == 0
    psi = pow(nonresidue(q), (q - 1) // (2 * n), q)
    assert pow(psi, n, q) == q - 1
    return psi


def prod(xs):
    r = 1
    for x in xs:
        r *= x
    return r


@dataclass
class Params:
    log_n: int
    n_q: int
    n_p: int
    alpha: int
    t: int = 65537
    q_bits: int = 50
    p_bits: int = 60
    n: int = field(init=False)
    q: List[int] = field(init=False)
    p: List[int] = field(init=False)

    def __post_init__(self):
        self.n = 1 << self.log_n
        self.q = ntt_primes(self.q_bits, self.n_q, self.n)
        self.p = ntt_primes(self.p_bits, self.n_p, self.n)
        self.qp = self.q + self.p
        self.dnum = -(-self.n_q // self.alpha)
        self.psi = {m: root_2n(m, self.n) for m in self.qp}
        self.batching = (self.t - 1) % (2 * self.n) == 0
        self.zeta = root_2n(self.t, self.n) if self.batching else None

    # ---- moduli products ----
    def Q(self, level=None):
        return prod(self.q[: (self.n_q if level is None else level)])

    @property
    def P(self):
        return prod(self.p)

    def delta(self, level=None):
        """Delta = floor(Q / t), the BFV scaling factor (Sec. 2.1)."""
        return self.Q(level) // self.t

    def digit(self, j):
        """Indices of the ciphertext primes in key-switching digit j."""
        return list(range(j * self.alpha, min((j + 1) * self.alpha, self.n_q)))


# Parameter sets used across the tests and the benchmark.
def cfg_small_layer():
    """5x5 stride-2 layer ring: N = 8192, three 50-bit q's, one 60-bit special prime."""
    return Params(log_n=13, n_q=3, n_p=1, alpha=1)


def cfg_n14():
    """The three-layer network's ring: N = 2^14, six 50-bit q's, two 60-bit p's, digits of 2."""
    return Params(log_n=14, n_q=6, n_p=2, alpha=2)


def cfg_n15():
    """The benchmark layer's ring: N = 2^15, twelve 50-bit q's, three 60-bit p's, digits of 3."""
    return Params(log_n=15, n_q=12, n_p=3, alpha=3)
