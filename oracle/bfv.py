"""RNS-BFV in the coefficient representation: keys, encryption, decryption, key switching,
rotations (plain and hoisted), plaintext products and modulus switching.

TEST INFRASTRUCTURE: the independent CPU oracle the GPU library is checked against.  Only
tests/, the smoke check and the CPU-baseline leg of bench.py may import it.  It shares no
code with the CUDA path; its products are the exact ring products of oracle/ring.c.

The paper works with BFV (Sec. 2.1: parameters t, Q, N; plaintext-ciphertext products and
ciphertext additions (MulPC, AddCC, Table I) and slot rotations (Sec. 3.2, Fig. 1b)) but
says nothing of how rotations are keyed or how the ciphertext modulus is split.  The
readings implemented here (each is also listed among the design readings):

  * ciphertexts are pairs (c0, c1) over Q = q_0 ... q_{L-1}, decrypting as
    m = round(t [c0 + c1 s]_Q / Q) mod t; fresh ones are c1 = a, c0 = -a s + e + Delta m
    with Delta = floor(Q/t) and m's coefficients in [0, t);
  * rotation by k slots applies X -> X^g with g = 5^(k mod N/2) mod 2N, then switches the
    key back from s(X^g) to s with hybrid key switching: digits of alpha primes, special
    modulus P = p_0 ... p_{K-1};
  * ModUp extends each digit with the fast (non-centred) base conversion
        y_p = sum_{i in digit} [d_i (Q_j/q_i)^-1]_{q_i} (Q_j/q_i)  mod p;
  * key j is (b_j, a_j) over Q u P with b_j = -a_j s + e_j + G_j s', G_j = P mod the primes
    of digit j and 0 mod every other prime;
  * ModDown is u'_i = (u_i - sum_k [u_{p_k} (P/p_k)^-1]_{p_k} (P/p_k)) P^-1 mod q_i;
  * the hoisted form runs ModUp once on c1 and applies X -> X^g to the extended digits;
    it is a different algorithm from the plain one (the lifts differ), so each has its
    own ciphertext bits and both decrypt to the same slots;
  * modulus switching drops q_{L-1} with rounding: c' = round(c / q_{L-1});
  * ciphertext multiplication (Sec. 2.1) is the exact textbook product: both ciphertexts'
    residues lifted to centred integers, the three tensor polynomials formed over Z[X]/(X^N+1)
    exactly (CRT over auxiliary primes of this module), each coefficient scaled to
    round(t d / Q) mod Q; relinearisation key-switches the third component with the
    switching key of s^2 (streams 6 << 48 | j and 7 << 48 | j).
"""
import numpy as np

from . import prng, ring
from .encoder import lift_centered
from .params import Params, is_prime, root_2n


class Ct:
    """A ciphertext (c0, c1), each an array [L][N] of residues in the coefficient domain."""

    def __init__(self, c0, c1):
        self.c0 = np.asarray(c0, dtype=np.uint64)
        self.c1 = np.asarray(c1, dtype=np.uint64)

    @property
    def level(self):
        return self.c0.shape[0]

    def stack(self):
        """[2][L][N] uint64, the layout the GPU library exports."""
        return np.stack([self.c0, self.c1])

    def copy(self):
        return Ct(self.c0.copy(), self.c1.copy())


# ---------------------------------------------------------------- ring helpers (per limb)

def to_rns(coeffs, moduli):
    """Signed integer coefficients -> [len(moduli)][N] residues."""
    return np.stack([ring.from_signed(coeffs, q) for q in moduli])


def rns_mul(a, b, prm: Params, moduli):
    return np.stack([ring.polymul(a[l], b[l], q, prm.psi[q]) for l, q in enumerate(moduli)])


def rns_add(a, b, moduli):
    return np.stack([ring.vadd(a[l], b[l], q) for l, q in enumerate(moduli)])


def rns_sub(a, b, moduli):
    return np.stack([ring.vsub(a[l], b[l], q) for l, q in enumerate(moduli)])


def automorphism_int(c, g):
    """X -> X^g on a signed integer coefficient vector: X^i -> +-X^(i g mod N)."""
    n = c.size
    out = np.zeros(n, dtype=np.int64)
    for i in range(n):
        e = i * g % (2 * n)
        if e < n:
            out[e] += c[i]
        else:
            out[e - n] -= c[i]
    return out


def automorphism(a, g, moduli):
    """X -> X^g on every limb of [len][N] residues (coefficient domain)."""
    n = a.shape[1]
    idx = np.arange(n, dtype=np.int64) * g % (2 * n)
    out = np.empty_like(a)
    for l, q in enumerate(moduli):
        pos = idx < n
        row = np.empty(n, dtype=np.uint64)
        row[idx[pos]] = a[l][pos]
        neg_src = a[l][~pos]
        row[idx[~pos] - n] = ring.vsub(np.zeros_like(neg_src), neg_src, q)
        out[l] = row
    return out


def galois_element(step: int, n: int) -> int:
    """Rotation by `step` slots (left, within each row of N/2 slots) <-> g = 5^step mod 2N."""
    return pow(5, step % (n // 2), 2 * n)


ROW_SWAP = "swap"


def galois_of(step, n):
    return 2 * n - 1 if step == ROW_SWAP else galois_element(step, n)


# ---------------------------------------------------------------- keys and encryption

def keygen_secret(prm: Params, seed: int):
    return prng.ternary(seed, prm.n)


def encrypt(prm: Params, s, m, seed: int) -> Ct:
    """Symmetric BFV encryption of the plaintext polynomial m (coefficients in [0, t))."""
    n, L = prm.n, prm.n_q
    a = prng.uniform(seed, prng.STREAM_CT_A, prm.q, n)
    e = prng.gaussian(seed, prng.STREAM_CT_E, n)
    delta = prm.delta()
    m = np.asarray(m, dtype=np.uint64)
    c0 = np.empty((L, n), dtype=np.uint64)
    for l, q in enumerate(prm.q):
        s_l = ring.from_signed(s, q)
        as_ = ring.polymul(a[l], s_l, q, prm.psi[q])
        x = ring.vsub(ring.from_signed(e, q), as_, q)
        c0[l] = ring.vmac_scalar(x, ring.vreduce(m, q), delta % q, q)
    return Ct(c0, a)


def crt(x, moduli):
    """[len][N] residues -> Python ints in [0, prod(moduli)) by the Chinese remainder theorem."""
    M = 1
    for q in moduli:
        M *= q
    out = [0] * x.shape[1]
    for l, q in enumerate(moduli):
        Mq = M // q
        c = Mq * pow(Mq % q, -1, q)
        col = x[l]
        for k in range(x.shape[1]):
            out[k] += int(col[k]) * c
    return [v % M for v in out], M


def phase(prm: Params, s, ct: Ct):
    """[c0 + c1 s]_Q as Python ints in [0, Q)."""
    moduli = prm.q[: ct.level]
    s_rns = to_rns(s, moduli)
    x = rns_add(ct.c0, rns_mul(ct.c1, s_rns, prm, moduli), moduli)
    return crt(x, moduli)


def decrypt(prm: Params, s, ct: Ct):
    """m = round(t x / Q) mod t, coefficient by coefficient (int64 array)."""
    x, Q = phase(prm, s, ct)
    t = prm.t
    return np.array([((t * v + (Q - 1) // 2) // Q) % t for v in x], dtype=np.int64)


def noise_bits(prm: Params, s, ct: Ct, m=None):
    """log2 of the infinity norm of [c0 + c1 s - Delta m]_Q, and the budget log2(Delta/2) - that."""
    x, Q = phase(prm, s, ct)
    if m is None:
        m = decrypt(prm, s, ct)
    delta = Q // prm.t
    worst = 0
    for v, mk in zip(x, m):
        r = (v - delta * int(mk)) % Q
        if r > Q // 2:
            r -= Q
        worst = max(worst, abs(r))
    from math import log2
    nb = log2(worst) if worst > 0 else 0.0
    return nb, log2(delta / 2) - nb


def switching_key(prm: Params, s, target_rns, seed: int, stream_a, stream_e):
    """Key for switching from the secret `target` (residues [L+K][N] over Q u P) back to s:
    [dnum][2][L+K][N], digit j = (b_j, a_j) with b_j = -a_j s + e_j + G_j target."""
    n, qp = prm.n, prm.qp
    P = prm.P
    out = np.empty((prm.dnum, 2, len(qp), n), dtype=np.uint64)
    for j in range(prm.dnum):
        a = prng.uniform(seed, stream_a(j), qp, n)
        e = prng.gaussian(seed, stream_e(j), n)
        digit = prm.digit(j)
        for l, q in enumerate(qp):
            as_ = ring.polymul(a[l], ring.from_signed(s, q), q, prm.psi[q])
            b = ring.vsub(ring.from_signed(e, q), as_, q)
            if l in digit:
                b = ring.vmac_scalar(b, target_rns[l], P % q, q)
            out[j, 0, l] = b
            out[j, 1, l] = a[l]
    return out


def galois_key(prm: Params, s, g: int, seed: int):
    """Key for switching from s(X^g) back to s: [dnum][2][L+K][N] (index 0 = b, 1 = a)."""
    target = to_rns(automorphism_int(s, g), prm.qp)
    return switching_key(prm, s, target, seed, lambda j: prng.stream_key_a(g, j),
                         lambda j: prng.stream_key_e(g, j))


def relin_key(prm: Params, s, seed: int):
    """Relinearisation key: switches s^2 (the secret of the third component of a product)
    back to s; streams (6 << 48 | j) and (7 << 48 | j)."""
    s_rns = to_rns(s, prm.qp)
    target = rns_mul(s_rns, s_rns, prm, prm.qp)
    return switching_key(prm, s, target, seed, lambda j: (6 << 48) | j, lambda j: (7 << 48) | j)


# ---------------------------------------------------------------- ciphertext multiplication

def _aux_primes(prm: Params, bits_needed: int):
    """The oracle's own NTT primes (61-bit, 1 mod 2N, none of Q u P) for exact integer products."""
    out, p = [], ((2 ** 61 - 2) // (2 * prm.n)) * (2 * prm.n) + 1
    while sum(x.bit_length() - 1 for x in out) < bits_needed:
        if is_prime(p) and p not in prm.qp:
            out.append(p)
        p -= 2 * prm.n
    return out


def centered_ints(x_rns, moduli):
    """Residues [len][N] -> Python ints in (-M/2, M/2] (M = prod moduli) by CRT."""
    vals, M = crt(x_rns, moduli)
    return [v - M if v > M // 2 else v for v in vals]


def multiply(prm: Params, a: Ct, b: Ct):
    """BFV multiplication before relinearisation (Sec. 2.1's homomorphic multiplication):
    d = round(t/Q (a0 + a1 s)(b0 + b1 s)) coefficient-wise, i.e. with a_k, b_k lifted to
    centred integers, d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1 over Z[X]/(X^N+1), then
    round(t d_k / Q) mod Q.  Returns (d0, d1, d2) as [L][N] residue arrays."""
    L = a.level
    moduli = prm.q[:L]
    Q = prm.Q(L)
    n, t = prm.n, prm.t
    # exact integer products through enough auxiliary primes: |d| <= 2 N (Q/2)^2
    bound_bits = 2 * Q.bit_length() + (n.bit_length()) + 3
    aux = _aux_primes(prm, bound_bits)
    psi = {p: root_2n(p, n) for p in aux}
    lifted = [centered_ints(x, moduli) for x in (a.c0, a.c1, b.c0, b.c1)]
    a0, a1, b0, b1 = [np.stack([np.array([c % p for c in v], dtype=np.uint64) for p in aux])
                      for v in lifted]
    prods = []
    for pairs in ([(a0, b0)], [(a0, b1), (a1, b0)], [(a1, b1)]):
        acc = np.zeros((len(aux), n), dtype=np.uint64)
        for x, y in pairs:
            for l, p in enumerate(aux):
                acc[l] = ring.vadd(acc[l], ring.polymul(x[l], y[l], p, psi[p]), p)
        prods.append(acc)
    out = []
    for d in prods:
        scaled = scale_round(centered_ints(d, aux), t, Q)
        out.append(np.stack([np.array([v % q for v in scaled], dtype=np.uint64) for q in moduli]))
    return out


def scale_round(ints, t, Q):
    """round(t v / Q) for integers v (Q odd, gcd(Q, t) = 1: never a tie)."""
    return [(2 * t * v + Q) // (2 * Q) for v in ints]


def relinearize(prm: Params, d, rlk) -> Ct:
    """(d0, d1, d2) -> (d0 + u0, d1 + u1) with (u0, u1) the key switch of d2 from s^2 to s."""
    moduli = prm.q[: d[0].shape[0]]
    u0, u1 = keyswitch(prm, d[2], rlk)
    return Ct(rns_add(d[0], u0, moduli), rns_add(d[1], u1, moduli))


# ---------------------------------------------------------------- key switching

def modup(prm: Params, d, j: int):
    """Digit j of d (coefficient domain over Q) extended to every prime of Q u P."""
    digit = prm.digit(j)
    Qj = 1
    for i in digit:
        Qj *= prm.q[i]
    # [d_i (Q_j/q_i)^-1]_{q_i}
    ys = []
    for i in digit:
        qi = prm.q[i]
        ys.append(ring.vmul_scalar(d[i], pow((Qj // qi) % qi, -1, qi), qi))
    out = np.empty((len(prm.qp), prm.n), dtype=np.uint64)
    for l, p in enumerate(prm.qp):
        if l in digit:
            out[l] = d[l]
            continue
        acc = np.zeros(prm.n, dtype=np.uint64)
        for y, i in zip(ys, digit):
            acc = ring.vmac_scalar(acc, ring.vreduce(y, p), (Qj // prm.q[i]) % p, p)
        out[l] = acc
    return out


def moddown(prm: Params, u):
    """[u]_{Q u P} -> round-down of u / P over Q (the floor form above)."""
    L, K = prm.n_q, prm.n_p
    P = prm.P
    ys = []
    for k in range(K):
        pk = prm.p[k]
        ys.append(ring.vmul_scalar(u[L + k], pow((P // pk) % pk, -1, pk), pk))
    out = np.empty((L, prm.n), dtype=np.uint64)
    for i in range(L):
        qi = prm.q[i]
        v = np.zeros(prm.n, dtype=np.uint64)
        for y, k in zip(ys, range(K)):
            v = ring.vmac_scalar(v, ring.vreduce(y, qi), (P // prm.p[k]) % qi, qi)
        out[i] = ring.vmul_scalar(ring.vsub(u[i], v, qi), pow(P % qi, -1, qi), qi)
    return out


def key_inner_product(prm: Params, digits, ksk):
    """(sum_j digits_j * b_j, sum_j digits_j * a_j) over Q u P."""
    qp = prm.qp
    u = [np.zeros((len(qp), prm.n), dtype=np.uint64) for _ in range(2)]
    for j, y in enumerate(digits):
        for k in range(2):
            u[k] = rns_add(u[k], rns_mul(y, ksk[j][k], prm, qp), qp)
    return u


def keyswitch(prm: Params, d, ksk):
    """Hybrid key switch of d (coefficient domain over Q): returns (u0', u1') over Q."""
    digits = [modup(prm, d, j) for j in range(prm.dnum)]
    u0, u1 = key_inner_product(prm, digits, ksk)
    return moddown(prm, u0), moddown(prm, u1)


def rotate(prm: Params, ct: Ct, step, keys) -> Ct:
    """Slot rotation by `step` (Sec. 3.2, Fig. 1b): automorphism, then key switch."""
    g = galois_of(step, prm.n)
    q = prm.q
    c0g = automorphism(ct.c0, g, q)
    c1g = automorphism(ct.c1, g, q)
    d0, d1 = keyswitch(prm, c1g, keys[g])
    return Ct(rns_add(c0g, d0, q), d1)


def rotate_hoisted(prm: Params, ct: Ct, steps, keys):
    """Several rotations of one ciphertext sharing one ModUp of c1."""
    digits = [modup(prm, ct.c1, j) for j in range(prm.dnum)]
    outs = []
    for step in steps:
        g = galois_of(step, prm.n)
        rd = [automorphism(y, g, prm.qp) for y in digits]
        u0, u1 = key_inner_product(prm, rd, keys[g])
        c0g = automorphism(ct.c0, g, prm.q)
        outs.append(Ct(rns_add(c0g, moddown(prm, u0), prm.q), moddown(prm, u1)))
    return outs


# ---------------------------------------------------------------- plaintext ops, add, rescale

def rotate_hoisted_ext(prm: Params, ct: Ct, steps, keys):
    """Hoisted rotations left in the extended basis Q u P: for each step the pair
    (u0 + P phi_g(c0), u1) over Q u P, whose ModDown is the rotation's key-switched result
    up to the rounding of the division by P.  Sums of plaintext multiples of these pairs are
    divided by P once (ModDown after the sum instead of once per rotation)."""
    digits = [modup(prm, ct.c1, j) for j in range(prm.dnum)]
    L = prm.n_q
    out = []
    for step in steps:
        g = galois_of(step, prm.n)
        rd = [automorphism(y, g, prm.qp) for y in digits]
        u0, u1 = key_inner_product(prm, rd, keys[g])
        c0g = automorphism(ct.c0, g, prm.q)
        for i, q in enumerate(prm.q):
            u0[i] = ring.vmac_scalar(u0[i], c0g[i], prm.P % q, q)
        out.append((u0, u1))
    return out


def scale_by_p_ext(prm: Params, ct: Ct):
    """(P c0, P c1) over Q u P (zero modulo the special primes): the unrotated ciphertext in
    the form rotate_hoisted_ext returns, ModDown giving back (c0, c1) exactly."""
    L, n = prm.n_q, prm.n
    pair = []
    for c in (ct.c0, ct.c1):
        e = np.zeros((len(prm.qp), n), dtype=np.uint64)
        for i, q in enumerate(prm.q):
            e[i] = ring.vmul_scalar(c[i], prm.P % q, q)
        pair.append(e)
    return pair


def pt_rns_ext(m, prm: Params):
    """Centred lift of a plaintext modulo every prime of Q u P ([L+K][N])."""
    return to_rns(lift_centered(m, prm), prm.qp)


def pt_rns(m, prm: Params, level=None):
    """Plaintext polynomial (coefficients mod t) -> centred lift mod each q ([L][N])."""
    c = lift_centered(m, prm)
    return to_rns(c, prm.q[: (prm.n_q if level is None else level)])


def mul_plain(prm: Params, ct: Ct, pt) -> Ct:
    """MulPC (Table I): (c0 p, c1 p) with p the centred lift of the plaintext."""
    moduli = prm.q[: ct.level]
    return Ct(rns_mul(ct.c0, pt, prm, moduli), rns_mul(ct.c1, pt, prm, moduli))


def mul_scalar(prm: Params, ct: Ct, w: int) -> Ct:
    """Product with the constant plaintext w (an integer weight)."""
    moduli = prm.q[: ct.level]
    return Ct(np.stack([ring.vmul_scalar(ct.c0[l], w % q, q) for l, q in enumerate(moduli)]),
              np.stack([ring.vmul_scalar(ct.c1[l], w % q, q) for l, q in enumerate(moduli)]))


def add(prm: Params, a: Ct, b: Ct) -> Ct:
    """AddCC (Table I)."""
    moduli = prm.q[: a.level]
    return Ct(rns_add(a.c0, b.c0, moduli), rns_add(a.c1, b.c1, moduli))


def rescale(prm: Params, ct: Ct) -> Ct:
    """Drop the last ciphertext prime with rounding: c' = round(c / q_last)."""
    L = ct.level
    ql = prm.q[L - 1]
    half = (ql - 1) // 2
    polys = []
    for c in (ct.c0, ct.c1):
        r = ring.vreduce(ring.vadd(c[L - 1], np.full(prm.n, half, dtype=np.uint64), ql), ql)
        rows = []
        for i in range(L - 1):
            qi = prm.q[i]
            ct_i = ring.vadd(c[i], np.full(prm.n, half % qi, dtype=np.uint64), qi)
            diff = ring.vsub(ct_i, ring.vreduce(r, qi), qi)
            rows.append(ring.vmul_scalar(diff, pow(ql % qi, -1, qi), qi))
        polys.append(np.stack(rows))
    return Ct(polys[0], polys[1])
