"""Slot (batching) encoder for BFV plaintexts.

Test infrastructure (independent CPU oracle).

The paper packs a vector of messages into the slots of one ciphertext (Sec. 1, 'a vector of
slots'; Sec. 3.2 DensePack/ConvPack) and relies on slot-wise products and sums and on slot
rotations.  With t = 1 (mod 2N) the plaintext ring Z_t[X]/(X^N+1) splits into N slots, the
values of m(X) at the primitive 2N-th roots zeta^e (e odd).  The reading used here:
  slot j        (row 0, j < N/2) <-> m(zeta^(5^j mod 2N))
  slot N/2 + j  (row 1)          <-> m(zeta^(-5^j mod 2N))
so that X -> X^(5^k) shifts each row left by k slots and X -> X^(2N-1) swaps the rows.
"""
import numpy as np

from . import ring


def slot_exponents(n: int) -> np.ndarray:
    """e[slot], the odd exponent of zeta that slot `slot` evaluates m at."""
    half = n // 2
    e = np.empty(n, dtype=np.int64)
    x = 1
    for j in range(half):
        e[j] = x
        e[half + j] = (2 * n - x) % (2 * n)
        x = x * 5 % (2 * n)
    return e


def encode(values, prm) -> np.ndarray:
    """Slot values (ints, taken mod t) -> coefficients of m(X) in [0, t).

    m is the unique polynomial of degree < N with m(zeta^e[slot]) = values[slot]; it is
    found by interpolation at the odd powers of zeta (ring.neg_interp)."""
    n, t = prm.n, prm.t
    v = np.asarray([int(x) % t for x in values], dtype=np.uint64)
    assert v.size == n
    w = np.empty(n, dtype=np.uint64)
    w[(slot_exponents(n) - 1) // 2] = v
    return ring.neg_interp(w, t, prm.zeta)


def decode(m, prm) -> np.ndarray:
    """Coefficients of m(X) mod t -> slot values in [0, t) (int64)."""
    n, t = prm.n, prm.t
    w = ring.neg_eval(np.asarray(m, dtype=np.uint64), t, prm.zeta)
    return w[(slot_exponents(n) - 1) // 2].astype(np.int64)


def lift_centered(m, prm) -> np.ndarray:
    """Plaintext coefficients in [0, t) -> signed integers in (-t/2, t/2]."""
    m = np.asarray(m, dtype=np.int64)
    return np.where(m > (prm.t - 1) // 2, m - prm.t, m).astype(np.int64)


def plaintext_rns(values, prm, moduli) -> np.ndarray:
    """Slot values -> the centred lift of their encoding, reduced mod each modulus ([len][N])."""
    c = lift_centered(encode(values, prm), prm)
    return np.stack([ring.from_signed(c, q) for q in moduli])
