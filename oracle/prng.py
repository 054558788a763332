"""Counter-based randomness for keys and encryptions, and the three samplers.

Test infrastructure (independent CPU oracle).  The paper draws its secret, masks and errors
from BFV (Sec. 2.1) without saying how; the reading shared with the GPU library is the
following, and each side implements it on its own from this definition.

Generator: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014).  Its output i from state s is
    mix64(s + (i + 1) * GAMMA)  (mod 2^64),
    mix64(z): z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
              z ^= z >> 31.
A (seed, stream) pair starts at s = mix64(seed XOR mix64(stream)), so every draw is a pure
function of (seed, stream, counter) and can be taken in any order or in parallel.

Streams: 1 secret key; 2 / 3 the uniform part a / error e of a fresh ciphertext;
(4 << 48 | g << 8 | j) / (5 << 48 | g << 8 | j) the a / e of digit j of the Galois key for
Galois element g.

Samplers (counter = index of the coefficient):
  ternary   u = draw(k); v = floor(3u / 2^64) in {0,1,2}  ->  {0, +1, -1}
  uniform   limb l, coefficient k: hi = draw(2(lN+k)), lo = draw(2(lN+k)+1);
            value = floor((hi 2^64 + lo) q / 2^128)
  Gaussian  discrete Gaussian with sigma = 3.2 cut at |e| <= 19, by cumulative table:
            u = draw(k); |e| = min{m : (u >> 1) < T[m]}; e = -|e| if u is odd.
"""
from decimal import Decimal, getcontext

import numpy as np

from . import ring

GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1
STREAM_SECRET = 1
STREAM_CT_A = 2
STREAM_CT_E = 3
SIGMA = Decimal("3.2")
TAIL = 19


def stream_key_a(g: int, j: int) -> int:
    return (4 << 48) | (g << 8) | j


def stream_key_e(g: int, j: int) -> int:
    return (5 << 48) | (g << 8) | j


def mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def stream_state(seed: int, stream: int) -> int:
    return int(mix64(np.uint64((seed ^ int(mix64(np.uint64(stream & M64)))) & M64)))


def draws(seed: int, stream: int, first: int, count: int) -> np.ndarray:
    """Outputs first .. first+count-1 of the (seed, stream) generator."""
    s0 = np.uint64(stream_state(seed, stream))
    idx = np.arange(first + 1, first + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = s0 + idx * np.uint64(GAMMA)
    return mix64(x)


def ternary(seed: int, n: int) -> np.ndarray:
    """Secret key coefficients in {-1, 0, 1} (int64)."""
    u = draws(seed, STREAM_SECRET, 0, n)
    v = np.array([(int(x) * 3) >> 64 for x in u], dtype=np.int64)
    return np.where(v == 2, -1, v).astype(np.int64)


def uniform(seed: int, stream: int, moduli, n: int) -> np.ndarray:
    """[len(moduli)][n] residues, limb l uniform mod moduli[l]."""
    out = np.empty((len(moduli), n), dtype=np.uint64)
    for l, q in enumerate(moduli):
        d = draws(seed, stream, 2 * l * n, 2 * n)
        out[l] = ring.uniform_mod(d[0::2], d[1::2], q)
    return out


def cdt_table():
    """T[m] = floor(2^63 * Pr(|e| <= m)) for m < 19, T[19] = 2^63 (table of the sampler)."""
    getcontext().prec = 80
    two_s2 = 2 * SIGMA * SIGMA
    rho = [(-(Decimal(m * m)) / two_s2).exp() for m in range(TAIL + 1)]
    weights = [rho[0]] + [2 * r for r in rho[1:]]
    z = sum(weights)
    out, acc = [], Decimal(0)
    for m in range(TAIL):
        acc += weights[m]
        out.append(int((acc / z * (Decimal(2) ** 63)).to_integral_value(rounding="ROUND_FLOOR")))
    out.append(1 << 63)
    return out


_CDT = None


def gaussian(seed: int, stream: int, n: int) -> np.ndarray:
    """Error coefficients (int64) from the discrete Gaussian sampler above."""
    global _CDT
    if _CDT is None:
        _CDT = np.array(cdt_table(), dtype=np.uint64)
    u = draws(seed, stream, 0, n)
    mag = np.searchsorted(_CDT, u >> np.uint64(1), side="right").astype(np.int64)
    neg = (u & np.uint64(1)).astype(bool)
    return np.where(neg, -mag, mag).astype(np.int64)
