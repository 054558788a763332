"""Seeded synthetic inputs shaped like the paper's workloads (no method arithmetic here).

The paper evaluates on MNIST (1 x 28 x 28 grey images) and CIFAR-10 (3 x 32 x 32) with 8-bit
quantised weights and activations (Sec. 5).  Neither dataset nor trained weights are used:
these generators draw images with pixels uniform in [0, 255] and weights uniform in a small
signed integer range from numpy's PCG64 with a fixed seed, and stand in for them.
"""
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class LayerShape:
    I_c: int
    I_h: int
    I_w: int
    d: int
    stride: int
    pad: int
    r: int
    O_c: int

    def astuple(self):
        return (self.I_c, self.I_h, self.I_w, self.d, self.stride, self.pad, self.r, self.O_c)


# The single-image layer: 1 x 28 x 28 input, 5 x 5 stride-2 low-rank conv to r = 2 channels
# (pad 1 -> 13 x 13), 1 x 1 restore to 5 channels.
MNIST_LAYER = LayerShape(1, 28, 28, 5, 2, 1, 2, 5)


def image(seed, shape: LayerShape):
    return np.random.default_rng(seed).integers(0, 256, (shape.I_c, shape.I_h, shape.I_w), dtype=np.int64)


def images(seed, shape: LayerShape, count):
    rng = np.random.default_rng(seed)
    return [rng.integers(0, 256, (shape.I_c, shape.I_h, shape.I_w), dtype=np.int64) for _ in range(count)]


def weights(seed, shape: LayerShape, lo=-8, hi=8):
    rng = np.random.default_rng(seed + 1000)
    W1 = rng.integers(lo, hi + 1, (shape.r, shape.I_c, shape.d, shape.d), dtype=np.int64)
    W2 = rng.integers(lo, hi + 1, (shape.O_c, shape.r), dtype=np.int64)
    return W1, W2


def residues(seed, moduli, n, count=1):
    """count x [len(moduli)][n] uniform residues (the primitive sweep's random coefficients)."""
    rng = np.random.default_rng(seed)
    out = np.empty((count, len(moduli), n), dtype=np.uint64)
    for l, q in enumerate(moduli):
        out[:, l, :] = rng.integers(0, q, (count, n), dtype=np.uint64)
    return out


def slot_vector(seed, n, t):
    return np.random.default_rng(seed).integers(0, t, n, dtype=np.int64)
