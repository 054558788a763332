"""Deeper image network over several ciphertexts per tensor (multi-ciphertext DensePack).

TEST INFRASTRUCTURE (independent CPU oracle).

Network (the paper's factorized convolutions in a deeper stack, Sec. 4.1 Eq. 2 and Sec. 4.2;
the square activation of Sec. 3; a fully connected classifier): input C0 x H x W, then for
each convolution layer a d x d stride-1 convolution to O_c channels -- factorized as a d x d
low-rank convolution W1 (r filters) and a 1 x 1 restore W2 (O_c x r), or unfactorized (W1 with
O_c filters, no W2) -- followed by x^2; then a global sum pooling over H x W and a fully
connected layer to the classes.

Packing (the readings, each also listed among the design readings):
  * tensor layout: channel c of an H x W map occupies block c mod g of ciphertext c // g, block
    size Bk = next_pow2(H W), g = (N/2) / Bk blocks per row 0; pixel (h, w) at offset h W + w;
  * layer, W1 under DensePack: for every input ciphertext the d^2 filter taps are rotations by
    delta = (i - pad) W + (j - pad) (hoisted, left in Q u P as in ffconv.py's dp_shift_ext);
    for every low-rank channel c' the tap products of all input ciphertexts are summed in Q u P
    and divided by P once; the sum over the g blocks, y1[c'] = sum_{u<g} rot(acc, u Bk), then
    leaves the channel's output replicated in every block -- its g - 1 rotations are hoisted
    from one ModUp and summed in Q u P with one ModDown (cheaper than log2 g sequential
    rotate-and-sum steps, each with its own ModUp and ModDown);
  * W2 (and the unfactorized packing) without rotations: output ciphertext G is
    sum_c' y1[c'] * P[G][c'] with P[G][c'] holding W2[G g + j][c'] on the pixels of block j
    (a block-wise ConvPack product; the unfactorized layer uses W2 = identity, O_c = r);
  * pooling and classifier in one linear map: logit_j = sum_c F[j][c] sum_pixels a[c, pixel],
    i.e. a fully connected layer whose features are all C H W activations (feature (c, pixel)
    at slot (c mod g) Bk + pixel of ciphertext c // g, weight F[j][c]); evaluated with the
    diagonal schedule of network.py, the taps of every input ciphertext summed in Q u P before
    one ModDown, period N/2; output j at slots p = j mod M.  (The in-block rotate-and-sum
    he_pool is kept as a step of its own.)
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import bfv
from .encoder import encode
from .ffconv import OpCount
from .network import next_pow2


@dataclass
class ConvSpec:
    O_c: int
    r: Optional[int]          # None: unfactorized (W1 has O_c filters, no restore)
    d: int = 3
    pad: int = 1


@dataclass
class DeepShape:
    C0: int
    H: int
    W: int
    convs: List[ConvSpec] = field(default_factory=list)
    n_cls: int = 10

    @property
    def Bk(self):
        return next_pow2(self.H * self.W)


def per_ct(shape: DeepShape, n: int) -> int:
    g = (n // 2) // shape.Bk
    if g < 1:
        raise ValueError("one channel map must fit in a row")
    return g


def n_cts(channels: int, g: int) -> int:
    return -(-channels // g)


def pack_tensor(x, shape: DeepShape, n: int):
    """Slot vectors of a C x H x W tensor in the layout above."""
    x = np.asarray(x)
    g = per_ct(shape, n)
    out = [np.zeros(n, dtype=np.int64) for _ in range(n_cts(x.shape[0], g))]
    hw = shape.H * shape.W
    for c in range(x.shape[0]):
        out[c // g][(c % g) * shape.Bk:(c % g) * shape.Bk + hw] = x[c].reshape(-1)
    return out


def conv_same(x, Wt, d, pad, t):
    """Stride-1 cross-correlation with zero padding, mod t: [C_in][H][W] x [C_out][C_in][d][d]
    (int64 throughout: operands below t < 2^17, sums of at most 2^20 products fit)."""
    x = np.asarray(x, dtype=np.int64) % t
    Wt = np.asarray(Wt, dtype=np.int64) % t
    C, H, Wd = x.shape
    xp = np.zeros((C, H + 2 * pad, Wd + 2 * pad), dtype=np.int64)
    xp[:, pad:pad + H, pad:pad + Wd] = x
    Ho, Wo = H + 2 * pad - d + 1, Wd + 2 * pad - d + 1
    out = np.zeros((Wt.shape[0], Ho, Wo), dtype=np.int64)
    for i in range(d):
        for j in range(d):
            patch = xp[:, i:i + Ho, j:j + Wo]                      # C x Ho x Wo
            out = (out + np.tensordot(Wt[:, :, i, j], patch, axes=([1], [0]))) % t
    return out


def plain_deep(x, weights, shape: DeepShape, t: int):
    """Plain network with every value reduced mod t (exact: the result is compared mod t):
    (per-layer activations, logits)."""
    h = np.asarray(x, dtype=np.int64) % t
    acts = []
    for spec, (W1, W2) in zip(shape.convs, weights["convs"]):
        y = conv_same(h, W1, spec.d, spec.pad, t)
        if W2 is not None:
            y = np.tensordot(np.asarray(W2, dtype=np.int64) % t, y, axes=([1], [0])) % t
        h = (y * y) % t
        acts.append(h)
    pooled = h.reshape(h.shape[0], -1).sum(axis=1) % t
    logits = ((np.asarray(weights["fc"], dtype=np.int64) % t) @ pooled) % t
    return acts, logits


# ------------------------------------------------------------------ encrypted steps

def tap_offsets(spec: ConvSpec, shape: DeepShape):
    return [(i, j, (i - spec.pad) * shape.W + (j - spec.pad))
            for i in range(spec.d) for j in range(spec.d)]


def tap_slots(W1, spec: ConvSpec, shape: DeepShape, n: int, c: int, g_in: int, i: int, j: int,
              C_in: int):
    """Plaintext of tap (i, j) for low-rank channel c against input ciphertext g_in."""
    g = per_ct(shape, n)
    v = np.zeros(n, dtype=np.int64)
    for ci in range(g_in * g, min(C_in, (g_in + 1) * g)):
        base = (ci % g) * shape.Bk
        w = int(W1[c][ci][i][j])
        if w == 0:
            continue
        for oh in range(shape.H):
            h = oh + i - spec.pad
            if not 0 <= h < shape.H:
                continue
            for ow in range(shape.W):
                wi = ow + j - spec.pad
                if 0 <= wi < shape.W:
                    v[base + oh * shape.W + ow] = w
    return v


def restore_slots(W2, shape: DeepShape, n: int, G: int, c: int, O_c: int):
    """Block-wise plaintext P[G][c]: W2[G g + j][c] on the pixels of block j."""
    g = per_ct(shape, n)
    v = np.zeros(n, dtype=np.int64)
    hw = shape.H * shape.W
    for j in range(g):
        o = G * g + j
        if o < O_c:
            v[j * shape.Bk: j * shape.Bk + hw] = int(W2[o][c])
    return v


def fold_steps(shape: DeepShape, n: int):
    """Rotations of the block sum: u Bk for u = 1 .. g - 1."""
    g = per_ct(shape, n)
    return [u * shape.Bk for u in range(1, g)]


def he_conv(prm, cts_in, W1, W2, spec: ConvSpec, C_in: int, shape: DeepShape, keys,
            ops: OpCount = None):
    """One encrypted convolution layer (factorized, or unfactorized when W2 is None)."""
    ops = ops if ops is not None else OpCount()
    n = prm.n
    g = per_ct(shape, n)
    taps = tap_offsets(spec, shape)
    steps = [dl for (_, _, dl) in taps if dl != 0]
    by_ct = []
    for ct in cts_in:
        rotated = bfv.rotate_hoisted_ext(prm, ct, steps, keys)
        pairs = dict(zip(steps, rotated))
        pairs[0] = bfv.scale_by_p_ext(prm, ct)
        by_ct.append(pairs)
        ops.rot += len(steps)
    r = len(W1)
    y1 = []
    for c in range(r):
        acc = None
        for gi, pairs in enumerate(by_ct):
            for (i, j, dl) in taps:
                pt = bfv.pt_rns_ext(encode(tap_slots(W1, spec, shape, n, c, gi, i, j, C_in), prm),
                                    prm)
                term = [bfv.rns_mul(pairs[dl][h], pt, prm, prm.qp) for h in range(2)]
                ops.mulpc += 1
                if acc is None:
                    acc = term
                else:
                    acc = [bfv.rns_add(acc[h], term[h], prm.qp) for h in range(2)]
                    ops.addcc += 1
        ct = bfv.Ct(bfv.moddown(prm, acc[0]), bfv.moddown(prm, acc[1]))
        fs = fold_steps(shape, n)
        if fs:
            pairs = [bfv.scale_by_p_ext(prm, ct)] + bfv.rotate_hoisted_ext(prm, ct, fs, keys)
            tot = pairs[0]
            for pr in pairs[1:]:
                tot = [bfv.rns_add(tot[h], pr[h], prm.qp) for h in range(2)]
                ops.addcc += 1
            ops.rot += len(fs)
            ct = bfv.Ct(bfv.moddown(prm, tot[0]), bfv.moddown(prm, tot[1]))
        y1.append(ct)
    O_c = spec.O_c
    W2m = np.eye(O_c, dtype=np.int64) if W2 is None else np.asarray(W2)
    outs = []
    for G in range(n_cts(O_c, g)):
        acc = None
        for c in range(r):
            sl = restore_slots(W2m, shape, n, G, c, O_c)
            if not sl.any():
                continue
            term = bfv.mul_plain(prm, y1[c], bfv.pt_rns(encode(sl, prm), prm))
            ops.mulpc += 1
            if acc is None:
                acc = term
            else:
                acc = bfv.add(prm, acc, term)
                ops.addcc += 1
        outs.append(acc)
    return outs


def pool_steps(shape: DeepShape):
    return [1 << e for e in range(shape.Bk.bit_length() - 1)]


def he_pool(prm, ct, shape: DeepShape, keys, ops: OpCount = None):
    ops = ops if ops is not None else OpCount()
    for st in pool_steps(shape):
        ct = bfv.add(prm, ct, bfv.rotate(prm, ct, st, keys))
        ops.rot += 1
        ops.addcc += 1
    return ct


def fc_inputs(C: int, shape: DeepShape, n: int):
    """(ciphertext, position) of every pooled feature c (block start)."""
    g = per_ct(shape, n)
    return [(c // g, (c % g) * shape.Bk) for c in range(C)]


def pooled_fc_features(F, C: int, shape: DeepShape, n: int):
    """The classifier with the sum pooling folded in: features (c, pixel) at (ciphertext c // g,
    slot (c mod g) Bk + pixel) with weight F[j][c]; returns (weights [m][C H W], ct_of, pos)."""
    g = per_ct(shape, n)
    hw = shape.H * shape.W
    F = np.asarray(F, dtype=np.int64)
    ct_of, pos = [], []
    for c in range(C):
        for p in range(hw):
            ct_of.append(c // g)
            pos.append((c % g) * shape.Bk + p)
    return np.repeat(F, hw, axis=1), ct_of, pos


def fc_diagonals_multi(F, ct_of, pos, n: int, per: int):
    """diag[G][k] of the fully connected layer over several ciphertexts: feature i at slot
    pos[i] (inside one period) of ciphertext ct_of[i]."""
    F = np.asarray(F, dtype=np.int64)
    m = F.shape[0]
    M = next_pow2(m)
    half = n // 2
    nG = max(ct_of) + 1
    inv = -np.ones((nG, per), dtype=np.int64)
    for i, (G, p) in enumerate(zip(ct_of, pos)):
        if not 0 <= p < per or inv[G, p] >= 0:
            raise ValueError("feature positions must be distinct and inside one period")
        inv[G, p] = i
    diags = [[np.zeros(n, dtype=np.int64) for _ in range(M)] for _ in range(nG)]
    p_all = np.arange(half)
    j_all = p_all % M
    for G in range(nG):
        for k in range(M):
            i_all = inv[G, (p_all + k) % per]
            ok = (j_all < m) & (i_all >= 0)
            diags[G][k][p_all[ok]] = F[j_all[ok], i_all[ok]]
    return diags


def fc_sum_steps(m: int, n: int):
    M = next_pow2(m)
    return [M << e for e in range((n // 2 // M).bit_length() - 1)]


def he_fc_multi(prm, cts, F, ct_of, pos, keys, ops: OpCount = None):
    """Fully connected layer over the ciphertexts cts (period N/2)."""
    ops = ops if ops is not None else OpCount()
    diags = fc_diagonals_multi(F, ct_of, pos, prm.n, prm.n // 2)
    M = len(diags[0])
    acc = None
    for G, ct in enumerate(cts):
        pairs = [bfv.scale_by_p_ext(prm, ct)] + bfv.rotate_hoisted_ext(prm, ct, list(range(1, M)),
                                                                        keys)
        ops.rot += M - 1
        for k in range(M):
            pt = bfv.pt_rns_ext(encode(diags[G][k], prm), prm)
            term = [bfv.rns_mul(pairs[k][h], pt, prm, prm.qp) for h in range(2)]
            ops.mulpc += 1
            if acc is None:
                acc = term
            else:
                acc = [bfv.rns_add(acc[h], term[h], prm.qp) for h in range(2)]
                ops.addcc += 1
    out = bfv.Ct(bfv.moddown(prm, acc[0]), bfv.moddown(prm, acc[1]))
    for st in fc_sum_steps(len(F), prm.n):
        out = bfv.add(prm, out, bfv.rotate(prm, out, st, keys))
        ops.rot += 1
        ops.addcc += 1
    return out


def deep_steps(shape: DeepShape, n: int):
    """Every rotation step of the network (Galois keys to generate)."""
    half = n // 2
    st = []
    for spec in shape.convs:
        st += [dl for (_, _, dl) in tap_offsets(spec, shape) if dl != 0]
    st += fold_steps(shape, n)
    st += list(range(1, next_pow2(shape.n_cls))) + fc_sum_steps(shape.n_cls, n)
    out = []
    for s in st:
        s = s % half
        if s and s not in out:
            out.append(s)
    return out


def he_deep(prm, cts_in, weights, shape: DeepShape, keys, rlk, ops: OpCount = None,
            trace=None):
    """The encrypted network; returns the logits ciphertext (logit j at slots p = j mod M)."""
    ops = ops if ops is not None else OpCount()
    cts = list(cts_in)
    C = shape.C0
    for spec, (W1, W2) in zip(shape.convs, weights["convs"]):
        cts = he_conv(prm, cts, W1, W2, spec, C, shape, keys, ops)
        cts = [bfv.relinearize(prm, bfv.multiply(prm, c, c), rlk) for c in cts]
        C = spec.O_c
        if trace is not None:
            trace.append(cts)
    Fx, ct_of, pos = pooled_fc_features(weights["fc"], C, shape, prm.n)
    return he_fc_multi(prm, cts, Fx, ct_of, pos, keys, ops)


def rand_weights(shape: DeepShape, seed: int, lo=-8, hi=8):
    """Seeded integer weights of the given shape (uniform in [lo, hi])."""
    rng = np.random.default_rng(seed)
    convs = []
    C = shape.C0
    for spec in shape.convs:
        r = spec.O_c if spec.r is None else spec.r
        W1 = rng.integers(lo, hi + 1, (r, C, spec.d, spec.d))
        W2 = None if spec.r is None else rng.integers(lo, hi + 1, (spec.O_c, spec.r))
        convs.append((W1, W2))
        C = spec.O_c
    return {"convs": convs, "fc": rng.integers(lo, hi + 1, (shape.n_cls, C))}


def expected_rotations(shape: DeepShape, n: int):
    """Rotation count per image of the schedule (Table I's quantity for this packing)."""
    g = per_ct(shape, n)
    rot, C = 0, shape.C0
    for spec in shape.convs:
        taps = sum(1 for (_, _, dl) in tap_offsets(spec, shape) if dl != 0)
        r = spec.O_c if spec.r is None else spec.r
        rot += n_cts(C, g) * taps + r * len(fold_steps(shape, n))
        C = spec.O_c
    nC = n_cts(C, g)
    rot += nC * (next_pow2(shape.n_cls) - 1) + len(fc_sum_steps(shape.n_cls, n))
    return rot
