"""Three-layer encrypted network: FFConv layer, x^2, fully connected, x^2, fully connected.

TEST INFRASTRUCTURE (independent CPU oracle).

The network follows the paper's pipeline for an image network under BFV (Sec. 3 and the
per-layer breakdown of Table VIII): a factorized convolution (the FFConv layer of ffconv.py),
the square activation (Sec. 3, the CryptoNets substitute for ReLU), the output channels
combined into one densely packed vector by rotations and additions (Table VIII, "combine to
one vector"), and fully connected layers evaluated as DensePack dot products over that
vector (Sec. 3: a fully connected layer is a convolution whose filter covers the whole input).

Plain network (exact integers, compared mod t as in ffconv.py):
    y   = FFConv(x)                     [O_c][O_h][O_w]
    a1  = y^2,   flattened in (c, oh, ow) order (length n1 = O_c O_h O_w)
    z1  = F1 a1  (F1: [m1][n1]),  a2 = z1^2,  z2 = F2 a2  (F2: [m2][m1])

Encrypted schedule (the readings, each also listed among the design readings):
  combine: ct = sum_c rot(ct_c, -c * blk), blk the smallest power of two above every output
           slot of the layer, so channel c's values move to slots c*blk + slot(oh, ow);
  square:  relinearize(multiply(ct, ct)) (bfv.py);
  fc:      the dot products y_j = sum_i F[j][i] x_i for all outputs at once.  With the input
           value x_i at slot pos_i of row 0, repeating with period `per` (a power of two
           dividing N/2; per = N/2 when the input does not repeat) and M the smallest power of
           two >= the output count m, the diagonals
               diag_k[p] = F[p mod M][i]  where (p + k) mod per = pos_i and p mod M < m
           (zero elsewhere, row 1 zero) give z = sum_{k<M} rot(x, k) * diag_k with
           z[p] = sum of the terms F[p mod M][i] x_i whose pos_i lies in the window
           p .. p + M - 1 (mod per); summing z over the per/M slots p = j (mod M) of one period
           (rotate-and-sum: z <- z + rot(z, M 2^e), e < log2(per/M)) covers every input exactly
           once, so slot p holds y_{p mod M} (0 when p mod M >= m): the output repeats with
           period M.  The M - 1 rotations of x share one ModUp and are summed in Q u P with a
           single ModDown (the same algorithm as the dp_shift_ext taps in ffconv.py).
"""
import numpy as np

from . import bfv
from .encoder import encode
from .ffconv import Layout, OpCount, he_layer, output_slot, plain_layer


def next_pow2(x: int) -> int:
    return 1 << max(0, (int(x) - 1).bit_length())


def combine_block(lay: Layout) -> int:
    """Slot distance between consecutive channels of the combined vector."""
    top = max(output_slot(lay, oh, ow) for oh in range(lay.O_h) for ow in range(lay.O_w))
    return next_pow2(top + 1)


def combined_positions(lay: Layout):
    """pos[c*S + oh*O_w + ow] = c*blk + slot(oh, ow): where the combined vector holds a1."""
    blk = combine_block(lay)
    return [c * blk + output_slot(lay, oh, ow)
            for c in range(lay.O_c) for oh in range(lay.O_h) for ow in range(lay.O_w)]


def plain_net(x, W1, W2, lay: Layout, F1, F2, t: int):
    """Exact plain network, reduced mod t at the end: (a1, z1, z2) as int64 arrays mod t."""
    _, y2 = plain_layer(x, W1, W2, lay)
    a1 = (np.asarray(y2, dtype=object).reshape(-1) ** 2)
    z1 = np.asarray(F1, dtype=object) @ a1
    a2 = z1 ** 2
    z2 = np.asarray(F2, dtype=object) @ a2
    red = lambda v: np.array([int(e) % t for e in v], dtype=np.int64)
    return red(a1), red(z1), red(z2)


def fc_diagonals(F, pos, per: int, n: int):
    """The M plaintext slot vectors diag_k (k < M) of the fc schedule above."""
    F = np.asarray(F, dtype=np.int64)
    m, n_in = F.shape
    M = next_pow2(m)
    half = n // 2
    if per & (per - 1) or per < M or half % per:
        raise ValueError("period must be a power of two with M <= per | N/2")
    inv = -np.ones(per, dtype=np.int64)
    for i, p in enumerate(pos):
        if not 0 <= p < per or inv[p] >= 0:
            raise ValueError("input positions must be distinct and inside one period")
        inv[p] = i
    diags = []
    for k in range(M):
        v = np.zeros(n, dtype=np.int64)
        for p in range(half):
            j = p % M
            if j >= m:
                continue
            i = inv[(p + k) % per]
            if i >= 0:
                v[p] = F[j, i]
        diags.append(v)
    return diags


def fc_sum_steps(m: int, per: int):
    M = next_pow2(m)
    return [M << e for e in range((per // M).bit_length() - 1)]


def fc_steps(m: int, per: int):
    """Rotation steps of one fc layer: the M - 1 diagonal offsets, then the sum steps."""
    return list(range(1, next_pow2(m))) + fc_sum_steps(m, per)


def he_fc(prm, ct: bfv.Ct, F, pos, per: int, keys, ops: OpCount = None) -> bfv.Ct:
    """Encrypted fully connected layer (the fc schedule of the module docstring)."""
    ops = ops if ops is not None else OpCount()
    diags = fc_diagonals(F, pos, per, prm.n)
    M = len(diags)
    rotated = bfv.rotate_hoisted_ext(prm, ct, list(range(1, M)), keys)
    pairs = [bfv.scale_by_p_ext(prm, ct)] + rotated
    ops.rot += M - 1
    acc = None
    for k in range(M):
        pt = bfv.pt_rns_ext(encode(diags[k], prm), prm)
        term = [bfv.rns_mul(pairs[k][h], pt, prm, prm.qp) for h in range(2)]
        ops.mulpc += 1
        if acc is None:
            acc = term
        else:
            acc = [bfv.rns_add(acc[h], term[h], prm.qp) for h in range(2)]
            ops.addcc += 1
    out = bfv.Ct(bfv.moddown(prm, acc[0]), bfv.moddown(prm, acc[1]))
    for st in fc_sum_steps(len(F), per):
        out = bfv.add(prm, out, bfv.rotate(prm, out, st, keys))
        ops.rot += 1
        ops.addcc += 1
    return out


def he_combine(prm, cts, blk: int, keys, ops: OpCount = None) -> bfv.Ct:
    """ct = ct_0 + sum_{c >= 1} rot(ct_c, -c blk), in ascending c."""
    ops = ops if ops is not None else OpCount()
    acc = cts[0]
    for c in range(1, len(cts)):
        acc = bfv.add(prm, acc, bfv.rotate(prm, cts[c], -c * blk, keys))
        ops.rot += 1
        ops.addcc += 1
    return acc


def he_square(prm, ct: bfv.Ct, rlk) -> bfv.Ct:
    return bfv.relinearize(prm, bfv.multiply(prm, ct, ct), rlk)


def net_steps(lay: Layout, m1: int, m2: int, n: int):
    """Every rotation step the network uses (Galois keys to generate)."""
    from .ffconv import required_steps
    half = n // 2
    blk = combine_block(lay)
    steps = list(required_steps(lay, n))
    steps += [(-c * blk) % half for c in range(1, lay.O_c)]
    steps += fc_steps(m1, half) + fc_steps(m2, next_pow2(m1))
    out = []
    for s in steps:
        if s not in out:
            out.append(s)
    return out


def check_net(lay: Layout, m1: int, m2: int, n: int):
    half = n // 2
    blk = combine_block(lay)
    if lay.O_c * blk > half:
        raise ValueError("the combined channels must fit in one row")
    if next_pow2(m1) > half or next_pow2(m2) > next_pow2(m1):
        raise ValueError("fc output counts do not fit their periods")


def he_net(prm, ct_in, W1, W2, lay: Layout, F1, F2, keys, rlk, ops: OpCount = None):
    """The encrypted network; returns the final ciphertext (z2_j at slots p = j mod M2)."""
    ops = ops if ops is not None else OpCount()
    n = prm.n
    F1 = np.asarray(F1, dtype=np.int64)
    F2 = np.asarray(F2, dtype=np.int64)
    check_net(lay, F1.shape[0], F2.shape[0], n)
    cts = he_layer(prm, ct_in, W1, W2, lay, keys, ops)
    ct = he_combine(prm, cts, combine_block(lay), keys, ops)
    ct = he_square(prm, ct, rlk)
    ct = he_fc(prm, ct, F1, combined_positions(lay), n // 2, keys, ops)
    ct = he_square(prm, ct, rlk)
    M1 = next_pow2(F1.shape[0])
    ct = he_fc(prm, ct, F2, list(range(F1.shape[0])), M1, keys, ops)
    return ct


def output_slots(m2: int, n: int):
    """Slots of row 0 holding z2_j after he_net: p with p mod M2 = j < m2."""
    M2 = next_pow2(m2)
    return [p for p in range(n // 2) if p % M2 < m2]
