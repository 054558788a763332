"""FFConv layer: the plain factorized convolution and its two encrypted schedules.

TEST INFRASTRUCTURE (independent CPU oracle).

Plain layer (Sec. 3.1 Eq. 1, Sec. 4.1 Eq. 2): a d x d convolution written as the product
I x W of the Im2Col matrix I (S = O_h O_w rows, K = d^2 I_c columns) with the weight matrix,
here factorized as W = W1 W2 with W1 (K x r) the d x d low-rank filters and W2 (r x O_c) the
1 x 1 restoring convolution.  Filters are applied as a cross-correlation (no flip), zero
padding `pad` on every side, output size floor((I + 2 pad - d) / stride) + 1.

Encrypted layer, FFConv packing DP-HI2C-CP (Sec. 4.2, Fig. 4): W1 under DensePack (Sec. 3.2,
Fig. 1), the DP -> CP transition with a 1 x 1 kernel (Table III, d = 1 row), W2 under
ConvPack (Sec. 3.2, Fig. 2a).  Schedules of W1:

  dp_dot   (the paper's DensePack): the input is packed densely in row 0,
           slot ci*I_h*I_w + h*I_w + w.  For every output channel c' and output position o
           the filter is zero-padded to the input size at its shifted location (Fig. 1a),
           multiplied into the ciphertext, and all slots are summed by rotate-and-sum
           (Fig. 1b): prod <- prod + rot(prod, 2^e), e = 0 .. k-1 with 2^k covering the
           occupied slots (log2(N/2) steps plus one row swap when the input fills both
           rows), after which slot o holds the dot product of output o.  The DP -> CP step multiplies by the
           one-hot mask of slot o and adds over o (no rotation, Table III), giving one
           ciphertext per low-rank channel with y1[c', o] at slot o = oh*O_w + ow.
  dp_shift (one rotation per filter tap, hoisted): input channel ci occupies a block of
           B_c slots, slot ci*B_c + h*I_w + w.  For every tap (i, j), in ascending order,
           the input is rotated by delta = (i - pad) I_w + (j - pad) (one shared ModUp for
           all taps) and multiplied by a plaintext holding W1[c', ci, i, j] at slot
           ci*B_c + (s oh) I_w + s ow wherever that input pixel lies inside the image;
           channels are then folded with acc <- acc + rot(acc, B_c 2^k).  y1[c', oh, ow]
           lands at slot (s oh) I_w + s ow.
  cp_cp    (CP-HI2C-CP, Sec. 4.2 'ConvPack for W1', Fig. 5): the client packs the Im2Col
           columns of the input (one ciphertext per column, I[o, k] at slot o); W1 and W2 are
           both ConvPack scalar products and the layer needs no rotation.
  dp_dp    (DP-DP, Table IX's DensePack-DensePack baseline): W1 exactly as dp_dot, then the
           r channel ciphertexts are combined into one dense vector Y (channel c' rotated by
           -c' S, so y1[c', o] sits at slot c' S + o) and W2 is a DensePack layer too: for every
           output (c, o), Y times the plaintext holding W2[c, c'] at slot c' S + o, rotate-and-
           sum with steps 1, 2, .., 2^(k2-1) where 2^k2 > (r - 1) S (slot o then holds the dot
           product), and the one-hot mask of slot o gathers the O_c S products into the O_c
           output ciphertexts (y2[c, oh, ow] at slot oh O_w + ow).
  dp_shift_ext (the same slots and plaintexts as dp_shift): the hoisted rotations stay in the
           extended basis Q u P, each as (u0 + P phi(c0), u1); the tap products are summed
           there (plaintexts lifted to Q u P) and divided by P once per channel (one ModDown
           per channel instead of one per rotation).  A different algorithm from dp_shift,
           with its own ciphertext bits; both decrypt to the same slots.

W2 (ConvPack, Table II): ct_out[c] = sum_c' W2[c, c'] ct_w1[c'], each weight a constant
plaintext.  An optional modulus switch drops the last prime at the end.
"""
from dataclasses import dataclass

import numpy as np

from . import bfv
from .encoder import encode


@dataclass
class Layout:
    I_c: int
    I_h: int
    I_w: int
    d: int
    stride: int
    pad: int
    r: int
    O_c: int
    pack: str = "dp_shift"      # "dp_dot" | "dp_shift" | "dp_shift_ext" | "cp_cp" | "dp_dp"
    modswitch: bool = False

    @property
    def O_h(self):
        return (self.I_h + 2 * self.pad - self.d) // self.stride + 1

    @property
    def O_w(self):
        return (self.I_w + 2 * self.pad - self.d) // self.stride + 1

    @property
    def S(self):
        return self.O_h * self.O_w

    @property
    def B_c(self):
        hw = self.I_h * self.I_w
        if self.I_c == 1:
            return hw
        return 1 << (hw - 1).bit_length()

    def taps(self):
        """(i, j, delta) for every filter tap, ascending (i, j)."""
        return [(i, j, (i - self.pad) * self.I_w + (j - self.pad))
                for i in range(self.d) for j in range(self.d)]

    def channel_fold_steps(self):
        k = (self.I_c - 1).bit_length()
        return [self.B_c << e for e in range(k)]


# ---------------------------------------------------------------- plain layer (Eq. 1, Eq. 2)

def im2col(x, lay: Layout):
    """The S x K matrix I of Eq. 1: row o = the d x d x I_c patch under output position o."""
    I = np.zeros((lay.S, lay.d * lay.d * lay.I_c), dtype=np.int64)
    for oh in range(lay.O_h):
        for ow in range(lay.O_w):
            row = []
            for ci in range(lay.I_c):
                for i in range(lay.d):
                    for j in range(lay.d):
                        h = lay.stride * oh + i - lay.pad
                        w = lay.stride * ow + j - lay.pad
                        inside = 0 <= h < lay.I_h and 0 <= w < lay.I_w
                        row.append(int(x[ci, h, w]) if inside else 0)
            I[oh * lay.O_w + ow] = row
    return I


def plain_layer(x, W1, W2, lay: Layout):
    """y1 = I W1 (low-rank d x d conv), y2 = y1 W2 (1 x 1 restore); shapes [r|O_c][O_h][O_w]."""
    I = im2col(np.asarray(x), lay)
    W1m = np.asarray(W1, dtype=np.int64).reshape(lay.r, -1).T          # K x r
    W2m = np.asarray(W2, dtype=np.int64).T                             # r x O_c
    y1 = I @ W1m
    y2 = y1 @ W2m
    return (y1.T.reshape(lay.r, lay.O_h, lay.O_w), y2.T.reshape(lay.O_c, lay.O_h, lay.O_w))


# ---------------------------------------------------------------- slot layouts

def input_slots(x, lay: Layout, n: int):
    """Slot vector of the packed input image (row 0)."""
    v = np.zeros(n, dtype=np.int64)
    hw = lay.I_h * lay.I_w
    block = hw if lay.pack in ("dp_dot", "dp_dp") else lay.B_c
    for ci in range(lay.I_c):
        v[ci * block: ci * block + hw] = np.asarray(x[ci]).reshape(-1)
    return v


def output_slot(lay: Layout, oh: int, ow: int) -> int:
    if lay.pack in ("dp_dot", "cp_cp", "dp_dp"):
        return oh * lay.O_w + ow
    return (lay.stride * oh) * lay.I_w + lay.stride * ow


def check_fits(lay: Layout, n: int):
    half = n // 2
    if lay.pack == "cp_cp":
        if lay.S > n:
            raise ValueError("cp_cp output positions must fit in N slots")
        return
    if lay.pack in ("dp_dot", "dp_dp"):
        if lay.I_c * lay.I_h * lay.I_w > n or lay.S > half:
            raise ValueError("dp_dot input must fit in N slots and its output in N/2")
        if lay.pack == "dp_dp" and (lay.r * lay.S > half or lay.modswitch):
            raise ValueError("dp_dp needs r S <= N/2 (one dense vector) and no modulus switch")
    else:
        span = lay.B_c * (1 << (lay.I_c - 1).bit_length())
        if span > half:
            raise ValueError("dp_shift channel blocks must fit in one row of N/2 slots")


def spans_both_rows(lay: Layout, n: int) -> bool:
    return lay.pack in ("dp_dot", "dp_dp") and lay.I_c * lay.I_h * lay.I_w > n // 2


def _window_covers(lay: Layout, k: int) -> bool:
    """After k rotate-and-sum steps slot o holds sum_{m < 2^k} prod[o + m]; true when every
    output's padded filter lies inside [o, o + 2^k), so slot o holds exactly its dot product."""
    hw = lay.I_h * lay.I_w
    for oh in range(lay.O_h):
        for ow in range(lay.O_w):
            o = oh * lay.O_w + ow
            hs = [lay.stride * oh + i - lay.pad for i in range(lay.d)]
            ws = [lay.stride * ow + j - lay.pad for j in range(lay.d)]
            hs = [h for h in hs if 0 <= h < lay.I_h]
            ws = [w for w in ws if 0 <= w < lay.I_w]
            if not hs or not ws:
                continue
            lo = min(hs) * lay.I_w + min(ws)
            hi = (lay.I_c - 1) * hw + max(hs) * lay.I_w + max(ws)
            if lo < o or hi >= o + (1 << k):
                return False
    return True


def dp_dot_sum_depth(lay: Layout, n: int) -> int:
    """Rotate-and-sum depth k: ceil(log2 of the occupied slots) when every output's window
    covers its filter, else log2(N/2) (every slot of the row then holds the row's sum)."""
    half = n // 2
    full = half.bit_length() - 1
    span = lay.I_c * lay.I_h * lay.I_w
    if span > half:
        return full
    k = max(0, (span - 1).bit_length())
    return k if k < full and _window_covers(lay, k) else full


def dp_dot_steps(lay: Layout, n: int):
    """Rotate-and-sum steps 1, 2, ..., 2^(k-1), then the row swap when the input occupies both
    rows.  This reproduces Table VIII: 14 steps for the 16268-slot input at N = 16384 (7000 =
    500 x 14) and 12 for the 4075-slot FC input (120 = 10 x 12)."""
    steps = [1 << e for e in range(dp_dot_sum_depth(lay, n))]
    return steps + ([bfv.ROW_SWAP] if spans_both_rows(lay, n) else [])


def dp_dp_combine_steps(lay: Layout):
    """Rotations moving channel c' of W1's output to slots c' S + o (c' = 1 .. r-1)."""
    return [-c * lay.S for c in range(1, lay.r)]


def dp_dp_sum_steps(lay: Layout):
    """W2's rotate-and-sum: 1, 2, .., 2^(k2-1) with 2^k2 > (r - 1) S."""
    k2 = ((lay.r - 1) * lay.S).bit_length()
    return [1 << e for e in range(k2)]


def required_steps(lay: Layout, n: int):
    """Rotation steps (slots) whose Galois keys the layer needs."""
    if lay.pack == "cp_cp":
        return []
    if lay.pack == "dp_dot":
        return dp_dot_steps(lay, n)
    if lay.pack == "dp_dp":
        out = []
        for st in dp_dot_steps(lay, n) + dp_dp_combine_steps(lay) + dp_dp_sum_steps(lay):
            if st not in out:
                out.append(st)
        return out
    steps = [dl for (_, _, dl) in lay.taps() if dl != 0]
    return steps + lay.channel_fold_steps()


# ---------------------------------------------------------------- plaintexts of the schedules

def dp_dot_filter_slots(W1, lay: Layout, n: int, c: int, oh: int, ow: int):
    """Filter c zero-padded to the input size at output position (oh, ow) (Fig. 1a)."""
    v = np.zeros(n, dtype=np.int64)
    hw = lay.I_h * lay.I_w
    for ci in range(lay.I_c):
        for i in range(lay.d):
            for j in range(lay.d):
                h = lay.stride * oh + i - lay.pad
                w = lay.stride * ow + j - lay.pad
                if 0 <= h < lay.I_h and 0 <= w < lay.I_w:
                    v[ci * hw + h * lay.I_w + w] = W1[c][ci][i][j]
    return v


def dp_shift_tap_slots(W1, lay: Layout, n: int, c: int, i: int, j: int):
    """Plaintext of tap (i, j) for channel c: W1[c, ci, i, j] at every output base slot."""
    v = np.zeros(n, dtype=np.int64)
    for ci in range(lay.I_c):
        for oh in range(lay.O_h):
            for ow in range(lay.O_w):
                h = lay.stride * oh + i - lay.pad
                w = lay.stride * ow + j - lay.pad
                if 0 <= h < lay.I_h and 0 <= w < lay.I_w:
                    v[ci * lay.B_c + output_slot(lay, oh, ow)] = W1[c][ci][i][j]
    return v


def dp_dp_row_slots(W2, lay: Layout, n: int, c: int, o: int):
    """Row (c, o) of W2 under DensePack: W2[c, c'] at slot c' S + o of the dense vector."""
    v = np.zeros(n, dtype=np.int64)
    for cp in range(lay.r):
        v[cp * lay.S + o] = W2[c][cp]
    return v


def mask_slots(n: int, o: int):
    v = np.zeros(n, dtype=np.int64)
    v[o] = 1
    return v


# ---------------------------------------------------------------- encrypted layer

class OpCount:
    def __init__(self):
        self.mulpc = 0
        self.addcc = 0
        self.rot = 0

    def as_dict(self):
        return {"mulpc": self.mulpc, "addcc": self.addcc, "rot": self.rot}


def _restore(prm, cts_w1, W2, lay: Layout, ops: OpCount):
    """W2 under ConvPack: ct_out[c] = sum_c' W2[c][c'] ct_w1[c'] (Table II)."""
    outs = []
    for c in range(lay.O_c):
        acc = None
        for cp in range(lay.r):
            term = bfv.mul_scalar(prm, cts_w1[cp], int(W2[c][cp]))
            ops.mulpc += 1
            if acc is None:
                acc = term
            else:
                acc = bfv.add(prm, acc, term)
                ops.addcc += 1
        if lay.modswitch:
            acc = bfv.rescale(prm, acc)
        outs.append(acc)
    return outs


def im2col_slots(x, lay: Layout, n: int):
    """Client-side plaintext Im2Col (Sec. 3.1 Eq. 1, Table VI's 64 x 144 input): one slot
    vector per column k = (ci, i, j) of I, holding I[o, k] at slot o = oh O_w + ow."""
    I = im2col(np.asarray(x), lay)
    out = []
    for k in range(I.shape[1]):
        v = np.zeros(n, dtype=np.int64)
        v[: lay.S] = I[:, k]
        out.append(v)
    return out


def he_layer_cp_cp(prm, cts_in, W1, W2, lay: Layout, ops: OpCount = None):
    """FFConv packing CP-HI2C-CP (Sec. 4.2 'ConvPack for W1', Fig. 5): the K = d^2 I_c input
    ciphertexts hold the Im2Col columns; W1 under ConvPack is ct_w1[c'] = sum_k W1[c', k] ct_k
    (Table II), HGrouping for the 1 x 1 W2 is free (Table III, CP-HI2C-CP, d = 1: the r
    results already hold one channel each), W2 under ConvPack as in the other schedules."""
    check_fits(lay, prm.n)
    ops = ops if ops is not None else OpCount()
    W1m = np.asarray(W1, dtype=np.int64).reshape(lay.r, -1)
    cts_w1 = []
    for c in range(lay.r):
        acc = None
        for k, ct in enumerate(cts_in):
            term = bfv.mul_scalar(prm, ct, int(W1m[c, k]))
            ops.mulpc += 1
            if acc is None:
                acc = term
            else:
                acc = bfv.add(prm, acc, term)
                ops.addcc += 1
        cts_w1.append(acc)
    return _restore(prm, cts_w1, W2, lay, ops)


def he_layer(prm, ct_in, W1, W2, lay: Layout, keys, ops: OpCount = None,
             channels=None):
    """Encrypted FFConv layer; returns the O_c output ciphertexts (coefficient domain).
    For the cp_cp schedule ct_in is the list of K Im2Col column ciphertexts."""
    if lay.pack == "cp_cp":
        return he_layer_cp_cp(prm, ct_in, W1, W2, lay, ops)
    check_fits(lay, prm.n)
    ops = ops if ops is not None else OpCount()
    n = prm.n
    half = n // 2
    cts_w1 = []
    if lay.pack in ("dp_dot", "dp_dp"):
        sum_steps = dp_dot_steps(lay, n)
        for c in range(lay.r):
            acc = None
            for oh in range(lay.O_h):
                for ow in range(lay.O_w):
                    o = oh * lay.O_w + ow
                    pt = bfv.pt_rns(encode(dp_dot_filter_slots(W1, lay, n, c, oh, ow), prm), prm)
                    prod = bfv.mul_plain(prm, ct_in, pt)
                    ops.mulpc += 1
                    for st in sum_steps:
                        prod = bfv.add(prm, prod, bfv.rotate(prm, prod, st, keys))
                        ops.rot += 1
                        ops.addcc += 1
                    mask = bfv.pt_rns(encode(mask_slots(n, o), prm), prm)
                    term = bfv.mul_plain(prm, prod, mask)
                    ops.mulpc += 1
                    if acc is None:
                        acc = term
                    else:
                        acc = bfv.add(prm, acc, term)
                        ops.addcc += 1
            cts_w1.append(acc)
    else:
        taps = lay.taps()
        steps = [dl for (_, _, dl) in taps if dl != 0]
        ext = lay.pack == "dp_shift_ext"
        if ext:
            # rotations left in the extended basis Q u P (before ModDown), Sec. 3.2's
            # rotate-then-multiply with the division by P moved after the tap sum
            rotated = bfv.rotate_hoisted_ext(prm, ct_in, steps, keys)
            by_delta = dict(zip(steps, rotated))
            by_delta[0] = bfv.scale_by_p_ext(prm, ct_in)
        else:
            rotated = bfv.rotate_hoisted(prm, ct_in, steps, keys)
            by_delta = dict(zip(steps, rotated))
            by_delta[0] = ct_in
        ops.rot += len(steps)
        for c in range(lay.r):
            acc = None
            for (i, j, dl) in taps:
                m = encode(dp_shift_tap_slots(W1, lay, n, c, i, j), prm)
                if ext:
                    pt = bfv.pt_rns_ext(m, prm)
                    term = [bfv.rns_mul(by_delta[dl][k], pt, prm, prm.qp) for k in range(2)]
                else:
                    term = bfv.mul_plain(prm, by_delta[dl], bfv.pt_rns(m, prm))
                ops.mulpc += 1
                if acc is None:
                    acc = term
                elif ext:
                    acc = [bfv.rns_add(acc[k], term[k], prm.qp) for k in range(2)]
                    ops.addcc += 1
                else:
                    acc = bfv.add(prm, acc, term)
                    ops.addcc += 1
            if ext:
                acc = bfv.Ct(bfv.moddown(prm, acc[0]), bfv.moddown(prm, acc[1]))
            for st in lay.channel_fold_steps():
                acc = bfv.add(prm, acc, bfv.rotate(prm, acc, st, keys))
                ops.rot += 1
                ops.addcc += 1
            cts_w1.append(acc)
    if lay.pack == "dp_dp":
        return _w2_dense(prm, cts_w1, W2, lay, keys, ops)
    return _restore(prm, cts_w1, W2, lay, ops)


def _w2_dense(prm, cts_w1, W2, lay: Layout, keys, ops: OpCount):
    """W2 under DensePack (dp_dp): combine the channel ciphertexts into one dense vector, then
    one dense vector-row product per output (c, o), gathered by one-hot masks."""
    n = prm.n
    Y = cts_w1[0]
    for cp, st in zip(range(1, lay.r), dp_dp_combine_steps(lay)):
        Y = bfv.add(prm, Y, bfv.rotate(prm, cts_w1[cp], st, keys))
        ops.rot += 1
        ops.addcc += 1
    outs = []
    for c in range(lay.O_c):
        acc = None
        for o in range(lay.S):
            z = bfv.mul_plain(prm, Y, bfv.pt_rns(encode(dp_dp_row_slots(W2, lay, n, c, o), prm), prm))
            ops.mulpc += 1
            for st in dp_dp_sum_steps(lay):
                z = bfv.add(prm, z, bfv.rotate(prm, z, st, keys))
                ops.rot += 1
                ops.addcc += 1
            term = bfv.mul_plain(prm, z, bfv.pt_rns(encode(mask_slots(n, o), prm), prm))
            ops.mulpc += 1
            if acc is None:
                acc = term
            else:
                acc = bfv.add(prm, acc, term)
                ops.addcc += 1
        outs.append(acc)
    return outs


def expected_ops(lay: Layout, n: int):
    """Operation counts of the schedules (Tables I-III for the paper's dp_dot form)."""
    n_sum = len(dp_dot_steps(lay, n)) if lay.pack in ("dp_dot", "dp_dp") else 0
    r, S, O_c = lay.r, lay.S, lay.O_c
    restore_mul, restore_add = O_c * r, O_c * (r - 1)
    if lay.pack == "cp_cp":
        K = lay.d * lay.d * lay.I_c     # Table II, FFConv row: MulPC O'_c (K + O_c)
        return {"mulpc": r * (K + O_c), "addcc": r * (K - 1) + restore_add, "rot": 0}
    if lay.pack == "dp_dp":
        k2 = len(dp_dp_sum_steps(lay))
        return {"mulpc": 2 * r * S + 2 * O_c * S,
                "addcc": r * S * n_sum + r * (S - 1) + (r - 1) + O_c * S * k2 + O_c * (S - 1),
                "rot": r * S * n_sum + (r - 1) + O_c * S * k2}
    if lay.pack == "dp_dot":
        return {"mulpc": 2 * r * S + restore_mul,
                "addcc": r * S * n_sum + r * (S - 1) + restore_add,
                "rot": r * S * n_sum}
    taps = lay.d * lay.d
    fold = len(lay.channel_fold_steps())
    n_rot = sum(1 for (_, _, dl) in lay.taps() if dl != 0)
    return {"mulpc": r * taps + restore_mul,
            "addcc": r * (taps - 1) + r * fold + restore_add,
            "rot": n_rot + r * fold}
