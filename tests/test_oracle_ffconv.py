"""Pins for the oracle's FFConv layer: the plain factorized convolution against PyTorch's
conv2d, the encrypted layer's decrypted output against the plain one (exact, mod t), and the
rotation counts against the paper's Table VIII."""
import os

import numpy as np
import pytest
import torch

from oracle import bfv, encoder, ffconv, params

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def torch_reference(x, W1, W2, lay):
    xt = torch.tensor(np.asarray(x), dtype=torch.float64)[None]
    y1 = torch.nn.functional.conv2d(xt, torch.tensor(np.asarray(W1), dtype=torch.float64),
                                    stride=lay.stride, padding=lay.pad)
    y2 = torch.nn.functional.conv2d(y1, torch.tensor(np.asarray(W2), dtype=torch.float64)[:, :, None, None])
    return y1[0].round().long().numpy(), y2[0].round().long().numpy()


@pytest.mark.parametrize("shape", [(1, 28, 28, 5, 2, 1, 2, 5), (3, 9, 7, 3, 1, 1, 4, 6),
                                   (2, 8, 8, 3, 2, 0, 3, 2), (1, 5, 5, 5, 1, 2, 1, 1)])
def test_plain_layer_matches_conv2d(shape):
    I_c, I_h, I_w, d, s, p, r, O_c = shape
    lay = ffconv.Layout(I_c, I_h, I_w, d, s, p, r, O_c)
    rng = np.random.default_rng(sum(shape))
    x = rng.integers(0, 256, (I_c, I_h, I_w))
    W1 = rng.integers(-8, 9, (r, I_c, d, d))
    W2 = rng.integers(-8, 9, (O_c, r))
    y1, y2 = ffconv.plain_layer(x, W1, W2, lay)
    t1, t2 = torch_reference(x, W1, W2, lay)
    assert (y1 == t1).all() and (y2 == t2).all()
    assert lay.O_h == t1.shape[1] and lay.O_w == t1.shape[2]


def test_planted_transposed_filter_is_caught():
    lay = ffconv.Layout(1, 6, 6, 3, 1, 1, 1, 1)
    rng = np.random.default_rng(0)
    x = rng.integers(0, 256, (1, 6, 6))
    W1 = rng.integers(-8, 9, (1, 1, 3, 3))
    W2 = np.ones((1, 1), dtype=np.int64)
    y1, _ = ffconv.plain_layer(x, np.transpose(W1, (0, 1, 3, 2)), W2, lay)
    t1, _ = torch_reference(x, W1, W2, lay)
    assert not (y1 == t1).all()


def run_he(prm, lay, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 256, (lay.I_c, lay.I_h, lay.I_w))
    W1 = rng.integers(-8, 9, (lay.r, lay.I_c, lay.d, lay.d))
    W2 = rng.integers(-8, 9, (lay.O_c, lay.r))
    s = bfv.keygen_secret(prm, seed + 1)
    keys = {}
    for st in ffconv.required_steps(lay, prm.n):
        g = bfv.galois_of(st, prm.n)
        keys[g] = bfv.galois_key(prm, s, g, seed + 2)
    if lay.pack == "cp_cp":
        ct = [bfv.encrypt(prm, s, encoder.encode(v, prm), seed + 3 + k)
              for k, v in enumerate(ffconv.im2col_slots(x, lay, prm.n))]
    else:
        ct = bfv.encrypt(prm, s, encoder.encode(ffconv.input_slots(x, lay, prm.n), prm), seed + 3)
    ops = ffconv.OpCount()
    outs = ffconv.he_layer(prm, ct, W1, W2, lay, keys, ops)
    _, y2 = ffconv.plain_layer(x, W1, W2, lay)
    return prm, s, lay, outs, y2, ops


def check_outputs(prm, s, lay, outs, y2):
    for c, ct in enumerate(outs):
        v = encoder.decode(bfv.decrypt(prm, s, ct), prm)
        want = np.zeros(prm.n, dtype=np.int64)
        for oh in range(lay.O_h):
            for ow in range(lay.O_w):
                want[ffconv.output_slot(lay, oh, ow)] = y2[c, oh, ow] % prm.t
        if lay.I_c == 1 or lay.pack in ("dp_dot", "cp_cp", "dp_dp"):
            assert (v == want).all()
        else:   # folded channels leave partial sums in the other channel blocks
            pos = [ffconv.output_slot(lay, oh, ow) for oh in range(lay.O_h) for ow in range(lay.O_w)]
            assert (v[pos] == want[pos]).all()
        assert bfv.noise_bits(prm, s, ct)[1] > 10


@pytest.mark.parametrize("pack", ["dp_dot", "dp_shift", "dp_shift_ext", "cp_cp", "dp_dp"])
@pytest.mark.parametrize("shape", [(1, 6, 6, 3, 2, 1, 2, 3), (2, 5, 5, 3, 1, 1, 2, 2), (3, 4, 4, 3, 2, 1, 2, 3)])
def test_encrypted_layer_decrypts_to_plain_layer(pack, shape):
    prm = params.Params(log_n=7, n_q=3, n_p=1, alpha=1)
    lay = ffconv.Layout(*shape, pack=pack)
    prm, s, lay, outs, y2, ops = run_he(prm, lay, seed=shape[0])
    check_outputs(prm, s, lay, outs, y2)
    assert ops.as_dict() == ffconv.expected_ops(lay, prm.n)


def test_encrypted_layer_with_modswitch_and_wide_digits():
    prm = params.Params(log_n=7, n_q=4, n_p=2, alpha=2)
    lay = ffconv.Layout(1, 6, 6, 3, 2, 1, 2, 3, pack="dp_shift", modswitch=True)
    prm, s, lay, outs, y2, ops = run_he(prm, lay, seed=4)
    assert all(o.level == 3 for o in outs)
    check_outputs(prm, s, lay, outs, y2)


@pytest.mark.slow
def test_full_size_dp_shift_layer():
    """The 1x28x28, 5x5 stride-2 pad-1, r=2 -> 5 channel layer at N = 8192."""
    prm = params.cfg_small_layer()
    lay = ffconv.Layout(1, 28, 28, 5, 2, 1, 2, 5, pack="dp_shift")
    prm, s, lay, outs, y2, ops = run_he(prm, lay, seed=0)
    check_outputs(prm, s, lay, outs, y2)
    assert ops.rot == 24


def test_rotation_counts_match_table_viii():
    rows = [l.split() for l in open(os.path.join(GOLD, "paper_rotation_counts.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    for r in rows:
        n = int(r[1])
        I_c, I_h, I_w, d, s, p, rk, O_c, rot = map(int, r[2:11])
        lay = ffconv.Layout(I_c, I_h, I_w, d, s, p, rk, O_c, pack="dp_dot")
        assert ffconv.expected_ops(lay, n)["rot"] == rot


def test_layer_counts_of_the_28x28_workload():
    lay = ffconv.Layout(1, 28, 28, 5, 2, 1, 2, 5, pack="dp_dot")
    assert (lay.O_h, lay.O_w, lay.S) == (13, 13, 169)
    assert ffconv.dp_dot_sum_depth(lay, 8192) == 10
    assert ffconv.expected_ops(lay, 8192)["rot"] == 2 * 169 * 10


def test_extended_basis_schedule_differs_in_bits_but_not_in_slots():
    """dp_shift and dp_shift_ext divide by P at different points: different ciphertexts,
    identical decryptions."""
    prm = params.Params(log_n=7, n_q=3, n_p=1, alpha=1)
    outs = {}
    for pack in ("dp_shift", "dp_shift_ext"):
        lay = ffconv.Layout(1, 6, 6, 3, 2, 1, 2, 3, pack=pack)
        outs[pack] = run_he(prm, lay, seed=5)
    a, b = outs["dp_shift"][3], outs["dp_shift_ext"][3]
    s = outs["dp_shift"][1]
    assert not (a[0].stack() == b[0].stack()).all()
    for x, y in zip(a, b):
        assert (bfv.decrypt(prm, s, x) == bfv.decrypt(prm, s, y)).all()


def test_conv_pack_counts_follow_table_ii():
    """Table II, FFConv row: MulPC = O'_c (K + O_c) for the factorized pair under ConvPack,
    here at the TinyNet layer of Table VI (8 x 8 stride-2 conv, 13 low-rank channels, 56
    restored channels, 144 output positions, K = 64)."""
    lay = ffconv.Layout(1, 28, 28, 8, 2, 1, 13, 56, pack="cp_cp")
    assert (lay.S, lay.d * lay.d * lay.I_c) == (144, 64)
    ops = ffconv.expected_ops(lay, 8192)
    assert ops["mulpc"] == 13 * (64 + 56) and ops["rot"] == 0


@pytest.mark.parametrize("slip", ["combine_sign", "short_sum"])
def test_planted_dp_dp_slips_are_caught(monkeypatch, slip):
    """DP-DP: combining the channels with the wrong rotation direction, or stopping W2's
    rotate-and-sum one step short of (r - 1) S, breaks the decryption pin."""
    prm = params.Params(log_n=7, n_q=3, n_p=1, alpha=1)
    lay = ffconv.Layout(2, 5, 5, 3, 1, 1, 2, 2, pack="dp_dp")
    if slip == "combine_sign":
        monkeypatch.setattr(ffconv, "dp_dp_combine_steps", lambda l: [c * l.S for c in range(1, l.r)])
    else:
        real = ffconv.dp_dp_sum_steps
        monkeypatch.setattr(ffconv, "dp_dp_sum_steps", lambda l: real(l)[:-1])
    prm, s, lay, outs, y2, ops = run_he(prm, lay, seed=2)
    with pytest.raises(AssertionError):
        check_outputs(prm, s, lay, outs, y2)
