"""Pins of the oracle's deeper network over several ciphertexts per tensor (oracle/deepnet.py):
the plain network against PyTorch's conv2d and brute-force loops, the tensor layout, every
encrypted step decrypting to the plain result on a small ring (factorized and unfactorized
layers, one and two input ciphertexts), the rotation counts, and a planted mistake."""
import numpy as np
import pytest
import torch

from oracle import bfv, deepnet, encoder, params
from oracle.ffconv import OpCount
from tests.gpu_common import oracle_keys

SHAPE = deepnet.DeepShape(3, 8, 8, [deepnet.ConvSpec(20, 4), deepnet.ConvSpec(24, None)], n_cls=4)


def test_conv_same_matches_torch():
    rng = np.random.default_rng(0)
    x = rng.integers(0, 256, (5, 7, 9))
    W = rng.integers(-8, 9, (6, 5, 3, 3))
    t = 65537
    want = torch.nn.functional.conv2d(torch.tensor(x, dtype=torch.float64)[None],
                                      torch.tensor(W, dtype=torch.float64), padding=1)[0]
    got = deepnet.conv_same(x, W, 3, 1, t)
    assert (got == (want.numpy().astype(np.int64) % t)).all()


def test_plain_deep_matches_brute_force():
    t = 65537
    shape = deepnet.DeepShape(2, 4, 4, [deepnet.ConvSpec(3, 2), deepnet.ConvSpec(2, None)], n_cls=3)
    w = deepnet.rand_weights(shape, 5)
    x = np.random.default_rng(6).integers(0, 256, (2, 4, 4))
    h = [[[int(x[c][i][j]) for j in range(4)] for i in range(4)] for c in range(2)]
    for spec, (W1, W2) in zip(shape.convs, w["convs"]):
        C = len(h)
        r = len(W1)
        y = [[[sum(int(W1[o][c][i][j]) * h[c][a + i - 1][b + j - 1]
                   for c in range(C) for i in range(3) for j in range(3)
                   if 0 <= a + i - 1 < 4 and 0 <= b + j - 1 < 4)
               for b in range(4)] for a in range(4)] for o in range(r)]
        if W2 is not None:
            y = [[[sum(int(W2[o][k]) * y[k][a][b] for k in range(r)) for b in range(4)]
                  for a in range(4)] for o in range(spec.O_c)]
        h = [[[v * v for v in row] for row in ch] for ch in y]
    pooled = [sum(sum(row) for row in ch) for ch in h]
    logits = [sum(int(w["fc"][j][c]) * pooled[c] for c in range(len(pooled))) % t for j in range(3)]
    acts, got = deepnet.plain_deep(x, w, shape, t)
    assert list(got) == logits
    assert (acts[-1] == np.array([[[v % t for v in row] for row in ch] for ch in h])).all()


def test_pack_tensor_layout():
    shape = deepnet.DeepShape(20, 5, 6, [], n_cls=1)            # 30 pixels -> blocks of 32
    n = 1024                                                     # 512 slots: 16 blocks
    x = np.arange(20 * 30).reshape(20, 5, 6)
    cts = deepnet.pack_tensor(x, shape, n)
    assert len(cts) == 2
    assert cts[0][0:30].tolist() == list(range(30)) and cts[0][30:32].tolist() == [0, 0]
    assert cts[1][3 * 32 + 7] == x[19].reshape(-1)[7]
    assert not cts[1][4 * 32:].any()


@pytest.fixture(scope="module")
def ring():
    prm = params.Params(log_n=11, n_q=5, n_p=2, alpha=2)
    s = bfv.keygen_secret(prm, 1)
    keys, _ = oracle_keys(prm, s, deepnet.deep_steps(SHAPE, prm.n) + deepnet.pool_steps(SHAPE))
    rlk = bfv.relin_key(prm, s, 2)
    return prm, s, keys, rlk


def dec(prm, s, ct):
    return encoder.decode(bfv.decrypt(prm, s, ct), prm)


def check_tensor(prm, s, cts, y, shape):
    g = deepnet.per_ct(shape, prm.n)
    hw = shape.H * shape.W
    for c in range(y.shape[0]):
        d = dec(prm, s, cts[c // g])
        assert (d[(c % g) * shape.Bk:(c % g) * shape.Bk + hw] == y[c].reshape(-1)).all(), c
    for G, ct in enumerate(cts):                 # every other slot zero
        d = dec(prm, s, ct)
        used = np.zeros(prm.n, dtype=bool)
        for c in range(G * g, min(y.shape[0], (G + 1) * g)):
            used[(c % g) * shape.Bk:(c % g) * shape.Bk + hw] = True
        assert not d[~used].any()


def test_encrypted_layers_decrypt_to_plain(ring):
    prm, s, keys, rlk = ring
    t = prm.t
    w = deepnet.rand_weights(SHAPE, 7)
    x = np.random.default_rng(8).integers(0, 256, (3, 8, 8))
    cts = [bfv.encrypt(prm, s, encoder.encode(v, prm), 10 + i)
           for i, v in enumerate(deepnet.pack_tensor(x, SHAPE, prm.n))]
    h = x % t
    C = SHAPE.C0
    for spec, (W1, W2) in zip(SHAPE.convs, w["convs"]):
        ops = OpCount()
        y_ct = deepnet.he_conv(prm, cts, W1, W2, spec, C, SHAPE, keys, ops)
        y = deepnet.conv_same(h, W1, 3, 1, t)
        if W2 is not None:
            y = np.tensordot(np.asarray(W2) % t, y, axes=([1], [0])) % t
        check_tensor(prm, s, y_ct, y, SHAPE)
        r = spec.O_c if spec.r is None else spec.r
        assert ops.rot == len(cts) * 8 + r * len(deepnet.fold_steps(SHAPE, prm.n))
        cts = [bfv.relinearize(prm, bfv.multiply(prm, c, c), rlk) for c in y_ct]
        h = (y * y) % t
        check_tensor(prm, s, cts, h, SHAPE)
        C = spec.O_c


def test_pooling_folded_into_the_classifier(ring):
    """The classifier over all activations with repeated weights equals sum pooling followed
    by the classifier over the pooled sums (both decrypted)."""
    prm, s, keys, rlk = ring
    rng = np.random.default_rng(13)
    C = 20
    a = rng.integers(0, prm.t, (C, 8, 8))
    cts = [bfv.encrypt(prm, s, encoder.encode(v, prm), 40 + i)
           for i, v in enumerate(deepnet.pack_tensor(a, SHAPE, prm.n))]
    F = rng.integers(-8, 9, (SHAPE.n_cls, C))
    Fx, ct_of, pos = deepnet.pooled_fc_features(F, C, SHAPE, prm.n)
    merged = dec(prm, s, deepnet.he_fc_multi(prm, cts, Fx, ct_of, pos, keys))
    pooled = [deepnet.he_pool(prm, c, SHAPE, keys) for c in cts]
    feats = deepnet.fc_inputs(C, SHAPE, prm.n)
    two = dec(prm, s, deepnet.he_fc_multi(prm, pooled, F, [G for G, _ in feats],
                                          [p for _, p in feats], keys))
    want = (F.astype(object) @ a.reshape(C, -1).sum(axis=1).astype(object)) % prm.t
    M = deepnet.next_pow2(SHAPE.n_cls)
    assert (merged[:M][:SHAPE.n_cls] == want).all() and (two[:M][:SHAPE.n_cls] == want).all()


def test_network_decrypts_to_plain_and_counts(ring):
    prm, s, keys, rlk = ring
    w = deepnet.rand_weights(SHAPE, 9)
    x = np.random.default_rng(10).integers(0, 256, (3, 8, 8))
    cts = [bfv.encrypt(prm, s, encoder.encode(v, prm), 20 + i)
           for i, v in enumerate(deepnet.pack_tensor(x, SHAPE, prm.n))]
    ops = OpCount()
    out = deepnet.he_deep(prm, cts, w, SHAPE, keys, rlk, ops)
    _, logits = deepnet.plain_deep(x, w, SHAPE, prm.t)
    d = dec(prm, s, out)
    M = deepnet.next_pow2(SHAPE.n_cls)
    for p in range(prm.n // 2):
        assert d[p] == (logits[p % M] if p % M < SHAPE.n_cls else 0)
    assert ops.rot == deepnet.expected_rotations(SHAPE, prm.n)


def test_factorized_needs_fewer_rotations():
    """Table I: DensePack rotations grow with the output channels; the factorized layer folds
    r channels instead of O_c."""
    n = 2 ** 15
    fac = deepnet.DeepShape(3, 32, 32, [deepnet.ConvSpec(64, 8), deepnet.ConvSpec(64, 8),
                                        deepnet.ConvSpec(128, 8)])
    unf = deepnet.DeepShape(3, 32, 32, [deepnet.ConvSpec(64, None), deepnet.ConvSpec(64, None),
                                        deepnet.ConvSpec(128, None)])
    rf, ru = deepnet.expected_rotations(fac, n), deepnet.expected_rotations(unf, n)
    # taps: 8 (1 ct) + 32 + 32 (4 cts); block sums 15 hoisted per channel; pooling folded
    # into the classifier: 8 x 15 + 10
    assert rf == 8 + 32 + 32 + 15 * (8 + 8 + 8) + 130
    assert ru == 8 + 32 + 32 + 15 * (64 + 64 + 128) + 130


def test_planted_restore_block_slip_is_caught(ring, monkeypatch):
    prm, s, keys, rlk = ring
    w = deepnet.rand_weights(SHAPE, 11)
    x = np.random.default_rng(12).integers(0, 256, (3, 8, 8))
    cts = [bfv.encrypt(prm, s, encoder.encode(v, prm), 30 + i)
           for i, v in enumerate(deepnet.pack_tensor(x, SHAPE, prm.n))]
    spec = SHAPE.convs[0]
    W1, W2 = w["convs"][0]
    real = deepnet.restore_slots
    monkeypatch.setattr(deepnet, "restore_slots",
                        lambda W2_, sh, n, G, c, O_c: np.roll(real(W2_, sh, n, G, c, O_c), sh.Bk))
    y_ct = deepnet.he_conv(prm, cts, W1, W2, spec, 3, SHAPE, keys)
    y = np.tensordot(np.asarray(W2) % prm.t, deepnet.conv_same(x, W1, 3, 1, prm.t),
                     axes=([1], [0])) % prm.t
    with pytest.raises(AssertionError):
        check_tensor(prm, s, y_ct, y, SHAPE)
