"""GPU parity of the deeper network over several ciphertexts per tensor against the CPU oracle
(oracle/deepnet.py): the layer (factorized, one input ciphertext; unfactorized, two), the
in-block rotate-and-sum, the classifier over several ciphertexts and the whole network bit
for bit on a small ring with the oracle's keys; at N = 2^15 with 12 + 3 primes the 3x32x32
network (64, 64, 128 channels at rank 8) decrypts to the plain network mod t."""
import numpy as np
import pytest

from oracle import bfv, deepnet, encoder, params
from tests.gpu_common import download_coeff, encrypt_slots, gpu_steps, make_ctx, upload_ntt

pytestmark = pytest.mark.gpu

SHAPE = deepnet.DeepShape(3, 8, 8, [deepnet.ConvSpec(20, 4), deepnet.ConvSpec(24, None)], n_cls=4)


def gpu_convs(ctx, shape):
    out, C = [], shape.C0
    for spec in shape.convs:
        out.append(ctx.mc_conv(C, shape.H, shape.W, spec.d, spec.r, spec.O_c))
        C = spec.O_c
    return out


def w32(w):
    return None if w is None else np.asarray(w, dtype=np.int32)


@pytest.fixture(scope="module")
def small():
    from paper_2102_03494_gb300 import he
    prm = params.Params(log_n=11, n_q=5, n_p=2, alpha=2)
    ctx = make_ctx(prm)
    s = bfv.keygen_secret(prm, 1)
    steps = deepnet.deep_steps(SHAPE, prm.n)
    steps += [st for st in deepnet.pool_steps(SHAPE) if st not in steps]
    keys, blob = {}, []
    for st in steps:
        g = bfv.galois_of(st, prm.n)
        if g not in keys:
            keys[g] = bfv.galois_key(prm, s, g, 2)
        blob.append(keys[g].reshape(-1))
    rlk = bfv.relin_key(prm, s, 2)
    ctx.he_load_keys(np.concatenate(blob + [rlk.reshape(-1)]), gpu_steps(steps) + [he.HE_RELIN_KEY])
    return prm, ctx, s, keys, rlk


def encrypt_tensor(prm, s, x, shape, seed):
    return [encrypt_slots(prm, s, v, seed + i) for i, v in enumerate(deepnet.pack_tensor(x, shape, prm.n))]


@pytest.mark.parametrize("arith", [0, 2], ids=["chains", "products"])
def test_layers_are_bit_exact(small, arith):
    prm, ctx, s, keys, rlk = small
    from paper_2102_03494_gb300 import he as _he
    ctx.he_tune_set(_he.HE_TUNE_TAP_ARITH, arith)   # the tap kernel's arithmetic (same bits)
    w = deepnet.rand_weights(SHAPE, 3)
    convs = gpu_convs(ctx, SHAPE)
    rng = np.random.default_rng(4)
    # layer 1 (factorized, one input ciphertext per image), two images
    xs = [rng.integers(0, 256, (3, 8, 8)) for _ in range(2)]
    cts = [encrypt_tensor(prm, s, x, SHAPE, 10 * b) for b, x in enumerate(xs)]
    W1, W2 = w["convs"][0]
    got = ctx.he_mc_conv_batch([upload_ntt(ctx, c) for img in cts for c in img], w32(W1), w32(W2),
                               convs[0])
    n_out = len(got) // 2
    for b in range(2):
        want = deepnet.he_conv(prm, cts[b], W1, W2, SHAPE.convs[0], 3, SHAPE, keys)
        for G in range(n_out):
            assert (download_coeff(ctx, got[b * n_out + G]) == want[G].stack()).all(), (b, G)
    # layer 2 (unfactorized, two input ciphertexts per image) on random 20-channel tensors
    ys = [rng.integers(0, prm.t, (20, 8, 8)) for _ in range(2)]
    cts = [encrypt_tensor(prm, s, y, SHAPE, 100 + 10 * b) for b, y in enumerate(ys)]
    W1, W2 = w["convs"][1]
    assert W2 is None
    got = ctx.he_mc_conv_batch([upload_ntt(ctx, c) for img in cts for c in img], w32(W1), None,
                               convs[1])
    n_out = len(got) // 2
    for b in range(2):
        want = deepnet.he_conv(prm, cts[b], W1, None, SHAPE.convs[1], 20, SHAPE, keys)
        for G in range(n_out):
            assert (download_coeff(ctx, got[b * n_out + G]) == want[G].stack()).all(), (b, G)


def test_pool_and_classifier_are_bit_exact(small):
    prm, ctx, s, keys, rlk = small
    rng = np.random.default_rng(5)
    cts = [encrypt_slots(prm, s, rng.integers(0, prm.t, prm.n), 200 + i) for i in range(4)]
    d = [upload_ntt(ctx, c) for c in cts]
    ctx.he_rotate_sum_batch(d, deepnet.pool_steps(SHAPE))
    for i in range(4):
        want = deepnet.he_pool(prm, cts[i], SHAPE, keys)
        assert (download_coeff(ctx, d[i]) == want.stack()).all(), i
    # classifier over two pooled ciphertexts per image (24 channels), two images
    C = 24
    F = rng.integers(-8, 9, (SHAPE.n_cls, C))
    feats = deepnet.fc_inputs(C, SHAPE, prm.n)
    imgs = [[deepnet.he_pool(prm, encrypt_slots(prm, s, rng.integers(0, prm.t, prm.n), 300 + 10 * b + g),
                             SHAPE, keys) for g in range(2)] for b in range(2)]
    ct_of, pos = [G for G, _ in feats], [p for _, p in feats]
    got = ctx.he_fc_mc_batch([upload_ntt(ctx, c) for img in imgs for c in img], 2, F, ct_of, pos,
                             prm.n // 2)
    for b in range(2):
        want = deepnet.he_fc_multi(prm, imgs[b], F, ct_of, pos, keys)
        assert (download_coeff(ctx, got[b]) == want.stack()).all(), b


@pytest.mark.parametrize("arith", [0, 2], ids=["chains", "products"])
def test_network_is_bit_exact(small, arith):
    from paper_2102_03494_gb300 import he
    prm, ctx, s, keys, rlk = small
    from paper_2102_03494_gb300 import he as _he
    ctx.he_tune_set(_he.HE_TUNE_TAP_ARITH, arith)   # the tap kernel's arithmetic (same bits)
    w = deepnet.rand_weights(SHAPE, 6)
    convs = gpu_convs(ctx, SHAPE)
    steps = ctx.he_deep_required_steps(convs, SHAPE.n_cls)
    assert steps[-1] == he.HE_RELIN_KEY
    assert sorted(steps[:-1]) == sorted(deepnet.deep_steps(SHAPE, prm.n))
    # pooling is folded into the classifier: no in-block steps beyond the classifier's
    rng = np.random.default_rng(7)
    xs = [rng.integers(0, 256, (3, 8, 8)) for _ in range(2)]
    cts = [encrypt_tensor(prm, s, x, SHAPE, 400 + 10 * b) for b, x in enumerate(xs)]
    outs = ctx.he_deep_batch([upload_ntt(ctx, c) for img in cts for c in img], convs,
                             [w32(a) for a, _ in w["convs"]], [w32(b) for _, b in w["convs"]],
                             w32(w["fc"]))
    M = deepnet.next_pow2(SHAPE.n_cls)
    for b in range(2):
        want = deepnet.he_deep(prm, cts[b], w, SHAPE, keys, rlk)
        assert (download_coeff(ctx, outs[b]) == want.stack()).all(), b
        _, logits = deepnet.plain_deep(xs[b], w, SHAPE, prm.t)
        d = ctx.he_decrypt(s, outs[b])
        assert (d[:M][:SHAPE.n_cls] == logits).all()


def test_cifar_shaped_network_n15_decrypts_to_plain():
    """3 x 32 x 32 -> 64 -> 64 -> 128 channels (rank 8), x^2 after each, sum pooling, 10
    classes; N = 2^15, 12 + 3 primes, batch 2, keys generated on the GPU."""
    prm = params.cfg_n15()
    ctx = make_ctx(prm)
    shape = deepnet.DeepShape(3, 32, 32, [deepnet.ConvSpec(64, 8), deepnet.ConvSpec(64, 8),
                                          deepnet.ConvSpec(128, 8)], n_cls=10)
    convs = gpu_convs(ctx, shape)
    s = bfv.keygen_secret(prm, 5)
    ctx.he_keygen_galois(s, 6, ctx.he_deep_required_steps(convs, shape.n_cls))
    w = deepnet.rand_weights(shape, 8, lo=-4, hi=4)
    rng = np.random.default_rng(9)
    xs = [rng.integers(0, 256, (3, 32, 32)) for _ in range(2)]
    cts = [ctx.he_encrypt(s, v, 500 + 10 * b + i)
           for b, x in enumerate(xs) for i, v in enumerate(deepnet.pack_tensor(x, shape, prm.n))]
    ctx.he_reset_op_counts()
    outs = ctx.he_deep_batch(cts, convs, [w32(a) for a, _ in w["convs"]],
                             [w32(b) for _, b in w["convs"]], w32(w["fc"]))
    assert ctx.he_op_counts()["rot"] == 2 * deepnet.expected_rotations(shape, prm.n)
    M = deepnet.next_pow2(shape.n_cls)
    for b in range(2):
        _, logits = deepnet.plain_deep(xs[b], w, shape, prm.t)
        d = ctx.he_decrypt(s, outs[b])
        assert (d[: prm.n // 2].reshape(-1, M)[:, :shape.n_cls] == logits).all(), b
