"""GPU parity of the three-layer network (FFConv layer, channel combine, x^2, fully connected,
x^2, fully connected) and of its new steps against the CPU oracle (oracle/network.py).

Small ring (N = 2048, 4 primes): every step and the whole network bit for bit with the
oracle's keys.  The network's own ring (N = 2^14, 6 primes, the 1x28x28 -> 5x5 s2 (r=2) -> 5
channels -> 100 -> 10 shape): decryption of the batched network equals the plain network
mod t for every image, with the keys generated on the GPU."""
import numpy as np
import pytest

from oracle import bfv, encoder, network, params
from oracle.ffconv import Layout, input_slots
from tests.gpu_common import download_coeff, encrypt_slots, gpu_steps, make_ctx, upload_ntt

pytestmark = pytest.mark.gpu

SMALL = Layout(1, 12, 12, 3, 2, 1, 2, 3, pack="dp_shift_ext")
M1, M2 = 20, 4


def gpu_layout(ctx, lay):
    return ctx.layout(lay.I_c, lay.I_h, lay.I_w, lay.d, lay.stride, lay.pad, lay.r, lay.O_c,
                      pack=lay.pack, modswitch=lay.modswitch)


def rand_net(lay, m1, m2, seed):
    rng = np.random.default_rng(seed)
    return (rng.integers(0, 256, (lay.I_c, lay.I_h, lay.I_w)),
            rng.integers(-8, 9, (lay.r, lay.I_c, lay.d, lay.d)),
            rng.integers(-8, 9, (lay.O_c, lay.r)),
            rng.integers(-8, 9, (m1, lay.O_c * lay.S)),
            rng.integers(-8, 9, (m2, m1)))


@pytest.fixture(scope="module")
def small():
    from paper_2102_03494_gb300 import he
    prm = params.Params(log_n=11, n_q=4, n_p=2, alpha=2)
    ctx = make_ctx(prm)
    s = bfv.keygen_secret(prm, 1)
    steps = network.net_steps(SMALL, M1, M2, prm.n)
    steps += [st for st in network.fc_steps(100, prm.n // 2) if st not in steps]
    keys, blob = {}, []
    for st in steps:
        g = bfv.galois_of(st, prm.n)
        if g not in keys:
            keys[g] = bfv.galois_key(prm, s, g, 2)
        blob.append(keys[g].reshape(-1))           # one key per listed step
    rlk = bfv.relin_key(prm, s, 2)
    ctx.he_load_keys(np.concatenate(blob + [rlk.reshape(-1)]),
                     gpu_steps(steps) + [he.HE_RELIN_KEY])
    return prm, ctx, s, keys, rlk


def test_multiply_batch_is_bit_exact(small):
    prm, ctx, s, keys, rlk = small
    rng = np.random.default_rng(1)
    a = [encrypt_slots(prm, s, rng.integers(0, prm.t, prm.n), 10 + i) for i in range(3)]
    b = [encrypt_slots(prm, s, rng.integers(0, prm.t, prm.n), 20 + i) for i in range(3)]
    da = [upload_ntt(ctx, c) for c in a]
    db = [upload_ntt(ctx, c) for c in b]
    got = ctx.he_multiply_batch(da, db)
    for i in range(3):
        want = bfv.relinearize(prm, bfv.multiply(prm, a[i], b[i]), rlk)
        assert (download_coeff(ctx, got[i]) == want.stack()).all(), i
    sq = ctx.he_multiply_batch(da, da)
    for i in range(3):
        want = bfv.relinearize(prm, bfv.multiply(prm, a[i], a[i]), rlk)
        assert (download_coeff(ctx, sq[i]) == want.stack()).all(), i


@pytest.mark.parametrize("m,n_in,per,spread", [(20, 108, 1024, True), (4, 20, 32, False),
                                               (100, 300, 1024, True), (1, 7, 8, False)])
@pytest.mark.parametrize("arith", [0, 2], ids=["chains", "products"])
def test_fc_layer_is_bit_exact(small, m, n_in, per, spread, arith):
    """spread: sparse positions over a whole row (period N/2); else dense, repeating."""
    prm, ctx, s, keys, rlk = small
    from paper_2102_03494_gb300 import he as _he
    ctx.he_tune_set(_he.HE_TUNE_TAP_ARITH, arith)   # the tap kernel's arithmetic (same bits)
    half = prm.n // 2
    rng = np.random.default_rng(m + n_in)
    pos = (sorted(rng.choice(per, size=n_in, replace=False).tolist()) if spread
           else list(range(n_in)))
    F = rng.integers(-8, 9, (m, n_in))
    cts, xs = [], []
    for b in range(2):
        xv = rng.integers(0, prm.t, n_in)
        v = np.zeros(prm.n, dtype=np.int64)
        for rep in range(half // per):
            for i, p in enumerate(pos):
                v[rep * per + p] = xv[i]
        cts.append(encrypt_slots(prm, s, v, 30 + b))
        xs.append(xv)
    got = ctx.he_fc_layer_batch([upload_ntt(ctx, c) for c in cts], F, pos, per)
    M = network.next_pow2(m)
    for b in range(2):
        want = network.he_fc(prm, cts[b], F, pos, per, keys)
        assert (download_coeff(ctx, got[b]) == want.stack()).all(), b
        y = (F.astype(object) @ xs[b].astype(object)) % prm.t
        dec = ctx.he_decrypt(s, got[b])
        for p in range(half):
            assert dec[p] == (y[p % M] if p % M < m else 0)


def test_combine_is_bit_exact(small):
    prm, ctx, s, keys, rlk = small
    rng = np.random.default_rng(5)
    blk = network.combine_block(SMALL)
    cts = [encrypt_slots(prm, s, np.pad(rng.integers(0, prm.t, blk), (0, prm.n - blk)), 40 + i)
           for i in range(2 * SMALL.O_c)]
    got = ctx.he_combine_batch([upload_ntt(ctx, c) for c in cts], SMALL.O_c, blk)
    for b in range(2):
        want = network.he_combine(prm, cts[b * SMALL.O_c:(b + 1) * SMALL.O_c], blk, keys)
        assert (download_coeff(ctx, got[b]) == want.stack()).all(), b


@pytest.mark.parametrize("arith", [0, 2], ids=["chains", "products"])
def test_network_is_bit_exact(small, arith):
    prm, ctx, s, keys, rlk = small
    from paper_2102_03494_gb300 import he as _he
    ctx.he_tune_set(_he.HE_TUNE_TAP_ARITH, arith)   # the tap kernel's arithmetic (same bits)
    imgs, cts = [], []
    for b in range(2):
        x, W1, W2, F1, F2 = rand_net(SMALL, M1, M2, seed=7)      # shared weights
        x = np.random.default_rng(100 + b).integers(0, 256, x.shape)
        imgs.append(x)
        cts.append(encrypt_slots(prm, s, input_slots(x, SMALL, prm.n), 50 + b))
    net = ctx.net(gpu_layout(ctx, SMALL), M1, M2)
    want_steps = network.net_steps(SMALL, M1, M2, prm.n)
    from paper_2102_03494_gb300 import he
    got_steps = ctx.he_net_required_steps(net)
    assert got_steps[-1] == he.HE_RELIN_KEY
    assert sorted(gpu_steps(want_steps)) == sorted(got_steps[:-1])
    outs = ctx.he_net_batch([upload_ntt(ctx, c) for c in cts], W1, W2, F1, F2, net)
    M2p = network.next_pow2(M2)
    for b in range(2):
        want = network.he_net(prm, cts[b], W1, W2, SMALL, F1, F2, keys, rlk)
        assert (download_coeff(ctx, outs[b]) == want.stack()).all(), b
        _, _, z2 = network.plain_net(imgs[b], W1, W2, SMALL, F1, F2, prm.t)
        dec = ctx.he_decrypt(s, outs[b])
        for p in network.output_slots(M2, prm.n):
            assert dec[p] == z2[p % M2p]


def test_network_errors(small):
    from paper_2102_03494_gb300 import he
    prm, ctx, s, keys, rlk = small
    d = upload_ntt(ctx, encrypt_slots(prm, s, np.zeros(prm.n, np.int64), 1))
    with pytest.raises(he.HeError) as e:
        ctx.he_fc_layer_batch([d], np.ones((5, 3)), [0, 1, 2], 4)        # M = 8 > period
    assert e.value.code == he.HE_EINVAL
    with pytest.raises(he.HeError) as e:
        ctx.he_fc_layer_batch([d], np.ones((2, 3)), [0, 1, 1], 16)       # repeated position
    assert e.value.code == he.HE_EINVAL
    big = Layout(1, 12, 12, 3, 2, 1, 2, 9, pack="dp_shift_ext")         # 9 x 256 > 1024 slots
    with pytest.raises(he.HeError):
        ctx.he_net_required_steps(ctx.net(gpu_layout(ctx, big), 4, 2))


def test_mnist_network_n14_decrypts_to_plain():
    """The network's own ring and shape, batch 4, keys generated on the GPU."""
    from paper_2102_03494_gb300 import he
    prm = params.Params(log_n=14, n_q=6, n_p=2, alpha=2)
    ctx = make_ctx(prm)
    lay = Layout(1, 28, 28, 5, 2, 1, 2, 5, pack="dp_shift_ext")
    m1, m2 = 100, 10
    s = bfv.keygen_secret(prm, 3)
    net = ctx.net(gpu_layout(ctx, lay), m1, m2)
    ctx.he_keygen_galois(s, 4, ctx.he_net_required_steps(net))
    rng = np.random.default_rng(0)
    W1 = rng.integers(-8, 9, (2, 1, 5, 5))
    W2 = rng.integers(-8, 9, (5, 2))
    F1 = rng.integers(-8, 9, (m1, 845))
    F2 = rng.integers(-8, 9, (m2, m1))
    imgs = [rng.integers(0, 256, (1, 28, 28)) for _ in range(4)]
    cts = [ctx.he_encrypt(s, input_slots(x, lay, prm.n), 60 + b) for b, x in enumerate(imgs)]
    outs = ctx.he_net_batch(cts, W1, W2, F1, F2, net)
    for b in range(4):
        _, _, z2 = network.plain_net(imgs[b], W1, W2, lay, F1, F2, prm.t)
        dec = ctx.he_decrypt(s, outs[b])
        assert (dec[:16][:m2] == z2).all(), b
        assert not dec[m2:16].any()
        assert (dec[: prm.n // 2].reshape(-1, 16)[:, :m2] == z2).all()


def test_recorded_network_replays_bit_exact(small):
    """The whole network recorded as a CUDA graph (he_graph_begin .. he_graph_end) gives, at
    every replay, the bits of the plain call on whatever the bound inputs hold; a refused call
    spoils a recording; a graph stops replaying once the network buffer is reallocated."""
    from paper_2102_03494_gb300 import he
    prm, ctx, s, keys, rlk = small
    _, W1, W2, F1, F2 = rand_net(SMALL, M1, M2, seed=7)
    net = ctx.net(gpu_layout(ctx, SMALL), M1, M2)
    cts = [encrypt_slots(prm, s, input_slots(np.random.default_rng(200 + b).integers(0, 256, (1, 12, 12)),
                                             SMALL, prm.n), 70 + b) for b in range(2)]
    ins = [upload_ntt(ctx, c) for c in cts]
    outs = [ctx.new_ct() for _ in range(2)]
    ctx.he_net_batch(ins, W1, W2, F1, F2, net, outs)          # sizes scratch and network buffer
    want = [download_coeff(ctx, o) for o in outs]
    assert (want[0] == network.he_net(prm, cts[0], W1, W2, SMALL, F1, F2, keys, rlk).stack()).all()
    ctx.he_graph_begin(share_scratch=True)
    ctx.he_net_batch(ins, W1, W2, F1, F2, net, outs)
    with pytest.raises(he.HeError):
        ctx.he_decrypt(s, outs[0])                            # refused while recording
    with pytest.raises(he.HeError):
        ctx.he_graph_end()                                    # ... which spoiled the recording
    graphs = []
    for share in (True, False):
        ctx.he_graph_begin(share_scratch=share)
        ctx.he_net_batch(ins, W1, W2, F1, F2, net, outs)
        graphs.append(ctx.he_graph_end(keep=ins + outs))
    for gid in graphs:
        for o in outs:
            o.zero_()
        ctx.he_graph_launch(gid)
        for b in range(2):
            assert (download_coeff(ctx, outs[b]) == want[b]).all(), (gid, b)
    a, b = ins[0].clone(), ins[1].clone()
    ins[0].copy_(b)
    ins[1].copy_(a)
    ctx.he_graph_launch(graphs[1])
    assert (download_coeff(ctx, outs[0]) == want[1]).all() and (download_coeff(ctx, outs[1]) == want[0]).all()
    ctx.he_net_batch(ins * 4, W1, W2, F1, F2, net)            # a larger batch regrows the buffers
    for gid in graphs:
        with pytest.raises(he.HeError):
            ctx.he_graph_launch(gid)
        ctx.he_graph_free(gid)
