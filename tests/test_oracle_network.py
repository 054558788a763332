"""Pins of the oracle's three-layer network (oracle/network.py) against what the mathematics
fixes: a brute-force plain network, the diagonal identity of the fully connected schedule on
plain slot vectors, the rotation counts of the combine step (Table VIII: one rotation per
channel but the first) and decryption of every encrypted step on a small ring."""
import numpy as np
import pytest

from oracle import bfv, encoder, network, params
from oracle.ffconv import Layout, OpCount, input_slots, output_slot
from tests.gpu_common import oracle_keys

SMALL = Layout(1, 12, 12, 3, 2, 1, 2, 3, pack="dp_shift_ext")


def brute_net(x, W1, W2, lay, F1, F2, t):
    """Direct loops: conv (cross-correlation, zero padding), 1x1 restore, square, fc, square,
    fc, all over Python integers."""
    y = [[[0] * lay.O_w for _ in range(lay.O_h)] for _ in range(lay.O_c)]
    for c in range(lay.O_c):
        for oh in range(lay.O_h):
            for ow in range(lay.O_w):
                acc = 0
                for cp in range(lay.r):
                    s = 0
                    for ci in range(lay.I_c):
                        for i in range(lay.d):
                            for j in range(lay.d):
                                h = lay.stride * oh + i - lay.pad
                                w = lay.stride * ow + j - lay.pad
                                if 0 <= h < lay.I_h and 0 <= w < lay.I_w:
                                    s += int(W1[cp][ci][i][j]) * int(x[ci][h][w])
                    acc += int(W2[c][cp]) * s
                y[c][oh][ow] = acc
    a1 = [v * v for ch in y for row in ch for v in row]
    z1 = [sum(int(F1[j][i]) * a1[i] for i in range(len(a1))) for j in range(len(F1))]
    a2 = [v * v for v in z1]
    z2 = [sum(int(F2[j][i]) * a2[i] for i in range(len(a2))) for j in range(len(F2))]
    return [v % t for v in a1], [v % t for v in z1], [v % t for v in z2]


def rand_net(lay, m1, m2, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 256, (lay.I_c, lay.I_h, lay.I_w))
    W1 = rng.integers(-8, 9, (lay.r, lay.I_c, lay.d, lay.d))
    W2 = rng.integers(-8, 9, (lay.O_c, lay.r))
    F1 = rng.integers(-8, 9, (m1, lay.O_c * lay.S))
    F2 = rng.integers(-8, 9, (m2, m1))
    return x, W1, W2, F1, F2


def test_plain_net_matches_brute_force():
    x, W1, W2, F1, F2 = rand_net(SMALL, 20, 4)
    got = network.plain_net(x, W1, W2, SMALL, F1, F2, 65537)
    want = brute_net(x, W1, W2, SMALL, F1, F2, 65537)
    for g, w in zip(got, want):
        assert list(g) == w


def rot(v, k, half):
    """Plain slot rotation (left by k inside each row of `half` slots)."""
    return np.concatenate([np.roll(v[:half], -k), np.roll(v[half:], -k)])


@pytest.mark.parametrize("m,n_in,per,n", [(20, 108, 512, 1024), (4, 20, 32, 1024),
                                          (10, 100, 128, 2048), (3, 4, 4, 64), (1, 5, 8, 64)])
def test_fc_diagonals_compute_the_matrix_product(m, n_in, per, n):
    half = n // 2
    rng = np.random.default_rng(m * 1000 + n_in)
    pos = sorted(rng.choice(per, size=n_in, replace=False).tolist()) if n_in <= per else None
    F = rng.integers(-8, 9, (m, n_in))
    xv = rng.integers(-50, 50, n_in)
    x = np.zeros(n, dtype=np.int64)
    for rep in range(half // per):          # the input repeats with period `per` in row 0
        for i, p in enumerate(pos):
            x[rep * per + p] = xv[i]
    diags = network.fc_diagonals(F, pos, per, n)
    M = network.next_pow2(m)
    assert len(diags) == M
    z = sum(rot(x, k, half) * diags[k] for k in range(M))
    for st in network.fc_sum_steps(m, per):
        z = z + rot(z, st, half)
    y = F @ xv
    for p in range(half):
        assert z[p] == (y[p % M] if p % M < m else 0), p
    assert not z[half:].any()
    assert len(network.fc_steps(m, per)) == (M - 1) + (per // M).bit_length() - 1


def test_fc_diagonals_reject_bad_layouts():
    F = np.ones((5, 3), dtype=np.int64)
    with pytest.raises(ValueError):
        network.fc_diagonals(F, [0, 1, 2], 4, 64)        # M = 8 > period
    with pytest.raises(ValueError):
        network.fc_diagonals(F, [0, 1, 1], 16, 64)       # repeated position
    with pytest.raises(ValueError):
        network.fc_diagonals(F, [0, 1, 2], 12, 64)       # not a power of two


def test_combined_positions_and_block():
    lay = Layout(1, 28, 28, 5, 2, 1, 2, 5, pack="dp_shift_ext")
    assert network.combine_block(lay) == 1024            # last output slot 24*28 + 24 = 696
    pos = network.combined_positions(lay)
    assert len(pos) == 845 and len(set(pos)) == 845
    assert pos[169] == 1024 and pos[-1] == 4 * 1024 + output_slot(lay, 12, 12)


@pytest.fixture(scope="module")
def small_setup():
    prm = params.Params(log_n=11, n_q=4, n_p=2, alpha=2)
    m1, m2 = 20, 4
    s = bfv.keygen_secret(prm, 1)
    keys, _ = oracle_keys(prm, s, network.net_steps(SMALL, m1, m2, prm.n))
    rlk = bfv.relin_key(prm, s, 2)
    return prm, s, keys, rlk, m1, m2


def dec_slots(prm, s, ct):
    return encoder.decode(bfv.decrypt(prm, s, ct), prm)


def test_encrypted_steps_decrypt(small_setup):
    from oracle.ffconv import he_layer
    prm, s, keys, rlk, m1, m2 = small_setup
    x, W1, W2, F1, F2 = rand_net(SMALL, m1, m2, seed=3)
    a1, z1, z2 = brute_net(x, W1, W2, SMALL, F1, F2, prm.t)
    ct = bfv.encrypt(prm, s, encoder.encode(input_slots(x, SMALL, prm.n), prm), 5)
    ops = OpCount()
    cts = he_layer(prm, ct, W1, W2, SMALL, keys)
    comb = network.he_combine(prm, cts, network.combine_block(SMALL), keys, ops)
    assert ops.rot == SMALL.O_c - 1                      # Table VIII: O_c - 1 rotations
    _, y2 = network.plain_layer(x, W1, W2, SMALL)
    want = np.zeros(prm.n, dtype=np.int64)
    for i, p in enumerate(network.combined_positions(SMALL)):
        want[p] = int(np.asarray(y2).reshape(-1)[i]) % prm.t
    assert (dec_slots(prm, s, comb) == want).all()
    sq = network.he_square(prm, comb, rlk)
    want_sq = np.zeros(prm.n, dtype=np.int64)
    for i, p in enumerate(network.combined_positions(SMALL)):
        want_sq[p] = a1[i]
    assert (dec_slots(prm, s, sq) == want_sq).all()
    ops = OpCount()
    f1 = network.he_fc(prm, sq, F1, network.combined_positions(SMALL), prm.n // 2, keys, ops)
    assert ops.rot == len(network.fc_steps(m1, prm.n // 2))
    got = dec_slots(prm, s, f1)
    M1 = network.next_pow2(m1)
    for p in range(prm.n // 2):
        assert got[p] == (z1[p % M1] if p % M1 < m1 else 0)
    assert not got[prm.n // 2:].any()


def test_network_decrypts_to_plain(small_setup):
    prm, s, keys, rlk, m1, m2 = small_setup
    x, W1, W2, F1, F2 = rand_net(SMALL, m1, m2, seed=4)
    _, _, z2 = network.plain_net(x, W1, W2, SMALL, F1, F2, prm.t)
    ct = bfv.encrypt(prm, s, encoder.encode(input_slots(x, SMALL, prm.n), prm), 6)
    out = network.he_net(prm, ct, W1, W2, SMALL, F1, F2, keys, rlk)
    got = dec_slots(prm, s, out)
    M2 = network.next_pow2(m2)
    want = np.zeros(prm.n, dtype=np.int64)
    for p in network.output_slots(m2, prm.n):
        want[p] = z2[p % M2]
    assert (got == want).all()
    used, left = bfv.noise_bits(prm, s, out, encoder.encode(want, prm))
    assert left > 10


def test_planted_mistake_in_fc_is_caught(small_setup, monkeypatch):
    """A diagonal off by one slot must break the fc decryption."""
    prm, s, keys, rlk, m1, m2 = small_setup
    orig = network.fc_diagonals

    def shifted(F, pos, per, n):
        d = orig(F, pos, per, n)
        return [np.roll(v, 1) for v in d]

    rng = np.random.default_rng(8)
    F = rng.integers(-8, 9, (4, 20))
    xv = rng.integers(0, 100, 20)
    v = np.zeros(prm.n, dtype=np.int64)
    for rep in range(prm.n // 2 // 32):     # an input repeating with period 32 in row 0
        v[rep * 32: rep * 32 + 20] = xv
    ct = bfv.encrypt(prm, s, encoder.encode(v, prm), 9)
    ok = dec_slots(prm, s, network.he_fc(prm, ct, F, list(range(20)), 32, keys))
    assert (ok[:4] == (F @ xv) % prm.t).all()
    monkeypatch.setattr(network, "fc_diagonals", shifted)
    bad = dec_slots(prm, s, network.he_fc(prm, ct, F, list(range(20)), 32, keys))
    assert not (bad[:4] == (F @ xv) % prm.t).all()
