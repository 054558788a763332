"""Pins for the oracle's BFV layer: exact noise of fresh ciphertexts, decryption identities of
key switching, rotation (plain and hoisted), MulPC/AddCC and modulus switching.  Ciphertext
bits of key switching have no closed form; they are pinned through these identities."""
import numpy as np
import pytest

from oracle import bfv, encoder, params, prng, ring


@pytest.fixture(scope="module", params=[(8, 3, 1, 1), (8, 4, 2, 2), (8, 5, 2, 2)],
                ids=["L3K1a1", "L4K2a2", "L5K2a2-partial-digit"])
def setup(request):
    log_n, nq, np_, alpha = request.param
    prm = params.Params(log_n=log_n, n_q=nq, n_p=np_, alpha=alpha)
    s = bfv.keygen_secret(prm, 17)
    return prm, s


def encrypt_slots(prm, s, v, seed):
    return bfv.encrypt(prm, s, encoder.encode(v, prm), seed)


def rand_slots(prm, seed):
    return np.random.default_rng(seed).integers(0, prm.t, prm.n)


def test_fresh_noise_is_exactly_the_error(setup):
    prm, s = setup
    v = rand_slots(prm, 0)
    m = encoder.encode(v, prm)
    ct = bfv.encrypt(prm, s, m, 5)
    assert (encoder.decode(bfv.decrypt(prm, s, ct), prm) == v).all()
    x, Q = bfv.phase(prm, s, ct)
    e = prng.gaussian(5, prng.STREAM_CT_E, prm.n)
    delta = prm.delta()
    for k in range(prm.n):
        assert (x[k] - delta * int(m[k]) - int(e[k])) % Q == 0


def test_galois_key_decrypts_to_gadget_times_rotated_secret(setup):
    prm, s = setup
    g = bfv.galois_element(1, prm.n)
    ksk = bfv.galois_key(prm, s, g, 3)
    sg = bfv.automorphism_int(s, g)
    for j in range(prm.dnum):
        e = prng.gaussian(3, prng.stream_key_e(g, j), prm.n)
        for l, q in enumerate(prm.qp):
            b, a = ksk[j, 0, l], ksk[j, 1, l]
            lhs = ring.vadd(b, ring.polymul_schoolbook(a, ring.from_signed(s, q), q), q)
            gj = prm.P % q if l in prm.digit(j) else 0
            want = ring.vmac_scalar(ring.from_signed(e, q), ring.from_signed(sg, q), gj, q)
            assert (lhs == want).all()


def test_automorphism_matches_integer_definition(setup):
    prm, s = setup
    g = bfv.galois_element(3, prm.n)
    a = bfv.to_rns(s * 3 + 1, prm.q)
    assert (bfv.automorphism(a, g, prm.q) == bfv.to_rns(bfv.automorphism_int(s * 3 + 1, g), prm.q)).all()


def test_keyswitch_error_is_small(setup):
    prm, s = setup
    g = bfv.galois_element(2, prm.n)
    ksk = bfv.galois_key(prm, s, g, 8)
    sg = bfv.automorphism_int(s, g)
    d = np.stack([np.random.default_rng(l).integers(0, q, prm.n, dtype=np.uint64) for l, q in enumerate(prm.q)])
    u0, u1 = bfv.keyswitch(prm, d, ksk)
    lhs = bfv.rns_add(u0, bfv.rns_mul(u1, bfv.to_rns(s, prm.q), prm, prm.q), prm.q)
    want = bfv.rns_mul(d, bfv.to_rns(sg, prm.q), prm, prm.q)
    err, Q = bfv.crt(bfv.rns_sub(lhs, want, prm.q), prm.q)
    worst = max(min(v, Q - v) for v in err)
    qmax = max(prm.q) ** prm.alpha
    bound = prm.dnum * prm.n * qmax * 19 // prm.P + prm.n * prm.n_p + prm.n
    assert worst <= bound


@pytest.mark.parametrize("step", [1, 5, -3, "swap"])
def test_rotation_plain_and_hoisted_shift_slots(setup, step):
    prm, s = setup
    n, half = prm.n, prm.n // 2
    v = rand_slots(prm, 4)
    ct = bfv.encrypt(prm, s, encoder.encode(v, prm), 9)
    g = bfv.galois_of(step, n)
    keys = {g: bfv.galois_key(prm, s, g, 2)}
    if step == "swap":
        want = np.concatenate([v[half:], v[:half]])
    else:
        want = np.concatenate([np.roll(v[:half], -step), np.roll(v[half:], -step)])
    r = bfv.rotate(prm, ct, step, keys)
    h = bfv.rotate_hoisted(prm, ct, [step], keys)[0]
    for out in (r, h):
        assert (encoder.decode(bfv.decrypt(prm, s, out), prm) == want).all()
        assert bfv.noise_bits(prm, s, out)[1] > 20


def test_plain_product_sum_and_scalar(setup):
    prm, s = setup
    a, b = rand_slots(prm, 1), rand_slots(prm, 2)
    ca = bfv.encrypt(prm, s, encoder.encode(a, prm), 1)
    cb = bfv.encrypt(prm, s, encoder.encode(b, prm), 2)
    pt = bfv.pt_rns(encoder.encode(b, prm), prm)
    dec = lambda c: encoder.decode(bfv.decrypt(prm, s, c), prm)
    assert (dec(bfv.mul_plain(prm, ca, pt)) == (a * b) % prm.t).all()
    assert (dec(bfv.add(prm, ca, cb)) == (a + b) % prm.t).all()
    assert (dec(bfv.mul_scalar(prm, ca, -7)) == (a * -7) % prm.t).all()


def test_rescale_keeps_the_message(setup):
    prm, s = setup
    v = rand_slots(prm, 6)
    ct = bfv.encrypt(prm, s, encoder.encode(v, prm), 6)
    r = bfv.rescale(prm, ct)
    assert r.level == prm.n_q - 1
    assert (encoder.decode(bfv.decrypt(prm, s, r), prm) == v).all()
    # the coefficients are round(c / q_last) of the CRT value
    x, Q = bfv.crt(ct.c0, prm.q)
    y, Q2 = bfv.crt(r.c0, prm.q[:-1])
    ql = prm.q[-1]
    for k in range(0, prm.n, 37):
        assert y[k] == ((x[k] + (ql - 1) // 2) // ql) % Q2


def test_full_size_rotation_round_trip():
    prm = params.cfg_small_layer()
    s = bfv.keygen_secret(prm, 1)
    v = rand_slots(prm, 3)
    ct = bfv.encrypt(prm, s, encoder.encode(v, prm), 4)
    g = bfv.galois_element(29, prm.n)
    keys = {g: bfv.galois_key(prm, s, g, 5)}
    half = prm.n // 2
    want = np.concatenate([np.roll(v[:half], -29), np.roll(v[half:], -29)])
    out = bfv.rotate_hoisted(prm, ct, [29], keys)[0]
    assert (encoder.decode(bfv.decrypt(prm, s, out), prm) == want).all()


# ---- planted mistakes: each plausible slip in the oracle must trip one of the pins above

def test_planted_automorphism_sign_slip_is_caught(monkeypatch):
    prm = params.Params(log_n=6, n_q=2, n_p=1, alpha=1)
    s = bfv.keygen_secret(prm, 2)
    v = rand_slots(prm, 1)
    ct = bfv.encrypt(prm, s, encoder.encode(v, prm), 1)
    g = bfv.galois_element(1, prm.n)
    keys = {g: bfv.galois_key(prm, s, g, 1)}

    def wrong(a, g, moduli):          # forgets the sign flip of X^N = -1
        n = a.shape[1]
        idx = np.arange(n) * g % (2 * n) % n
        out = np.empty_like(a)
        out[:, idx] = a
        return out
    monkeypatch.setattr(bfv, "automorphism", wrong)
    out = bfv.rotate(prm, ct, 1, keys)
    half = prm.n // 2
    want = np.concatenate([np.roll(v[:half], -1), np.roll(v[half:], -1)])
    assert not (encoder.decode(bfv.decrypt(prm, s, out), prm) == want).all()


def test_planted_moddown_slip_is_caught(monkeypatch):
    prm = params.Params(log_n=6, n_q=2, n_p=1, alpha=1)
    s = bfv.keygen_secret(prm, 2)
    v = rand_slots(prm, 1)
    ct = bfv.encrypt(prm, s, encoder.encode(v, prm), 1)
    g = bfv.galois_element(1, prm.n)
    keys = {g: bfv.galois_key(prm, s, g, 1)}
    real = bfv.moddown
    monkeypatch.setattr(bfv, "moddown", lambda prm, u: u[: prm.n_q])   # drops the division by P
    out = bfv.rotate(prm, ct, 1, keys)
    monkeypatch.setattr(bfv, "moddown", real)
    half = prm.n // 2
    want = np.concatenate([np.roll(v[:half], -1), np.roll(v[half:], -1)])
    assert not (encoder.decode(bfv.decrypt(prm, s, out), prm) == want).all()


def test_multiply_three_component_decryption_and_relinearisation(setup):
    """(d0, d1, d2) decrypts under (1, s, s^2) to the slot-wise product; after relinearising
    with the s^2 -> s key, (c0, c1) decrypts to it under s (Sec. 2.1's homomorphic multiply)."""
    prm, s = setup
    rng = np.random.default_rng(12)
    v, w = rng.integers(0, prm.t, prm.n), rng.integers(0, prm.t, prm.n)
    a = encrypt_slots(prm, s, v, 21)
    b = encrypt_slots(prm, s, w, 22)
    d = bfv.multiply(prm, a, b)
    # three-component phase d0 + d1 s + d2 s^2
    sr = bfv.to_rns(s, prm.q)
    s2 = bfv.rns_mul(sr, sr, prm, prm.q)
    x = bfv.rns_add(bfv.rns_add(d[0], bfv.rns_mul(d[1], sr, prm, prm.q), prm.q),
                    bfv.rns_mul(d[2], s2, prm, prm.q), prm.q)
    vals, Q = bfv.crt(x, prm.q)
    m = np.array([((prm.t * v_ + (Q - 1) // 2) // Q) % prm.t for v_ in vals], dtype=np.int64)
    assert (encoder.decode(m, prm) == (v * w) % prm.t).all()
    c = bfv.relinearize(prm, d, bfv.relin_key(prm, s, 23))
    assert (encoder.decode(bfv.decrypt(prm, s, c), prm) == (v * w) % prm.t).all()
    assert bfv.noise_bits(prm, s, c)[1] > 20


def test_planted_scaling_slip_in_multiply_is_caught(monkeypatch, setup):
    """Dropping the t/Q scaling of the tensor product must break the product."""
    prm, s = setup
    rng = np.random.default_rng(13)
    v, w = rng.integers(0, prm.t, prm.n), rng.integers(0, prm.t, prm.n)
    a, b = encrypt_slots(prm, s, v, 31), encrypt_slots(prm, s, w, 32)
    rlk = bfv.relin_key(prm, s, 33)
    monkeypatch.setattr(bfv, "scale_round", lambda ints, t, Q: ints)
    bad = bfv.relinearize(prm, bfv.multiply(prm, a, b), rlk)
    assert not (encoder.decode(bfv.decrypt(prm, s, bad), prm) == (v * w) % prm.t).all()


@pytest.mark.parametrize("cfg", [(4, 2, 1, 1), (5, 3, 1, 1)])
def test_multiply_equals_brute_force_definition(cfg):
    """On tiny rings, for arbitrary residues (not only encryptions): d_k = round(t D_k / Q)
    mod q_i with D_k the exact negacyclic products of the centred lifts, written out with
    Python integers (no CRT over auxiliary primes, no NTT)."""
    log_n, nq, np_, alpha = cfg
    prm = params.Params(log_n=log_n, n_q=nq, n_p=np_, alpha=alpha)
    n, t, Q = prm.n, prm.t, prm.Q(nq)
    rng = np.random.default_rng(log_n)
    rand = lambda: np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in prm.q])
    a, b = bfv.Ct(rand(), rand()), bfv.Ct(rand(), rand())

    def lift(x):
        out = []
        for j in range(n):
            v = 0
            for i, q in enumerate(prm.q):          # CRT by the textbook formula
                Qi = Q // q
                v += int(x[i][j]) * Qi * pow(Qi, -1, q)
            v %= Q
            out.append(v - Q if 2 * v > Q else v)
        return out

    def negacyclic(x, y):
        z = [0] * n
        for i in range(n):
            for j in range(n):
                if i + j < n:
                    z[i + j] += x[i] * y[j]
                else:
                    z[i + j - n] -= x[i] * y[j]
        return z

    A0, A1, B0, B1 = lift(a.c0), lift(a.c1), lift(b.c0), lift(b.c1)
    D = [negacyclic(A0, B0),
         [u + v for u, v in zip(negacyclic(A0, B1), negacyclic(A1, B0))],
         negacyclic(A1, B1)]
    got = bfv.multiply(prm, a, b)
    for k in range(3):
        # floor(t D / Q + 1/2); no ties, as 2 t D + Q is odd and 2Q is even
        want = [(2 * t * v + Q) // (2 * Q) for v in D[k]]
        for i, q in enumerate(prm.q):
            assert [int(e) for e in got[k][i]] == [w % q for w in want], (k, i)
