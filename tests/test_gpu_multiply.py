"""GPU parity of ciphertext multiplication with relinearisation (Sec. 2.1's homomorphic
multiplication; the square is the x^2 activation of Sec. 3) against the CPU oracle, bit for bit.

The relinearisation key generated on the GPU must equal the oracle's; he_multiply on oracle
ciphertexts with the oracle's key must give exactly relinearize(multiply(a, b)), and its
decryption must be the slot-wise product mod t."""
import numpy as np
import pytest

from oracle import bfv, encoder, params
from tests.gpu_common import download_coeff, encrypt_slots, make_ctx, upload_ntt

pytestmark = pytest.mark.gpu

CONFIGS = {"n512": (9, 3, 1, 1), "n1024_a2": (10, 4, 2, 2), "n1024_partial": (10, 5, 2, 2),
           "n8192": (13, 3, 1, 1), "n32768_l12": (15, 12, 3, 3)}


def prm_of(name):
    c = CONFIGS[name]
    return params.Params(log_n=c[0], n_q=c[1], n_p=c[2], alpha=c[3])


@pytest.mark.parametrize("name", ["n512", "n1024_partial", "n32768_l12"])
def test_relin_key_is_bit_exact(name):
    from paper_2102_03494_gb300 import he
    prm = prm_of(name)
    ctx = make_ctx(prm)
    s = bfv.keygen_secret(prm, 21)
    ctx.he_keygen_galois(s, 8, [he.HE_RELIN_KEY, 1])
    assert (ctx.he_export_galois(he.HE_RELIN_KEY) == bfv.relin_key(prm, s, 8)).all()
    # the rotation key beside it is unaffected
    assert (ctx.he_export_galois(1) == bfv.galois_key(prm, s, bfv.galois_of(1, prm.n), 8)).all()


@pytest.mark.parametrize("name", list(CONFIGS))
def test_multiply_is_bit_exact(name):
    from paper_2102_03494_gb300 import he
    prm = prm_of(name)
    ctx = make_ctx(prm)
    s = bfv.keygen_secret(prm, 31)
    rlk = bfv.relin_key(prm, s, 6)
    ctx.he_load_keys(rlk.reshape(-1), [he.HE_RELIN_KEY])
    rng = np.random.default_rng(7)
    v = rng.integers(0, prm.t, prm.n)
    w = rng.integers(0, prm.t, prm.n)
    a = encrypt_slots(prm, s, v, 50)
    b = encrypt_slots(prm, s, w, 51)
    da, db = upload_ntt(ctx, a), upload_ntt(ctx, b)
    want = bfv.relinearize(prm, bfv.multiply(prm, a, b), rlk)
    got = ctx.he_multiply(da, db)
    assert (download_coeff(ctx, got) == want.stack()).all()
    assert (ctx.he_decrypt(s, got) == (v * w) % prm.t).all()
    # inputs untouched; square through the same buffer; output aliasing an input
    assert (download_coeff(ctx, da) == a.stack()).all()
    sq = bfv.relinearize(prm, bfv.multiply(prm, a, a), rlk)
    assert (download_coeff(ctx, ctx.he_multiply(da, da)) == sq.stack()).all()
    ctx.he_multiply(da, db, out=da)
    assert (download_coeff(ctx, da) == want.stack()).all()


def test_square_of_small_values_and_depth_two():
    """x -> x^2 -> x^4 on small slot values: exact products, noise within budget."""
    from paper_2102_03494_gb300 import he
    prm = prm_of("n8192")
    ctx = make_ctx(prm)
    s = bfv.keygen_secret(prm, 41)
    ctx.he_keygen_galois(s, 3, [he.HE_RELIN_KEY])
    x = np.random.default_rng(9).integers(-9, 10, prm.n)
    ct = encrypt_slots(prm, s, x % prm.t, 12)
    d = upload_ntt(ctx, ct)
    x2 = ctx.he_multiply(d, d)
    assert (ctx.he_decrypt(s, x2) == (x * x) % prm.t).all()
    want2 = bfv.relinearize(prm, bfv.multiply(prm, ct, ct), bfv.relin_key(prm, s, 3))
    assert (download_coeff(ctx, x2) == want2.stack()).all()
    x4 = ctx.he_multiply(x2, x2)
    assert (ctx.he_decrypt(s, x4) == (x ** 4) % prm.t).all()
    m = encoder.decode(bfv.decrypt(prm, s, bfv.Ct(*download_coeff(ctx, x4))), prm)
    assert (m == (x ** 4) % prm.t).all()


def test_multiply_errors():
    from paper_2102_03494_gb300 import he
    prm = prm_of("n512")
    ctx = make_ctx(prm)
    s = bfv.keygen_secret(prm, 1)
    d = upload_ntt(ctx, encrypt_slots(prm, s, np.zeros(prm.n, np.int64), 1))
    with pytest.raises(he.HeError) as e:
        ctx.he_multiply(d, d)
    assert e.value.code == he.HE_ENOKEY
    ctx.he_keygen_galois(s, 3, [he.HE_RELIN_KEY])
    low = ctx.he_rescale(d)
    with pytest.raises(he.HeError) as e:
        ctx.he_multiply(low, low)                     # below full level
    assert e.value.code == he.HE_EINVAL


def test_multiword_rounding_path_is_bit_exact(monkeypatch):
    """HE_MULT_EXACT=1 sends every coefficient through the multi-word path (the one the fast
    fixed-point rounding falls back to); it must give the same bits as the oracle."""
    from paper_2102_03494_gb300 import he
    prm = prm_of("n1024_partial")
    ctx = make_ctx(prm)
    s = bfv.keygen_secret(prm, 13)
    rlk = bfv.relin_key(prm, s, 4)
    ctx.he_load_keys(rlk.reshape(-1), [he.HE_RELIN_KEY])
    rng = np.random.default_rng(17)
    a = encrypt_slots(prm, s, rng.integers(0, prm.t, prm.n), 70)
    b = encrypt_slots(prm, s, rng.integers(0, prm.t, prm.n), 71)
    want = bfv.relinearize(prm, bfv.multiply(prm, a, b), rlk)
    da, db = upload_ntt(ctx, a), upload_ntt(ctx, b)
    monkeypatch.setenv("HE_MULT_EXACT", "1")
    got = ctx.he_multiply(da, db)
    assert (download_coeff(ctx, got) == want.stack()).all()
    monkeypatch.delenv("HE_MULT_EXACT")
    fast = ctx.he_multiply(da, db)
    assert (download_coeff(ctx, fast) == want.stack()).all()
