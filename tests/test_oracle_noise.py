"""Pins for the oracle's noise measurement, bfv.noise_bits (Sec. 2.1: a BFV ciphertext decrypts
while its noise stays below Delta / 2, Delta = floor(Q / t); the noise budget is the number of
bits left between the two).

noise_bits is checked against closed forms that do not go through it:

  * a fresh symmetric encryption has c0 + c1 s = e + Delta m exactly, so its noise is the
    sampled error e itself (re-drawn here from the sampler at the encryption's stream) and
    noise_bits must return log2(max |e|) and log2(Delta / 2) minus that;
  * after the product with a constant w > 0, c0 + c1 s = w e + w Delta m.  Decryption gives
    m' = w m mod t, and w Delta m - Delta m' = Delta t floor(w m / t), which is
    -floor(w m / t) (Q mod t) modulo Q because Delta t = Q - (Q mod t).  The noise is therefore
    w e_k - floor(w m_k / t) (Q mod t) per coefficient: exactly w e when no w m_k reaches t.

A planted slip (the remainder left in [0, Q) instead of centred) must fail both pins."""
from math import log2

import numpy as np
import pytest

from oracle import bfv, params, prng


@pytest.fixture(scope="module", params=[(8, 3, 1, 1), (8, 4, 2, 2), (9, 2, 1, 1)],
                ids=["n256-L3", "n256-L4", "n512-L2"])
def setup(request):
    log_n, nq, np_, alpha = request.param
    prm = params.Params(log_n=log_n, n_q=nq, n_p=np_, alpha=alpha)
    return prm, bfv.keygen_secret(prm, 23)


def _Q(prm, level=None):
    Q = 1
    for q in prm.q[: (prm.n_q if level is None else level)]:
        Q *= q
    return Q


def fresh_pin_holds(noise_fn, prm, s, seed):
    """noise_fn on a fresh encryption equals log2 of the largest sampled error."""
    m = np.random.default_rng(seed).integers(0, prm.t, prm.n).astype(np.uint64)
    ct = bfv.encrypt(prm, s, m, seed)
    e = prng.gaussian(seed, prng.STREAM_CT_E, prm.n)
    worst = int(np.abs(e.astype(np.int64)).max())
    nb, budget = noise_fn(prm, s, ct)
    delta = _Q(prm) // prm.t
    return nb == log2(worst) and budget == log2(delta / 2) - log2(worst)


def scalar_pin_holds(noise_fn, prm, s, seed, w, m_max):
    """noise_fn after a product with the constant w equals the closed form above."""
    m = np.random.default_rng(seed).integers(0, m_max, prm.n).astype(np.uint64)
    ct = bfv.mul_scalar(prm, bfv.encrypt(prm, s, m, seed), w)
    e = prng.gaussian(seed, prng.STREAM_CT_E, prm.n).astype(np.int64)
    Q = _Q(prm)
    want = max(abs(w * int(ek) - (w * int(mk) // prm.t) * (Q % prm.t)) for ek, mk in zip(e, m))
    nb, _ = noise_fn(prm, s, ct)
    return nb == log2(want)


def test_fresh_noise_bits_is_log2_of_the_sampled_error(setup):
    prm, s = setup
    for seed in (3, 4, 5):
        assert fresh_pin_holds(bfv.noise_bits, prm, s, seed)


@pytest.mark.parametrize("w", [1, 5, 8, 127])
def test_scalar_product_noise_is_w_times_the_error_without_wrap(setup, w):
    prm, s = setup
    # message coefficients below t / w: w m never reaches t, so the noise is exactly w e
    assert scalar_pin_holds(bfv.noise_bits, prm, s, 7, w, prm.t // w)
    m = np.random.default_rng(7).integers(0, prm.t // w, prm.n)
    assert (w * m < prm.t).all()


@pytest.mark.parametrize("w", [3, 8])
def test_scalar_product_noise_with_wrap_matches_closed_form(setup, w):
    prm, s = setup
    assert scalar_pin_holds(bfv.noise_bits, prm, s, 11, w, prm.t)


def test_noise_bits_with_explicit_message_agrees(setup):
    prm, s = setup
    m = np.random.default_rng(2).integers(0, prm.t, prm.n).astype(np.uint64)
    ct = bfv.encrypt(prm, s, m, 2)
    assert bfv.noise_bits(prm, s, ct) == bfv.noise_bits(prm, s, ct, m.astype(np.int64))


def _uncentred_noise_bits(prm, s, ct, m=None):
    """A plausible slip: the same measurement with the remainder left in [0, Q)."""
    x, Q = bfv.phase(prm, s, ct)
    if m is None:
        m = bfv.decrypt(prm, s, ct)
    delta = Q // prm.t
    worst = max((v - delta * int(mk)) % Q for v, mk in zip(x, m))
    nb = log2(worst) if worst > 0 else 0.0
    return nb, log2(delta / 2) - nb


def test_planted_uncentred_remainder_is_caught(setup):
    prm, s = setup
    assert not fresh_pin_holds(_uncentred_noise_bits, prm, s, 3)
    assert not scalar_pin_holds(_uncentred_noise_bits, prm, s, 7, 5, prm.t // 5)
