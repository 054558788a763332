"""GPU parity of the RNS-BFV primitives against the CPU oracle, bit for bit.

Covers the NTT (against the oracle's evaluation at the odd powers of the same root), key and
encryption randomness, Galois keys, decryption, plain / batched / hoisted rotations, MulPC,
AddCC and modulus switching, at several ring sizes including N = 2^15 with 12 primes."""
import numpy as np
import pytest

from oracle import bfv, encoder, params, prng, ring
from tests.gpu_common import (download_coeff, encrypt_slots, gpu_steps, make_ctx, oracle_keys,
                              upload_ntt)

pytestmark = pytest.mark.gpu

CONFIGS = {"n512": (9, 3, 1, 1), "n1024_a2": (10, 4, 2, 2), "n1024_partial": (10, 5, 2, 2),
           "n8192": (13, 3, 1, 1)}


def brv(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2)


@pytest.mark.parametrize("radix", [8, 4])
@pytest.mark.parametrize("cfg", [(6, 2, 1, 1), (9, 3, 1, 1), (13, 3, 1, 1), (14, 6, 2, 2),
                                 (15, 12, 3, 3), (16, 24, 6, 6)])
def test_ntt_matches_oracle_evaluation(cfg, radix):
    """Forward / inverse NTT against the oracle's evaluation at the odd powers of psi, at every
    radix the autotuner may pick; the second item holds q - 1 everywhere (the largest growth
    of the unreduced forward butterflies used below 2^57)."""
    import torch
    from paper_2102_03494_gb300 import he
    prm = params.Params(log_n=cfg[0], n_q=cfg[1], n_p=cfg[2], alpha=cfg[3])
    ctx = make_ctx(prm)
    ctx.he_tune_set(he.HE_TUNE_NTT_RADIX, radix)
    assert ctx.he_tune_get(he.HE_TUNE_NTT_RADIX) == radix
    with pytest.raises(he.HeError):                 # rounds of 2 points are not built
        ctx.he_tune_set(he.HE_TUNE_NTT_RADIX, 2)
    items = 2
    a = np.stack([np.stack([np.random.default_rng(100 * i + l).integers(0, q, prm.n, dtype=np.uint64)
                            if i == 0 else np.full(prm.n, q - 1, dtype=np.uint64)
                            for l, q in enumerate(prm.qp)]) for i in range(items)])
    d = ctx.from_numpy(a)
    ctx.he_ntt(d, items, len(prm.qp), inverse=False)
    got = ctx.to_numpy(d)
    perm = np.array([brv(p, prm.log_n) for p in range(prm.n)])
    for i in range(items):
        for l in [0, len(prm.qp) - 1] + ([prm.n_q] if prm.n_q < len(prm.qp) else []):
            q = prm.qp[l]
            ev = ring.neg_eval(a[i, l], q, prm.psi[q])
            assert (got[i, l] == ev[perm]).all(), (i, l)
    ctx.he_ntt(d, items, len(prm.qp), inverse=True)
    assert (ctx.to_numpy(d) == a).all()
    # every split the autotuner may try (the row pass's twiddle order follows the split)
    for s1 in (prm.log_n // 2 - 1, prm.log_n // 2 + 1):
        if not (1 <= s1 < prm.log_n and 2 ** s1 <= 2048 and 2 ** (prm.log_n - s1) <= 2048):
            continue
        ctx.he_tune_set(he.HE_TUNE_NTT_SPLIT, s1)
        d = ctx.from_numpy(a)
        ctx.he_ntt(d, items, len(prm.qp), inverse=False)
        assert (ctx.to_numpy(d) == got).all(), s1
        ctx.he_ntt(d, items, len(prm.qp), inverse=True)
        assert (ctx.to_numpy(d) == a).all(), s1
    torch.cuda.synchronize()


@pytest.mark.parametrize("name", ["n512", "n1024_partial", "n8192"])
def test_secret_encryption_and_keys_are_bit_exact(name):
    prm = params.Params(*CONFIGS[name][:1], n_q=CONFIGS[name][1], n_p=CONFIGS[name][2],
                        alpha=CONFIGS[name][3])
    ctx = make_ctx(prm)
    sk = ctx.he_keygen_secret(77)
    s = bfv.keygen_secret(prm, 77)
    assert (sk == s).all()
    v = np.random.default_rng(5).integers(0, prm.t, prm.n)
    want = encrypt_slots(prm, s, v, 123)
    from paper_2102_03494_gb300 import he
    got = ctx.he_encrypt(sk, v, 123, domain=he.HE_COEFF)
    assert (ctx.to_numpy(got) == want.stack()).all()
    got_ntt = ctx.he_encrypt(sk, v, 123, domain=he.HE_NTT)
    assert (download_coeff(ctx, got_ntt) == want.stack()).all()
    steps = [1, -3, bfv.ROW_SWAP]
    ctx.he_keygen_galois(sk, 9, gpu_steps(steps))
    for st in steps:
        g = bfv.galois_of(st, prm.n)
        assert (ctx.he_export_galois(gpu_steps([st])[0]) == bfv.galois_key(prm, s, g, 9)).all()


def test_keys_at_n15_are_bit_exact():
    prm = params.cfg_n15()
    ctx = make_ctx(prm)
    s = bfv.keygen_secret(prm, 3)
    ctx.he_keygen_galois(s, 4, [7])
    want = bfv.galois_key(prm, s, bfv.galois_of(7, prm.n), 4)
    assert (ctx.he_export_galois(7) == want).all()


@pytest.mark.parametrize("name", list(CONFIGS))
def test_decrypt_matches_oracle(name):
    prm = params.Params(log_n=CONFIGS[name][0], n_q=CONFIGS[name][1], n_p=CONFIGS[name][2],
                        alpha=CONFIGS[name][3])
    ctx = make_ctx(prm)
    s = bfv.keygen_secret(prm, 1)
    v = np.random.default_rng(2).integers(0, prm.t, prm.n)
    ct = encrypt_slots(prm, s, v, 3)
    d = upload_ntt(ctx, ct)
    assert (ctx.he_decrypt(s, d) == v).all()
    from paper_2102_03494_gb300 import he
    assert (ctx.he_decrypt(s, ctx.from_numpy(ct.stack()), domain=he.HE_COEFF) == v).all()
    low = bfv.rescale(prm, ct)
    dl = ctx.from_numpy(low.stack())
    assert (ctx.he_decrypt(s, dl, domain=he.HE_COEFF) == v).all()


@pytest.mark.parametrize("name", list(CONFIGS))
def test_rotations_are_bit_exact(name):
    prm = params.Params(log_n=CONFIGS[name][0], n_q=CONFIGS[name][1], n_p=CONFIGS[name][2],
                        alpha=CONFIGS[name][3])
    ctx = make_ctx(prm)
    s = bfv.keygen_secret(prm, 11)
    steps = [1, 5, -3, bfv.ROW_SWAP]
    keys, blob = oracle_keys(prm, s, steps)
    ctx.he_load_keys(blob, gpu_steps(steps))
    cts = [encrypt_slots(prm, s, np.random.default_rng(i).integers(0, prm.t, prm.n), 40 + i)
           for i in range(3)]
    ds = [upload_ntt(ctx, c) for c in cts]
    # plain rotation, single and batched
    for st in steps:
        want = bfv.rotate(prm, cts[0], st, keys)
        got = ctx.he_rotate(ds[0], gpu_steps([st])[0])
        assert (download_coeff(ctx, got) == want.stack()).all(), st
    outs = ctx.he_rotate_batch(ds, 5)
    for c, o in zip(cts, outs):
        assert (download_coeff(ctx, o) == bfv.rotate(prm, c, 5, keys).stack()).all()
    # hoisted
    hs = ctx.he_rotate_hoisted(ds[1], gpu_steps(steps))
    for o, w in zip(hs, bfv.rotate_hoisted(prm, cts[1], steps, keys)):
        assert (download_coeff(ctx, o) == w.stack()).all()
    # batched hoisted: outs[i h + s] is ciphertext i rotated by step s
    hb = ctx.he_rotate_hoisted_batch(ds, gpu_steps(steps))
    for i, c in enumerate(cts):
        for j, w in enumerate(bfv.rotate_hoisted(prm, c, steps, keys)):
            assert (download_coeff(ctx, hb[i * len(steps) + j]) == w.stack()).all(), (i, j)
    with pytest.raises(RuntimeError):               # an output aliasing an input is refused
        ctx.he_rotate_hoisted_batch(ds[:2], gpu_steps(steps[:1]), [ctx.new_ct(), ds[0]])
    # decrypted slots shift as the paper's rotation does
    half = prm.n // 2
    v = encoder.decode(bfv.decrypt(prm, s, cts[1]), prm)
    got = ctx.he_decrypt(s, hs[0])
    assert (got[:half] == np.roll(v[:half], -1)).all() and (got[half:] == np.roll(v[half:], -1)).all()
    # in-place rotation (input and output alias)
    x = ds[2].clone()
    ctx.he_rotate(x, 1, out=x)
    assert (download_coeff(ctx, x) == bfv.rotate(prm, cts[2], 1, keys).stack()).all()


def test_rotations_at_n15_are_bit_exact():
    prm = params.cfg_n15()
    ctx = make_ctx(prm)
    s = bfv.keygen_secret(prm, 5)
    steps = [3, -29]
    keys, blob = oracle_keys(prm, s, steps)
    ctx.he_load_keys(blob, steps)
    ct = encrypt_slots(prm, s, np.random.default_rng(9).integers(0, prm.t, prm.n), 6)
    d = upload_ntt(ctx, ct)
    got = ctx.he_rotate(d, 3)
    assert (download_coeff(ctx, got) == bfv.rotate(prm, ct, 3, keys).stack()).all()
    hs = ctx.he_rotate_hoisted(d, steps)
    for o, w in zip(hs, bfv.rotate_hoisted(prm, ct, steps, keys)):
        assert (download_coeff(ctx, o) == w.stack()).all()


@pytest.mark.parametrize("name", ["n512", "n8192"])
def test_encode_mulpc_addcc_rescale_are_bit_exact(name):
    import torch
    prm = params.Params(log_n=CONFIGS[name][0], n_q=CONFIGS[name][1], n_p=CONFIGS[name][2],
                        alpha=CONFIGS[name][3])
    ctx = make_ctx(prm)
    s = bfv.keygen_secret(prm, 2)
    rng = np.random.default_rng(8)
    vs = [rng.integers(0, prm.t, prm.n) for _ in range(3)]
    ws = [rng.integers(-prm.t // 2, prm.t // 2, prm.n) for _ in range(3)]
    cts = [encrypt_slots(prm, s, v, 70 + i) for i, v in enumerate(vs)]
    pts_o = [bfv.pt_rns(encoder.encode(w, prm), prm) for w in ws]
    pts = torch.stack([ctx.he_encode(w) for w in ws])
    for p, po in zip(pts, pts_o):     # encoder: centred lift, NTT domain
        c = p.clone()
        ctx.he_ntt(c, 1, prm.n_q, inverse=True)
        assert (ctx.to_numpy(c) == po).all()
    ds = [upload_ntt(ctx, c) for c in cts]
    acc = upload_ntt(ctx, cts[0])
    ctx.he_mul_plain_acc(ds, pts, acc)
    want = cts[0]
    for c, po in zip(cts, pts_o):
        want = bfv.add(prm, want, bfv.mul_plain(prm, c, po))
    assert (download_coeff(ctx, acc) == want.stack()).all()
    got = ctx.he_add(ds[0], ds[1])
    assert (download_coeff(ctx, got) == bfv.add(prm, cts[0], cts[1]).stack()).all()
    r = ctx.he_rescale(ds[2])
    assert (download_coeff(ctx, r) == bfv.rescale(prm, cts[2]).stack()).all()
    assert (ctx.he_decrypt(s, r) == vs[2]).all()


def test_error_paths():
    from paper_2102_03494_gb300 import he
    prm = params.Params(log_n=9, n_q=3, n_p=1, alpha=1)
    ctx = make_ctx(prm)
    s = bfv.keygen_secret(prm, 1)
    d = upload_ntt(ctx, encrypt_slots(prm, s, np.zeros(prm.n, np.int64), 1))
    with pytest.raises(he.HeError) as e:
        ctx.he_rotate(d, 3)
    assert e.value.code == he.HE_ENOKEY
    with pytest.raises(he.HeError) as e:
        ctx.he_rescale(d, out=ctx.new_ct(level=3))     # wrong output level
    assert e.value.code == he.HE_EINVAL
    bad = ctx.layout(1, 40, 40, 5, 2, 1, 2, 5)          # 1600 slots > N/2 = 256
    with pytest.raises(he.HeError):
        ctx.he_ffconv_required_steps(bad)
    # corrupted key material (a residue equal to its modulus) is refused and not kept
    key = bfv.galois_key(prm, s, bfv.galois_of(3, prm.n), 7)
    blob = key.reshape(-1).copy()
    blob[5 * prm.n + 17] = prm.qp[5 % len(prm.qp)]     # row 5 of the first (b) polynomial
    with pytest.raises(he.HeError) as e:
        ctx.he_load_keys(blob, [3])
    assert e.value.code == he.HE_EINVAL
    with pytest.raises(he.HeError) as e:
        ctx.he_rotate(d, 3)
    assert e.value.code == he.HE_ENOKEY
    ctx.he_load_keys(key.reshape(-1), [3])                 # intact material loads
    ctx.he_rotate(d, 3)
    with pytest.raises(he.HeError) as e:
        ctx.he_ffconv_layer(d, np.ones((2, 1, 5, 5)), np.ones((5, 2)), bad)
    assert e.value.code == he.HE_EINVAL


def test_integer_rate_probe_is_sane():
    """The multiply-accumulate probes return rates below the derived issue-slot bounds: per
    SM and clock at most 64 multiply-adds of any kind, and a 64 x 64 -> 128-bit product takes
    at least four of them (2070 MHz maximum clock, with margin)."""
    import torch
    prm = params.Params(log_n=9, n_q=3, n_p=1, alpha=1)
    ctx = make_ctx(prm)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    slots = sms * 64 * 2070e6
    chain, cols = ctx.he_probe_int_mac()
    for v in (chain, cols):
        assert 0.02 * slots / 4 < v < 1.1 * slots / 4
    ops = ctx.he_probe_int_ops()
    for k in ("mad_lo", "mad_hi", "mad_wide"):
        assert 0.05 * slots < ops[k] < 1.1 * slots
    for k in ("chain", "chain_wide", "columns", "karatsuba"):
        assert 0.02 * slots / 4 < ops[k] < 1.1 * slots / 3
    mem = ctx.he_probe_mem()          # L2-resident reads outrun HBM reads; HBM below 8 TB/s
    assert 500 < mem["hbm_read_gbs"] < 8000 and mem["l2_read_gbs"] > mem["hbm_read_gbs"]


@pytest.mark.parametrize("cfg", [(13, 3, 1, 1), (14, 8, 2, 2), (15, 16, 4, 4), (16, 24, 6, 6)])
def test_sweep_rotations_are_bit_exact(cfg):
    """Corners of the primitive sweep: N = 2^13 .. 2^16 with 3, 8, 16, 24 primes of 50 bits and
    1, 2, 4, 6 special primes (alpha = K); uniform random residues as ciphertexts, two steps
    uniform in [1, N/2); plain, batched and hoisted rotations against the oracle."""
    prm = params.Params(log_n=cfg[0], n_q=cfg[1], n_p=cfg[2], alpha=cfg[3])
    ctx = make_ctx(prm)
    s = bfv.keygen_secret(prm, 21)
    rng = np.random.default_rng(cfg[0])
    steps = [int(x) for x in rng.integers(1, prm.n // 2, 2)]
    keys, blob = oracle_keys(prm, s, steps)
    ctx.he_load_keys(blob, steps)
    cts = [bfv.Ct(*[np.stack([rng.integers(0, q, prm.n, dtype=np.uint64) for q in prm.q])
                    for _ in range(2)]) for _ in range(2)]
    ds = [upload_ntt(ctx, c) for c in cts]
    want = bfv.rotate(prm, cts[0], steps[0], keys)
    assert (download_coeff(ctx, ctx.he_rotate(ds[0], steps[0])) == want.stack()).all()
    outs = ctx.he_rotate_batch(ds, steps[0])
    assert (download_coeff(ctx, outs[0]) == want.stack()).all()
    if prm.log_n < 16:
        assert (download_coeff(ctx, outs[1]) == bfv.rotate(prm, cts[1], steps[0], keys).stack()).all()
    hs = ctx.he_rotate_hoisted(ds[1], steps)
    for o, w in zip(hs, bfv.rotate_hoisted(prm, cts[1], steps, keys)):
        assert (download_coeff(ctx, o) == w.stack()).all()
    # the batched hoisted call over more ciphertexts than one key-switching chunk holds (about
    # 1 GiB of scratch: 8 ciphertexts at N = 2^16 with 24 + 6 primes) equals one call per
    # ciphertext, bit for bit
    import torch
    more = ds + [torch.randint_like(ds[0], 0, 1 << 40) for _ in range(8)]   # residues < 2^40 < q
    torch.cuda.synchronize()
    hb = ctx.he_rotate_hoisted_batch(more, steps)
    for i, m in enumerate(more):
        for j, o in enumerate(ctx.he_rotate_hoisted(m, steps)):
            assert torch.equal(hb[i * 2 + j], o), (i, j)


@pytest.mark.parametrize("cfg", [(9, 3, 1, 1), (13, 3, 1, 1), (15, 16, 4, 4), (16, 24, 6, 6)])
def test_automorphism_is_bit_exact(cfg):
    """he_automorphism (X -> X^g on both polynomials, no key switch) against the oracle's
    coefficient-domain automorphism, for ciphertexts stored back to back (one launch) and
    apart (a launch each), with a random step and the row swap."""
    from paper_2102_03494_gb300 import he
    prm = params.Params(log_n=cfg[0], n_q=cfg[1], n_p=cfg[2], alpha=cfg[3])
    ctx = make_ctx(prm)
    rng = np.random.default_rng(cfg[0] + 100)
    cts = [bfv.Ct(*[np.stack([rng.integers(0, q, prm.n, dtype=np.uint64) for q in prm.q])
                    for _ in range(2)]) for _ in range(3)]
    step = int(rng.integers(1, prm.n // 2))
    block = ctx.new_ct(count=3)
    for i, c in enumerate(cts):
        block[i].copy_(upload_ntt(ctx, c))
    for st, g in ((step, bfv.galois_of(step, prm.n)), (he.HE_ROW_SWAP, 2 * prm.n - 1)):
        # the lists marshalled once (as the sweep passes them), back to back: one launch
        outs = ctx.he_automorphism(ctx.ct_batch(list(block)), st,
                                   outs=ctx.ct_batch(list(ctx.new_ct(count=3))))
        apart = ctx.he_automorphism([block[2], block[0]], st)
        for i, c in enumerate(cts):
            want = np.stack([bfv.automorphism(c.c0, g, prm.q), bfv.automorphism(c.c1, g, prm.q)])
            assert (download_coeff(ctx, outs[i]) == want).all()
        for o, i in zip(apart, (2, 0)):
            want = np.stack([bfv.automorphism(cts[i].c0, g, prm.q), bfv.automorphism(cts[i].c1, g, prm.q)])
            assert (download_coeff(ctx, o) == want).all()
    with pytest.raises(he.HeError):
        ctx.he_automorphism([block[0]], 1, outs=[block[0]])
