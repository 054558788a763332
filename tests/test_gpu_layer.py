"""GPU parity of the encrypted FFConv layer (Sec. 4.2) against the CPU oracle.

Bit-exact on every output ciphertext coefficient where the oracle finishes in seconds (small
rings, and the 1 x 28 x 28 layer at N = 8192 under DP_SHIFT); at the benchmark's N = 2^15
configuration one sampled image of the timed batch of 64 is compared bit for bit, and every
image's decrypted outputs (as for DP_DOT at N = 8192) with the plain integer convolution mod t
(exact), and operation counts with the schedule's formulas."""
import numpy as np
import pytest

from oracle import bfv, encoder, ffconv, params
from paper_2102_03494_gb300 import workloads
from tests.gpu_common import download_coeff, gpu_steps, make_ctx, oracle_keys, upload_ntt

pytestmark = pytest.mark.gpu


def setup_layer(prm, shape, pack, seed=0, modswitch=False, B=1):
    lay_o = ffconv.Layout(*shape.astuple(), pack=pack, modswitch=modswitch)
    s = bfv.keygen_secret(prm, seed + 1)
    steps = ffconv.required_steps(lay_o, prm.n)
    keys, blob = oracle_keys(prm, s, steps, seed + 2)
    xs = workloads.images(seed, shape, B)
    W1, W2 = workloads.weights(seed, shape)
    if pack == "cp_cp":     # B * K Im2Col column ciphertexts
        cts = [bfv.encrypt(prm, s, encoder.encode(v, prm), seed + 3 + 100 * b + k)
               for b, x in enumerate(xs) for k, v in enumerate(ffconv.im2col_slots(x, lay_o, prm.n))]
    else:
        cts = [bfv.encrypt(prm, s, encoder.encode(ffconv.input_slots(x, lay_o, prm.n), prm), seed + 3 + b)
               for b, x in enumerate(xs)]
    return lay_o, s, steps, keys, blob, xs, W1, W2, cts


def check_decrypted(ctx, prm, s, lay_o, outs, x, W1, W2):
    _, y2 = ffconv.plain_layer(x, W1, W2, lay_o)
    for c, o in enumerate(outs):
        v = ctx.he_decrypt(s, o)
        for oh in range(lay_o.O_h):
            for ow in range(lay_o.O_w):
                assert v[ffconv.output_slot(lay_o, oh, ow)] == y2[c, oh, ow] % prm.t


SMALL = [workloads.LayerShape(1, 8, 8, 3, 2, 1, 2, 3), workloads.LayerShape(2, 6, 6, 3, 1, 1, 2, 2),
         workloads.LayerShape(3, 5, 7, 3, 2, 1, 3, 4), workloads.LayerShape(1, 9, 9, 5, 2, 2, 1, 2)]


@pytest.mark.parametrize("pack", ["dp_shift", "dp_shift_ext", "dp_dot", "dp_dp"])
@pytest.mark.parametrize("si", range(len(SMALL)))
def test_small_layers_are_bit_exact(pack, si):
    prm = params.Params(log_n=9, n_q=3, n_p=1, alpha=1)
    shape = SMALL[si]
    lay_o, s, steps, keys, blob, xs, W1, W2, cts = setup_layer(prm, shape, pack, seed=si)
    ctx = make_ctx(prm)
    ctx.he_load_keys(blob, gpu_steps(steps))
    lay = ctx.layout(*shape.astuple(), pack=pack)
    assert ctx.he_ffconv_required_steps(lay) == gpu_steps(steps)
    ops = ffconv.OpCount()
    want = ffconv.he_layer(prm, cts[0], W1, W2, lay_o, keys, ops)
    ctx.he_reset_op_counts()
    outs = ctx.he_ffconv_layer(upload_ntt(ctx, cts[0]), W1, W2, lay)
    for o, w in zip(outs, want):
        assert (download_coeff(ctx, o) == w.stack()).all()
    got_ops = ctx.he_op_counts()
    assert {k: got_ops[k] for k in ("mulpc", "addcc", "rot")} == ops.as_dict() == \
        ffconv.expected_ops(lay_o, prm.n)
    check_decrypted(ctx, prm, s, lay_o, outs, xs[0], W1, W2)


@pytest.mark.parametrize("pack", ["dp_shift", "dp_shift_ext", "dp_dot"])
def test_batched_layer_with_modswitch_and_wide_digits(pack):
    prm = params.Params(log_n=10, n_q=4, n_p=2, alpha=2)
    shape = workloads.LayerShape(2, 6, 6, 3, 2, 1, 2, 3)
    B = 3
    lay_o, s, steps, keys, blob, xs, W1, W2, cts = setup_layer(prm, shape, pack, seed=7,
                                                                modswitch=True, B=B)
    ctx = make_ctx(prm)
    ctx.he_load_keys(blob, gpu_steps(steps))
    lay = ctx.layout(*shape.astuple(), pack=pack, modswitch=True)
    outs = ctx.he_ffconv_layer_batch([upload_ntt(ctx, c) for c in cts], W1, W2, lay)
    for b in range(B):
        want = ffconv.he_layer(prm, cts[b], W1, W2, lay_o, keys)
        for c in range(shape.O_c):
            assert (download_coeff(ctx, outs[b * shape.O_c + c]) == want[c].stack()).all()
        single = ctx.he_ffconv_layer(upload_ntt(ctx, cts[b]), W1, W2, lay)
        for c in range(shape.O_c):
            assert (ctx.to_numpy(single[c]) == ctx.to_numpy(outs[b * shape.O_c + c])).all()


@pytest.mark.parametrize("pack", ["dp_shift", "dp_shift_ext"])
def test_mnist_layer_n8192_is_bit_exact(pack):
    """The 1 x 28 x 28, 5 x 5 stride-2, r = 2 -> 5 channel layer at N = 8192 (3 x 50-bit q)."""
    prm = params.cfg_small_layer()
    shape = workloads.MNIST_LAYER
    lay_o, s, steps, keys, blob, xs, W1, W2, cts = setup_layer(prm, shape, pack)
    ctx = make_ctx(prm)
    ctx.he_load_keys(blob, gpu_steps(steps))
    lay = ctx.layout(*shape.astuple(), pack=pack)
    want = ffconv.he_layer(prm, cts[0], W1, W2, lay_o, keys)
    outs = ctx.he_ffconv_layer(upload_ntt(ctx, cts[0]), W1, W2, lay)
    for o, w in zip(outs, want):
        assert (download_coeff(ctx, o) == w.stack()).all()
    check_decrypted(ctx, prm, s, lay_o, outs, xs[0], W1, W2)


def test_mnist_layer_dp_dot_n8192_decrypts_to_the_convolution():
    prm = params.cfg_small_layer()
    shape = workloads.MNIST_LAYER
    ctx = make_ctx(prm)
    lay_o = ffconv.Layout(*shape.astuple(), pack="dp_dot")
    lay = ctx.layout(*shape.astuple(), pack="dp_dot")
    sk = ctx.he_keygen_secret(1)
    ctx.he_keygen_galois(sk, 2, ctx.he_ffconv_required_steps(lay))
    x = workloads.image(0, shape)
    W1, W2 = workloads.weights(0, shape)
    ct = ctx.he_encrypt(sk, ffconv.input_slots(x, lay_o, prm.n), 3)
    ctx.he_reset_op_counts()
    outs = ctx.he_ffconv_layer(ct, W1, W2, lay)
    check_decrypted(ctx, prm, sk, lay_o, outs, x, W1, W2)
    got = ctx.he_op_counts()
    assert {k: got[k] for k in ("mulpc", "addcc", "rot")} == ffconv.expected_ops(lay_o, prm.n)
    assert got["rot"] == 2 * 169 * 10


@pytest.mark.parametrize("pack,B", [("dp_shift", 1), ("dp_shift", 4), ("dp_shift_ext", 1),
                                    ("dp_shift_ext", 64)])
def test_bench_layer_n15_decrypts_to_the_convolution(pack, B):
    """The benchmark configuration: N = 2^15, 12 x 50-bit q, 3 x 60-bit p, digits of 3, in the
    launch configuration the benchmark times (batch of 64 under dp_shift_ext)."""
    prm = params.cfg_n15()
    shape = workloads.MNIST_LAYER
    ctx = make_ctx(prm)
    lay_o = ffconv.Layout(*shape.astuple(), pack=pack)
    lay = ctx.layout(*shape.astuple(), pack=pack)
    sk = ctx.he_keygen_secret(1)
    ctx.he_keygen_galois(sk, 2, ctx.he_ffconv_required_steps(lay))
    xs = workloads.images(0, shape, B)
    W1, W2 = workloads.weights(0, shape)
    cts = [ctx.he_encrypt(sk, ffconv.input_slots(x, lay_o, prm.n), 3 + b) for b, x in enumerate(xs)]
    outs = ctx.he_ffconv_layer_batch(cts, W1, W2, lay)
    for b in range(B):
        check_decrypted(ctx, prm, sk, lay_o, outs[b * 5:(b + 1) * 5], xs[b], W1, W2)


def _oracle_layer(args):
    """One image's oracle layer (runs in a spawned worker)."""
    prm, ct, W1, W2, lay_o, keys = args
    return [w.stack() for w in ffconv.he_layer(prm, ct, W1, W2, lay_o, keys)]


def test_bench_layer_n15_sampled_images_are_bit_exact():
    """The benchmark's own launch: N = 2^15 (12 + 3 primes, digits of 3), dp_shift_ext, a batch
    of 64 images in one call (grid and tile as timed), under each of the tap kernel's
    arithmetic variants (carry chains, 30-bit columns, precomputed products).  Two sampled
    images are compared bit for bit with the oracle on all five output ciphertexts: image 41
    (second of its image pair, first thread half of its CTA of four) and image 62 (first of
    its pair, second half), so that a slip in either slot shows; the oracle runs them side
    by side (about three CPU-minutes of oracle work each)."""
    import concurrent.futures
    import multiprocessing as mp
    from paper_2102_03494_gb300 import he
    prm = params.cfg_n15()
    shape = workloads.MNIST_LAYER
    lay_o, s, steps, keys, blob, xs, W1, W2, cts = setup_layer(prm, shape, "dp_shift_ext",
                                                               seed=5, B=64)
    sampled = (41, 62)
    with concurrent.futures.ProcessPoolExecutor(2, mp_context=mp.get_context("spawn")) as pool:
        jobs = [pool.submit(_oracle_layer, (prm, cts[b], W1, W2, lay_o, keys)) for b in sampled]
        ctx = make_ctx(prm)
        lay = ctx.layout(*shape.astuple(), pack="dp_shift_ext")
        ctx.he_load_keys(blob, gpu_steps(steps))
        ins = [upload_ntt(ctx, c) for c in cts]
        got = {}
        for arith in (0, 1, 2):
            ctx.he_tune_set(he.HE_TUNE_TAP_ARITH, arith)
            outs = ctx.he_ffconv_layer_batch(ins, W1, W2, lay)
            ctx.he_check()
            got[arith] = {b: [download_coeff(ctx, outs[b * shape.O_c + c]) for c in range(shape.O_c)]
                          for b in sampled}
        wants = {b: j.result() for b, j in zip(sampled, jobs)}
    for arith in (0, 1, 2):
        for b in sampled:
            for c in range(shape.O_c):
                assert (got[arith][b][c] == wants[b][c]).all(), (arith, b, c)
    check_decrypted(ctx, prm, s, lay_o, outs[41 * shape.O_c:42 * shape.O_c], xs[41], W1, W2)


@pytest.mark.parametrize("pack", ["dp_dot", "dp_shift", "dp_shift_ext", "cp_cp"])
def test_planned_layer_matches_the_plain_call(pack):
    """A layer plan (weights resident, W1 plaintexts encoded once) gives the oracle's bits,
    call after call; freeing it makes the id unknown."""
    prm = params.Params(log_n=9, n_q=3, n_p=1, alpha=1)
    shape = workloads.LayerShape(2, 6, 6, 3, 1, 1, 2, 2)
    lay_o, s, steps, keys, blob, xs, W1, W2, cts = setup_layer(prm, shape, pack, seed=4, B=2)
    ctx = make_ctx(prm)
    lay = ctx.layout(*shape.astuple(), pack=pack)
    ctx.he_load_keys(blob, gpu_steps(steps))
    plan = ctx.he_ffconv_plan(W1, W2, lay)
    K = shape.d * shape.d * shape.I_c if pack == "cp_cp" else 1
    want = [ffconv.he_layer(prm, cts[b * K:(b + 1) * K] if pack == "cp_cp" else cts[b], W1, W2,
                            lay_o, keys) for b in range(2)]
    for _ in range(2):
        outs = ctx.he_ffconv_layer_planned(plan, [upload_ntt(ctx, c) for c in cts], lay)
        for b in range(2):
            for c in range(shape.O_c):
                assert (download_coeff(ctx, outs[b * shape.O_c + c]) == want[b][c].stack()).all()
    ctx.he_ffconv_plan_free(plan)
    from paper_2102_03494_gb300 import he
    with pytest.raises(he.HeError):
        ctx.he_ffconv_layer_planned(plan, [upload_ntt(ctx, c) for c in cts], lay)


@pytest.mark.parametrize("pack", ["dp_dot", "dp_shift", "dp_shift_ext", "cp_cp"])
def test_captured_layer_replays_bit_exact(pack):
    """A planned layer captured into a CUDA graph: the capture call, every replay and a replay
    on new inputs written into the bound buffers give the oracle's bits, also after another
    call grew the context's own scratch; a graph recorded on the context's scratch works
    until a call regrows it; freeing the graph or its plan ends its replays."""
    from paper_2102_03494_gb300 import he
    prm = params.Params(log_n=9, n_q=3, n_p=1, alpha=1)
    shape = workloads.LayerShape(2, 6, 6, 3, 1, 1, 2, 2)
    lay_o, s, steps, keys, blob, xs, W1, W2, cts = setup_layer(prm, shape, pack, seed=5, B=2)
    ctx = make_ctx(prm)
    lay = ctx.layout(*shape.astuple(), pack=pack)
    ctx.he_load_keys(blob, gpu_steps(steps))
    plan = ctx.he_ffconv_plan(W1, W2, lay)
    K = shape.d * shape.d * shape.I_c if pack == "cp_cp" else 1
    img = [cts[b * K:(b + 1) * K] if pack == "cp_cp" else [cts[b]] for b in range(2)]
    want = [ffconv.he_layer(prm, img[b] if pack == "cp_cp" else img[b][0], W1, W2, lay_o, keys)
            for b in range(2)]

    def check(outs, order):
        for b in range(2):
            for c in range(shape.O_c):
                got = download_coeff(ctx, outs[b * shape.O_c + c])
                assert (got == want[order[b]][c].stack()).all(), (b, c)

    ins = [upload_ntt(ctx, c) for c in cts]
    n0 = ctx.he_launch_count()
    gid, outs = ctx.he_ffconv_graph_create(plan, ins, lay)
    per_call = ctx.he_launch_count() - n0
    check(outs, [0, 1])
    for o in outs:
        o.zero_()
    n1 = ctx.he_launch_count()
    ctx.he_graph_launch(gid)
    assert ctx.he_launch_count() - n1 == per_call     # the replay counts the captured kernels
    check(outs, [0, 1])
    # new inputs in the bound buffers: the two images swapped
    for b in range(2):
        for k in range(K):
            ins[b * K + k].copy_(upload_ntt(ctx, img[1 - b][k]))
    ctx.he_graph_launch(gid)
    check(outs, [1, 0])
    # a larger uncaptured call regrows the context scratch; the graph keeps its own
    ctx.he_ffconv_layer_batch([upload_ntt(ctx, c) for c in cts * 3], W1, W2, lay)
    for b in range(2):
        for k in range(K):
            ins[b * K + k].copy_(upload_ntt(ctx, img[b][k]))
    ctx.he_graph_launch(gid)
    check(outs, [0, 1])
    ctx.he_graph_free(gid)
    with pytest.raises(he.HeError):
        ctx.he_graph_launch(gid)
    # recorded on the context's scratch: valid until a call regrows it
    gid2, _ = ctx.he_ffconv_graph_create(plan, ins, lay, outs=outs, share_scratch=True)
    for o in outs:
        o.zero_()
    ctx.he_graph_launch(gid2)
    check(outs, [0, 1])
    ctx.he_ffconv_layer_batch([upload_ntt(ctx, c) for c in cts * 10], W1, W2, lay)
    with pytest.raises(he.HeError):
        ctx.he_graph_launch(gid2)
    ctx.he_graph_free(gid2)
    gid3, _ = ctx.he_ffconv_graph_create(plan, ins, lay, outs=outs)
    ctx.he_ffconv_plan_free(plan)
    with pytest.raises(he.HeError):
        ctx.he_graph_launch(gid3)
    ctx.he_graph_free(gid3)


def test_autotuned_tap_tile_and_arithmetic_keep_the_bits():
    """he_autotune times the tap kernel's tiles and arithmetic variants and keeps one pair;
    every forced pair gives the oracle's bits."""
    from paper_2102_03494_gb300 import he
    prm = params.Params(log_n=10, n_q=4, n_p=2, alpha=2)
    shape = workloads.LayerShape(2, 6, 6, 3, 1, 1, 3, 2)
    lay_o, s, steps, keys, blob, xs, W1, W2, cts = setup_layer(prm, shape, "dp_shift_ext", seed=9, B=3)
    ctx = make_ctx(prm)
    lay = ctx.layout(*shape.astuple(), pack="dp_shift_ext")
    ctx.he_load_keys(blob, gpu_steps(steps))
    rep = ctx.he_autotune(3)
    assert all(v > 0 for v in rep["tap_ms"].values()) and rep["ntt_ms"] > 0
    assert 1 <= rep["ntt_log2_n1"] < prm.log_n and rep["tap_tile"] in (128, 256)
    assert ctx.he_tune_get(he.HE_TUNE_TAP_TILE) == rep["tap_tile"]
    want = [ffconv.he_layer(prm, c, W1, W2, lay_o, keys) for c in cts]
    for tile in (128, 256):
        for arith in (0, 1, 2):
            ctx.he_autotune(3, force_tile=tile)
            ctx.he_tune_set(he.HE_TUNE_TAP_ARITH, arith)
            outs = ctx.he_ffconv_layer_batch([upload_ntt(ctx, c) for c in cts], W1, W2, lay)
            for b in range(3):
                for c in range(shape.O_c):
                    assert (download_coeff(ctx, outs[b * shape.O_c + c]) == want[b][c].stack()).all()
    # the ModUp / ModDown conversions with their target limbs split over 1, 2 and 4 groups
    assert rep["limb_groups"] in (1, 2, 4) and all(v > 0 for v in rep["conversion_ms"].values())
    ctx.he_tune_set(he.HE_TUNE_TAP_ARITH, 0)
    ctx.he_tune_set(he.HE_TUNE_BCONV_FUSED, 0)        # limb groups apply to the separate kernels
    for groups in (1, 2, 4):
        ctx.he_tune_set(he.HE_TUNE_LIMB_GROUPS, groups)
        assert ctx.he_tune_get(he.HE_TUNE_LIMB_GROUPS) == groups
        outs = ctx.he_ffconv_layer_batch([upload_ntt(ctx, c) for c in cts], W1, W2, lay)
        for b in range(3):
            for c in range(shape.O_c):
                assert (download_coeff(ctx, outs[b * shape.O_c + c]) == want[b][c].stack()).all()
        st = gpu_steps(steps)[0]
        got = ctx.he_rotate(upload_ntt(ctx, cts[0]), st)
        assert (download_coeff(ctx, got) == bfv.rotate(prm, cts[0], steps[0], keys).stack()).all()
    # the base conversions as separate kernels and inside the NTT's first pass
    assert rep["bconv"] in ("separate", "fused") and all(v > 0 for v in rep["bconv_ms"].values())
    ctx.he_tune_set(he.HE_TUNE_LIMB_GROUPS, 1)
    for fused in (0, 1):
        ctx.he_tune_set(he.HE_TUNE_BCONV_FUSED, fused)
        assert ctx.he_tune_get(he.HE_TUNE_BCONV_FUSED) == fused
        outs = ctx.he_ffconv_layer_batch([upload_ntt(ctx, c) for c in cts], W1, W2, lay)
        for b in range(3):
            for c in range(shape.O_c):
                assert (download_coeff(ctx, outs[b * shape.O_c + c]) == want[b][c].stack()).all()
        st = gpu_steps(steps)[0]
        got = ctx.he_rotate(upload_ntt(ctx, cts[0]), st)
        assert (download_coeff(ctx, got) == bfv.rotate(prm, cts[0], steps[0], keys).stack()).all()
    with pytest.raises(he.HeError):
        ctx.he_tune_set(he.HE_TUNE_BCONV_FUSED, 2)
    with pytest.raises(he.HeError):
        ctx.he_autotune(3, force_tile=64)
    with pytest.raises(he.HeError):
        ctx.he_tune_set(he.HE_TUNE_TAP_ARITH, 3)
    with pytest.raises(he.HeError):
        ctx.he_tune_set(he.HE_TUNE_LIMB_GROUPS, 3)


@pytest.mark.parametrize("q_bits,p_bits,n_q,n_p,alpha",
                         [(58, 57, 3, 2, 1), (60, 59, 3, 2, 1), (50, 60, 6, 1, 1), (52, 56, 5, 1, 1)],
                         ids=["q58-p57", "q60-p59", "six-digits", "five-digits-p56"])
def test_tap_kernel_on_wide_primes_and_many_digits(q_bits, p_bits, n_q, n_p, alpha):
    """The tap kernel's column arithmetic has separate branches for ciphertext primes of 55 bits
    or more (no lazy sums), for special primes not just below 2^60 and for keys of more than
    four digits (a mid-sum normalisation); each gives the oracle's bits, as do the carry
    chains and (where every ciphertext prime is below 2^50) the precomputed products."""
    from paper_2102_03494_gb300 import he
    prm = params.Params(log_n=9, n_q=n_q, n_p=n_p, alpha=alpha, q_bits=q_bits, p_bits=p_bits)
    shape = SMALL[0]
    lay_o, s, steps, keys, blob, xs, W1, W2, cts = setup_layer(prm, shape, "dp_shift_ext", seed=5, B=2)
    ctx = make_ctx(prm)
    ctx.he_load_keys(blob, gpu_steps(steps))
    lay = ctx.layout(*shape.astuple(), pack="dp_shift_ext")
    want = [ffconv.he_layer(prm, c, W1, W2, lay_o, keys) for c in cts]
    for arith in (1, 0, 2):
        ctx.he_tune_set(he.HE_TUNE_TAP_ARITH, arith)
        outs = ctx.he_ffconv_layer_batch([upload_ntt(ctx, c) for c in cts], W1, W2, lay)
        for b in range(2):
            for c in range(shape.O_c):
                assert (download_coeff(ctx, outs[b * shape.O_c + c]) == want[b][c].stack()).all()


@pytest.mark.parametrize("B", [1, 2])
def test_cp_cp_layers_are_bit_exact(B):
    """CP-HI2C-CP (Table VI's TinyNet packing) on small rings and at the TinyNet-shaped layer
    (28 x 28 input, 8 x 8 stride-2 pad-1 filters, 13 -> 56 channels) at N = 8192."""
    for prm, shape in [(params.Params(log_n=9, n_q=3, n_p=1, alpha=1), workloads.LayerShape(2, 6, 6, 3, 1, 1, 3, 2)),
                       (params.cfg_small_layer(), workloads.LayerShape(1, 28, 28, 8, 2, 1, 13, 56))]:
        lay_o, s, steps, keys, blob, xs, W1, W2, cts = setup_layer(prm, shape, "cp_cp", seed=3, B=B)
        assert steps == []
        ctx = make_ctx(prm)
        lay = ctx.layout(*shape.astuple(), pack="cp_cp")
        ctx.he_reset_op_counts()
        outs = ctx.he_ffconv_layer_batch([upload_ntt(ctx, c) for c in cts], W1, W2, lay)
        K = shape.d * shape.d * shape.I_c
        for b in range(B):
            ops = ffconv.OpCount()
            want = ffconv.he_layer(prm, cts[b * K:(b + 1) * K], W1, W2, lay_o, {}, ops)
            for c in range(shape.O_c):
                assert (download_coeff(ctx, outs[b * shape.O_c + c]) == want[c].stack()).all()
            check_decrypted(ctx, prm, s, lay_o, outs[b * shape.O_c:(b + 1) * shape.O_c], xs[b], W1, W2)
        got = ctx.he_op_counts()
        assert got["rot"] == 0 and got["mulpc"] == B * ops.mulpc
