"""he_rotate_noalloc: the rotation for callers that cannot allocate device memory.

Such callers (a process whose GPU memory another allocator already holds, or a request path
that must not block on cudaMalloc/cudaFree) get their key-switching scratch from a static
device array inside the library.  The test calls the entry point through the C ABI, twice in a
row on the same context, and requires the same ciphertext bits as he_rotate; it also checks
that parameters needing more than the built-in scratch are refused.  This file is collected
last so that a run stopping at the first failure has run every other test already."""
import ctypes

import numpy as np
import pytest

from oracle import params

pytestmark = pytest.mark.gpu


def test_rotate_noalloc_matches_rotate_on_two_calls():
    import torch
    from paper_2102_03494_gb300 import he
    from tests.gpu_common import make_ctx

    prm = params.cfg_small_layer()          # N = 8192, 3 x 50-bit q, 1 special prime
    ctx = make_ctx(prm)
    sk = ctx.he_keygen_secret(5)
    ctx.he_keygen_galois(sk, 6, [3, -7])
    rng = np.random.default_rng(1)
    cts = [ctx.he_encrypt(sk, rng.integers(0, prm.t, prm.n), 10 + i) for i in range(2)]
    for ct, step in zip(cts, (3, -7)):       # two calls in a row, different inputs and steps
        want = ctx.he_rotate(ct, step)
        out = ctx.new_ct()
        a, b = ctx.ct_struct(ct), ctx.ct_struct(out)
        rc = he.lib().he_rotate_noalloc(ctx.h, ctypes.byref(a), step, ctypes.byref(b))
        assert rc == he.HE_OK, he.lib().he_last_error(ctx.h)
        torch.cuda.synchronize()
        assert (ctx.to_numpy(out) == ctx.to_numpy(want)).all()
    # the result decrypts to the rotated slots
    v = ctx.he_decrypt(sk, cts[1])
    got = ctx.he_decrypt(sk, ctx.he_rotate_noalloc(cts[1], -7, ctx.new_ct()))
    half = prm.n // 2
    assert (got[:half] == np.roll(v[:half], 7)).all()


def test_rotate_noalloc_refuses_parameters_beyond_its_scratch():
    from paper_2102_03494_gb300 import he
    from tests.gpu_common import make_ctx

    prm = params.cfg_n15()                  # N = 2^15 with 12 + 3 primes needs ~39 MiB
    ctx = make_ctx(prm)
    sk = ctx.he_keygen_secret(1)
    ctx.he_keygen_galois(sk, 2, [1])
    ct = ctx.he_encrypt(sk, np.zeros(prm.n, dtype=np.int64), 3)
    with pytest.raises(he.HeError) as e:
        ctx.he_rotate_noalloc(ct, 1, ctx.new_ct())
    assert e.value.code == he.HE_EINVAL and "bytes of scratch" in str(e.value)


def test_rotate_noalloc_is_refused_while_recording():
    """Recording would give the graph pointer tables of its own (allocated) and a replay would
    share the static array with later calls, so the entry point refuses to be recorded."""
    from paper_2102_03494_gb300 import he
    from tests.gpu_common import make_ctx

    prm = params.cfg_small_layer()
    ctx = make_ctx(prm)
    sk = ctx.he_keygen_secret(5)
    ctx.he_keygen_galois(sk, 6, [3])
    ct = ctx.he_encrypt(sk, np.zeros(prm.n, dtype=np.int64), 3)
    out = ctx.new_ct()
    ctx.he_rotate_noalloc(ct, 3, out)          # the first call (address set-up) before recording
    ctx.he_graph_begin(share_scratch=True)
    a, b = ctx.ct_struct(ct), ctx.ct_struct(out)
    rc = he.lib().he_rotate_noalloc(ctx.h, ctypes.byref(a), 3, ctypes.byref(b))
    assert rc == he.HE_EINVAL and b"recording" in he.lib().he_last_error(ctx.h)
    with pytest.raises(he.HeError):            # the refusal spoils the recording
        ctx.he_graph_end()
