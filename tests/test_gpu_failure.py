"""Failure detection on the GPU without a fault: a bounded device-side wait that is reported
reaches the caller as HE_ETIMEOUT, the error word is cleared by that report, and the next
call on the same context is clean and bit-exact.

The fused tap kernel's compute warps wait on an mbarrier for each shared-memory stage of
operands.  The test hook he_set_wait_report(0) makes every such wait report itself (error bit)
before its first poll, after which the warp still waits with the kernel's full bound: nothing
is skipped, no copy is left in flight, no wait is unbounded.  The check is he_check, which
the serving executors call for every finished batch and the benchmark after its timed
region."""
import pytest

from oracle import ffconv, params
from tests.gpu_common import download_coeff, gpu_steps, make_ctx, upload_ntt
from tests.test_gpu_layer import SMALL, setup_layer

pytestmark = pytest.mark.gpu


def test_reported_wait_gives_etimeout_then_a_clean_bit_exact_call():
    from paper_2102_03494_gb300 import he
    prm = params.Params(log_n=9, n_q=3, n_p=1, alpha=1)     # N = 512: the bulk-copy tap kernel
    shape = SMALL[0]
    lay_o, s, steps, keys, blob, xs, W1, W2, cts = setup_layer(prm, shape, "dp_shift_ext", seed=4)
    ctx = make_ctx(prm)
    ctx.he_load_keys(blob, gpu_steps(steps))
    lay = ctx.layout(*shape.astuple(), pack="dp_shift_ext")
    want = ffconv.he_layer(prm, cts[0], W1, W2, lay_o, keys)
    x = upload_ntt(ctx, cts[0])
    ctx.he_check()                                          # nothing reported so far

    ctx.he_set_wait_report(0)
    ctx.he_ffconv_layer(x, W1, W2, lay)
    with pytest.raises(he.HeError) as e:
        ctx.he_check()
    assert e.value.code == he.HE_ETIMEOUT
    ctx.he_check()                                          # the report cleared the word

    ctx.he_set_wait_report(-1)
    outs = ctx.he_ffconv_layer(x, W1, W2, lay)
    ctx.he_check()
    for o, w in zip(outs, want):
        assert (download_coeff(ctx, o) == w.stack()).all()


def test_wait_report_hook_is_refused_while_recording():
    from paper_2102_03494_gb300 import he
    ctx = make_ctx(params.Params(log_n=9, n_q=3, n_p=1, alpha=1))
    ctx.he_graph_begin(share_scratch=True)
    try:
        with pytest.raises(he.HeError) as e:
            ctx.he_set_wait_report(0)
        assert e.value.code == he.HE_EINVAL
        with pytest.raises(he.HeError):
            ctx.he_check()
    finally:
        with pytest.raises(he.HeError):                     # the refusals spoil the recording
            ctx.he_graph_end()
