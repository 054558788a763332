"""Serving loop on the GPU: requests for two rings arrive over time and are batched
continuously across worker streams (plain calls or captured CUDA graphs); every result is
bit-identical to the same request run alone (one image per call) and decrypts to the plain
layer."""
import numpy as np
import pytest
import torch

from oracle import ffconv
from paper_2102_03494_gb300 import serving, workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("graphs", [0, 4])
def test_results_are_identical_alone_and_in_the_mix(graphs):
    """graphs = 4: every batch runs as a captured CUDA graph of its size."""
    specs = {"a": serving.RingSpec(10, 3, 1, 1, (1, 8, 8, 3, 2, 1, 2, 3)),
             "b": serving.RingSpec(11, 4, 2, 2, (2, 6, 6, 3, 1, 1, 2, 2))}
    rings, weights = {}, {}
    for i, (name, sp) in enumerate(specs.items()):
        shape = workloads.LayerShape(*sp.shape)
        W1, W2 = workloads.weights(i, shape)
        weights[name] = (shape, W1, W2)
        rings[name] = serving.GpuRing(sp, workers=2, W1=W1, W2=W2, sk_seed=10 + i, key_seed=20 + i,
                                      graphs=graphs)
    reqs = serving.poisson_arrivals(seed=3, rate=2000.0, count=24, mix={"a": 0.5, "b": 0.5})
    images = {}
    for r in reqs:
        shape = weights[r.ring][0]
        x = workloads.image(100 + r.rid, shape)
        lay = ffconv.Layout(*shape.astuple(), pack="dp_shift_ext")
        images[r.rid] = x
        r.payload = rings[r.ring].encrypt(ffconv.input_slots(x, lay, 1 << specs[r.ring].log_n), 500 + r.rid)
    torch.cuda.synchronize()
    sched = serving.Scheduler(rings, max_batch=4, memory_budget=1 << 30, clock=serving_clock())
    done = sched.serve(reqs)
    torch.cuda.synchronize()
    assert len(done) == 24
    for r in done:
        ring = rings[r.ring]
        alone = ring.run_alone(r.payload)
        for got, want in zip(r.result, alone):
            assert (ring.ctx[0].to_numpy(got) == ring.ctx[0].to_numpy(want)).all()
        shape, W1, W2 = weights[r.ring]
        lay = ffconv.Layout(*shape.astuple(), pack="dp_shift_ext")
        _, y2 = ffconv.plain_layer(images[r.rid], W1, W2, lay)
        v = ring.ctx[0].he_decrypt(ring.sk, r.result[0])
        for oh in range(lay.O_h):
            for ow in range(lay.O_w):
                assert v[ffconv.output_slot(lay, oh, ow)] == y2[0, oh, ow] % 65537
    stats = serving.latency_stats(done)
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    for ring in rings.values():
        ring.close()


def serving_clock():
    import time
    return time.perf_counter
