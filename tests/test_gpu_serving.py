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


@pytest.mark.parametrize("graphs", [0, 4])
def test_networks_are_identical_alone_and_in_the_mix(graphs):
    """Whole networks served: the three-layer network (N = 2048, 1 x 12 x 12 -> 3 channels ->
    20 -> 4) and a multi-ciphertext network (N = 2048, 3 x 8 x 8 -> 20 -> 24 channels at rank
    4, 4 classes) on two rings, batches run as calls or replayed as recorded graphs; every
    result is bit-identical to the same request run alone and decrypts to the plain network
    mod t."""
    from oracle import deepnet, network
    from oracle.ffconv import Layout, input_slots
    rng = np.random.default_rng(17)
    lay = Layout(1, 12, 12, 3, 2, 1, 2, 3, pack="dp_shift_ext")
    m1, m2 = 20, 4
    W1 = rng.integers(-8, 9, (lay.r, lay.I_c, lay.d, lay.d))
    W2 = rng.integers(-8, 9, (lay.O_c, lay.r))
    F1 = rng.integers(-8, 9, (m1, lay.O_c * lay.S))
    F2 = rng.integers(-8, 9, (m2, m1))
    net_ring = serving.NetRing(serving.NetSpec(11, 4, 2, 2, (1, 12, 12, 3, 2, 1, 2, 3), m1, m2),
                               workers=2, W1=W1, W2=W2, F1=F1, F2=F2, sk_seed=31, key_seed=32,
                               graphs=graphs)
    shape = deepnet.DeepShape(3, 8, 8, [deepnet.ConvSpec(20, 4), deepnet.ConvSpec(24, 4)], n_cls=4)
    w = deepnet.rand_weights(shape, 5)
    deep_ring = serving.DeepRing(serving.DeepSpec(11, 5, 2, 2, 3, 8, 8, (20, 24), 4, 4), workers=2,
                                 W1s=[np.asarray(a, np.int32) for a, _ in w["convs"]],
                                 W2s=[np.asarray(b, np.int32) for _, b in w["convs"]],
                                 F=np.asarray(w["fc"], np.int32), sk_seed=41, key_seed=42,
                                 graphs=graphs)
    rings = {"net": net_ring, "deep": deep_ring}
    reqs = serving.poisson_arrivals(seed=5, rate=1000.0, count=20, mix={"net": 0.6, "deep": 0.4})
    images = {}
    for r in reqs:
        if r.ring == "net":
            images[r.rid] = x = rng.integers(0, 256, (1, 12, 12))
            r.payload = net_ring.encrypt(input_slots(x, lay, 2048), 600 + r.rid)
        else:
            images[r.rid] = x = rng.integers(0, 256, (3, 8, 8))
            r.payload = [deep_ring.encrypt(v, 700 + 10 * r.rid + i)
                         for i, v in enumerate(deepnet.pack_tensor(x, shape, 2048))]
    torch.cuda.synchronize()
    sched = serving.Scheduler(rings, max_batch=4, memory_budget=1 << 30, clock=serving_clock())
    done = sched.serve(reqs)
    torch.cuda.synchronize()
    assert len(done) == 20 and {r.ring for r in done} == {"net", "deep"}
    for r in done:
        ring = rings[r.ring]
        alone = ring.run_alone(r.payload)
        assert (ring.ctx[0].to_numpy(r.result[0]) == ring.ctx[0].to_numpy(alone[0])).all(), r.rid
        dec = ring.ctx[0].he_decrypt(ring.sk, r.result[0])
        if r.ring == "net":
            _, _, z2 = network.plain_net(images[r.rid], W1, W2, lay, F1, F2, 65537)
            for p in network.output_slots(m2, 2048):
                assert dec[p] == z2[p % network.next_pow2(m2)]
        else:
            _, logits = deepnet.plain_deep(images[r.rid], w, shape, 65537)
            assert (dec[:deepnet.next_pow2(shape.n_cls)][:shape.n_cls] == logits).all()
    for ring in rings.values():
        ring.close()
