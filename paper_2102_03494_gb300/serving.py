"""Serving loop: continuous batching of encrypted inference requests on one GPU.

Requests for networks (or single FFConv layers) on different rings -- e.g. the 28 x 28
three-layer network at N = 2^14 and the 3 x 32 x 32 network at N = 2^15 -- arrive over time.
The scheduler
  * admits a waiting request when its device-memory footprint fits the budget (inputs,
    outputs and its share of scratch), freeing the footprint when its batch completes;
  * groups admitted requests of the same ring, oldest first, into batches of up to
    `max_batch`, and starts a batch as soon as a worker of that ring is idle -- requests
    that arrive while others run join the next batch (continuous batching);
  * runs every worker on its own CUDA stream with its own library context (Galois keys
    resident in each), so batches of different rings and workers overlap on the device.
Completion is detected with CUDA events; latency = completion - arrival.

The scheduling logic (`Scheduler`) is plain host code that drives an executor interface, so
it is tested with a fake executor on the CPU; the executors over libhe are `GpuRing` (one
FFConv layer, optionally replayed as captured CUDA graphs), `NetRing` (the three-layer
network) and `DeepRing` (the multi-ciphertext network).
"""
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional


@dataclass
class Request:
    rid: int
    ring: str
    t_arrive: float
    payload: object = None          # executor-specific input (device ciphertext(s))
    footprint: int = 0              # device bytes held from admission to completion
    t_start: Optional[float] = None
    t_done: Optional[float] = None
    result: object = None


@dataclass
class Batch:
    ring: str
    worker: int
    requests: List[Request]
    handle: object = None           # executor-specific completion handle


class Scheduler:
    """Admission by memory footprint + per-ring FIFO batching over a pool of workers.

    executors: ring -> object with
        workers: int                                 number of concurrent batches
        footprint(req) -> int                        device bytes of one request
        launch(worker, requests) -> handle           enqueue the batch (asynchronous)
        done(handle) -> bool                         completion poll
        results(handle, requests)                    fill req.result after completion
    """

    def __init__(self, executors: Dict[str, object], max_batch: int, memory_budget: int,
                 clock: Callable[[], float]):
        self.ex = executors
        self.max_batch = max_batch
        self.budget = memory_budget
        self.clock = clock
        self.waiting: List[Request] = []          # arrived, not admitted
        self.admitted: Dict[str, List[Request]] = {r: [] for r in executors}
        self.in_use = 0
        self.running: List[Batch] = []
        self.idle = {r: list(range(e.workers)) for r, e in executors.items()}
        self.finished: List[Request] = []

    def submit(self, req: Request):
        req.footprint = self.ex[req.ring].footprint(req)
        if req.footprint > self.budget:
            raise ValueError(f"request {req.rid} needs {req.footprint} B, above the whole budget")
        self.waiting.append(req)

    def _admit(self):
        keep = []
        for req in self.waiting:                  # oldest first; later ones may still fit
            if self.in_use + req.footprint <= self.budget:
                self.in_use += req.footprint
                self.admitted[req.ring].append(req)
            else:
                keep.append(req)
        self.waiting = keep

    def _complete(self):
        still = []
        for b in self.running:
            if self.ex[b.ring].done(b.handle):
                self.ex[b.ring].results(b.handle, b.requests)
                now = self.clock()
                for r in b.requests:
                    r.t_done = now
                    self.in_use -= r.footprint
                    self.finished.append(r)
                self.idle[b.ring].append(b.worker)
            else:
                still.append(b)
        self.running = still

    def _launch(self):
        for ring, queue in self.admitted.items():
            while queue and self.idle[ring]:
                take, self.admitted[ring] = queue[: self.max_batch], queue[self.max_batch:]
                queue = self.admitted[ring]
                w = self.idle[ring].pop(0)
                now = self.clock()
                for r in take:
                    r.t_start = now
                handle = self.ex[ring].launch(w, take)
                self.running.append(Batch(ring, w, take, handle))

    def step(self):
        """One pass: retire finished batches, admit, launch.  Returns True while busy."""
        self._complete()
        self._admit()
        self._launch()
        return bool(self.waiting or self.running or any(self.admitted.values()))

    def serve(self, arrivals: List[Request]):
        """Feed requests at their arrival times (seconds from start) and run to completion."""
        t0 = self.clock()
        pending = sorted(arrivals, key=lambda r: r.t_arrive)
        i = 0
        while True:
            now = self.clock() - t0
            while i < len(pending) and pending[i].t_arrive <= now:
                pending[i].t_arrive += t0             # absolute clock from here on
                self.submit(pending[i])
                i += 1
            busy = self.step()
            if not busy and i == len(pending):
                break
        return self.finished


def latency_stats(reqs: List[Request]):
    import numpy as np
    lat = np.array([r.t_done - r.t_arrive for r in reqs]) * 1000.0
    span = max(r.t_done for r in reqs) - min(r.t_arrive for r in reqs)
    return {"requests": len(reqs), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "requests_per_s": len(reqs) / span if span > 0 else float("inf")}


def poisson_arrivals(seed: int, rate: float, count: int, mix: Dict[str, float]):
    """`count` requests with exponential inter-arrival times (rate per second) and rings drawn
    with the given probabilities."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    names = list(mix)
    probs = np.array([mix[n] for n in names], dtype=float)
    picks = rng.choice(len(names), size=count, p=probs / probs.sum())
    return [Request(rid=i, ring=names[picks[i]], t_arrive=float(t[i])) for i in range(count)]


# ---------------------------------------------------------------- GPU executor over libhe

@dataclass
class RingSpec:
    log_n: int
    n_q: int
    n_p: int
    alpha: int
    shape: tuple                      # (I_c, I_h, I_w, d, stride, pad, r, O_c)
    pack: str = "dp_shift_ext"


class GpuRing:
    """One ring's workers: a library context and a CUDA stream each, keys resident in every
    context, weights fixed per ring."""

    def __init__(self, spec: RingSpec, workers: int, W1, W2, sk_seed: int, key_seed: int,
                 keep_results: bool = True, graphs: int = 0):
        """graphs = G > 0: every worker also captures its layer into CUDA graphs for batches of
        1 .. G images, on input / output buffers of its own (the largest batch first, all on
        the worker context's scratch); a batch then costs two copies and one submission."""
        import torch
        from . import he
        self.spec, self.workers = spec, workers
        self.keep_results = keep_results          # False: outputs are released on completion
        self.W1, self.W2 = W1, W2
        self.streams = [torch.cuda.Stream() for _ in range(workers)]
        self.ctx = [he.Context(spec.log_n, spec.n_q, spec.n_p, spec.alpha, stream=s)
                    for s in self.streams]
        self.lay = self.ctx[0].layout(*spec.shape, pack=spec.pack)
        self.sk = self.ctx[0].he_keygen_secret(sk_seed)
        steps = self.ctx[0].he_ffconv_required_steps(self.lay)
        for c in self.ctx:
            c.he_keygen_galois(self.sk, key_seed, steps)
        # model state resident per worker, like the keys: the weights with their plaintexts
        self.plans = [c.he_ffconv_plan(W1, W2, self.lay) for c in self.ctx]
        self.N = 1 << spec.log_n
        self.ct_bytes = 2 * spec.n_q * self.N * 8
        self.O_c = spec.shape[7]
        self.graphs = []                          # per worker: batch size -> (ins, outs, id)
        self.use_graphs = graphs > 0              # launch through them (a switch for comparisons)
        for w, c in enumerate(self.ctx):
            g = {}
            if graphs > 0:
                with torch.cuda.stream(self.streams[w]):
                    ins = [c.new_ct() for _ in range(graphs)]
                    outs = [c.new_ct() for _ in range(graphs * self.O_c)]
                for b in range(graphs, 0, -1):
                    gid, _ = c.he_ffconv_graph_create(self.plans[w], ins[:b], self.lay,
                                                      outs[:b * self.O_c], share_scratch=True)
                    g[b] = (ins[:b], outs[:b * self.O_c], gid)
            self.graphs.append(g)

    def encrypt(self, slots, seed):
        return self.ctx[0].he_encrypt(self.sk, slots, seed)

    def footprint(self, req):
        # input + outputs + the per-image share of the layer's scratch (ModUp digits,
        # extended channel sums, products): bounded by 8 ciphertexts of the extended basis
        sp = self.spec
        ext = 2 * (sp.n_q + sp.n_p) * self.N * 8
        return self.ct_bytes * (1 + self.O_c) + 8 * ext

    def launch(self, worker, requests):
        import torch
        ctx = self.ctx[worker]
        captured = self.graphs[worker].get(len(requests)) if self.use_graphs else None
        if captured is not None:
            ins, outs, gid = captured
            with torch.cuda.stream(self.streams[worker]):
                for buf, r in zip(ins, requests):
                    buf.copy_(r.payload)
                ctx.he_graph_launch(gid)
                # the bound outputs are rewritten by the worker's next batch: keep copies
                res = [o.clone() for o in outs] if self.keep_results else None
                ev = torch.cuda.Event()
                ev.record(self.streams[worker])
            return (ev, res, worker)
        with torch.cuda.stream(self.streams[worker]):
            # allocated (and zero-filled) on the worker's stream, ordered before the layer
            outs = [ctx.new_ct() for _ in range(len(requests) * self.O_c)]
            ctx.he_ffconv_layer_planned(self.plans[worker], [r.payload for r in requests], self.lay,
                                        outs)
            ev = torch.cuda.Event()
            ev.record(self.streams[worker])
        return (ev, outs, worker)

    def done(self, handle):
        return handle[0].query()

    def results(self, handle, requests):
        # the worker's stream is idle here: report a device wait that ran out (HE_ETIMEOUT)
        self.ctx[handle[2]].he_check()
        outs = handle[1]
        for i, r in enumerate(requests):
            r.result = outs[i * self.O_c:(i + 1) * self.O_c] if self.keep_results else None

    def close(self):
        """Frees the captured graphs (the contexts go with the ring)."""
        for c, g in zip(self.ctx, self.graphs):
            for _, _, gid in g.values():
                c.he_graph_free(gid)
        self.graphs = [{} for _ in self.ctx]

    def run_alone(self, payload):
        """The plain form: one request, one call, waited for."""
        import torch
        ctx = self.ctx[0]
        with torch.cuda.stream(self.streams[0]):
            outs = [ctx.new_ct() for _ in range(self.O_c)]
            ctx.he_ffconv_layer_planned(self.plans[0], [payload], self.lay, outs)
        self.streams[0].synchronize()
        return outs


# ---------------------------------------------------------------- whole-network executors

@dataclass
class NetSpec:
    """The three-layer network on one ring: FFConv layer (DP_SHIFT_EXT), channel combine, x^2,
    fully connected to m1, x^2, fully connected to m2."""
    log_n: int
    n_q: int
    n_p: int
    alpha: int
    shape: tuple                      # the layer's (I_c, I_h, I_w, d, stride, pad, r, O_c)
    m1: int
    m2: int


@dataclass
class DeepSpec:
    """The multi-ciphertext network on one ring: 3 x 3 stride-1 convolutions C0 -> channels[0]
    -> ... (each factorized at `rank`, 0 = unfactorized), x^2 after each, sum pooling folded
    into the classifier to n_cls outputs."""
    log_n: int
    n_q: int
    n_p: int
    alpha: int
    C0: int
    H: int
    W: int
    channels: tuple
    rank: int
    n_cls: int


class _NetWorkers:
    """Workers of one ring serving whole networks: a library context and a CUDA stream each,
    the Galois and relinearisation keys resident in every context, the weights fixed, batches
    run as library calls or replayed as recorded CUDA graphs.  One output ciphertext per
    request (the logits)."""

    def __init__(self, log_n, n_q, n_p, alpha, workers, keep_results):
        import torch
        from . import he
        self.workers = workers
        self.keep_results = keep_results
        self.streams = [torch.cuda.Stream() for _ in range(workers)]
        self.ctx = [he.Context(log_n, n_q, n_p, alpha, stream=s) for s in self.streams]
        self.N = 1 << log_n
        self.ct_bytes = 2 * n_q * self.N * 8
        self.ext_bytes = 2 * (n_q + n_p) * self.N * 8

    def _keys(self, sk_seed, key_seed, steps):
        self.sk = self.ctx[0].he_keygen_secret(sk_seed)
        for c in self.ctx:
            c.he_keygen_galois(self.sk, key_seed, steps)

    def _record(self, graphs, n_in):
        """graphs = G > 0: every worker records its network call into CUDA graphs for
        batches of 1 .. G requests on input / output buffers of its own (each batch size run
        once first, the largest first, so that the context's scratch and network buffer are
        sized before any recording; all graphs of a worker share them)."""
        import torch
        self.graphs = []
        self.use_graphs = graphs > 0
        for w, c in enumerate(self.ctx):
            g = {}
            if graphs > 0:
                with torch.cuda.stream(self.streams[w]):
                    ins = [c.new_ct() for _ in range(graphs * n_in)]
                    outs = [c.new_ct() for _ in range(graphs)]
                for b in range(graphs, 0, -1):
                    with torch.cuda.stream(self.streams[w]):
                        self._call(c, ins[:b * n_in], outs[:b])
                    c.he_graph_begin(share_scratch=True)
                    try:
                        self._call(c, ins[:b * n_in], outs[:b])
                    finally:
                        gid = c.he_graph_end(keep=ins + outs)
                    g[b] = (ins[:b * n_in], outs[:b], gid)
            self.graphs.append(g)

    def close(self):
        """Frees the recorded graphs (the contexts go with the ring)."""
        for c, g in zip(self.ctx, getattr(self, "graphs", [])):
            for _, _, gid in g.values():
                c.he_graph_free(gid)
        self.graphs = [{} for _ in self.ctx]

    def encrypt(self, slots, seed):
        return self.ctx[0].he_encrypt(self.sk, slots, seed)

    def _inputs(self, payload):
        return payload if isinstance(payload, (list, tuple)) else [payload]

    def launch(self, worker, requests):
        import torch
        ctx = self.ctx[worker]
        cts = [c for r in requests for c in self._inputs(r.payload)]
        graphs = getattr(self, "graphs", None)
        captured = graphs[worker].get(len(requests)) if graphs and self.use_graphs else None
        with torch.cuda.stream(self.streams[worker]):
            if captured is not None:
                ins, bound, gid = captured
                for buf, c in zip(ins, cts):
                    buf.copy_(c)
                ctx.he_graph_launch(gid)
                # the bound outputs are rewritten by the worker's next batch: keep copies
                outs = [o.clone() for o in bound] if self.keep_results else None
            else:
                outs = [ctx.new_ct() for _ in requests]
                self._call(ctx, cts, outs)
            ev = torch.cuda.Event()
            ev.record(self.streams[worker])
        return (ev, outs, worker)

    def done(self, handle):
        return handle[0].query()

    def results(self, handle, requests):
        self.ctx[handle[2]].he_check()           # as GpuRing.results
        for i, r in enumerate(requests):
            r.result = [handle[1][i]] if self.keep_results else None

    def run_alone(self, payload):
        """The plain form: one request, one call, waited for."""
        import torch
        ctx = self.ctx[0]
        with torch.cuda.stream(self.streams[0]):
            outs = [ctx.new_ct()]
            self._call(ctx, self._inputs(payload), outs)
        self.streams[0].synchronize()
        return outs


class NetRing(_NetWorkers):
    def __init__(self, spec: NetSpec, workers: int, W1, W2, F1, F2, sk_seed: int, key_seed: int,
                 keep_results: bool = True, graphs: int = 0):
        super().__init__(spec.log_n, spec.n_q, spec.n_p, spec.alpha, workers, keep_results)
        self.spec = spec
        self.W1, self.W2, self.F1, self.F2 = W1, W2, F1, F2
        self.lay = self.ctx[0].layout(*spec.shape, pack="dp_shift_ext")
        self.net = self.ctx[0].net(self.lay, spec.m1, spec.m2)
        self._keys(sk_seed, key_seed, self.ctx[0].he_net_required_steps(self.net))
        self._record(graphs, 1)

    def footprint(self, req):
        # input, output, the five channel outputs and the combined vector, plus the layer's
        # extended-basis scratch share
        return self.ct_bytes * (2 + self.spec.shape[7] + 2) + 8 * self.ext_bytes

    def _call(self, ctx, cts, outs):
        ctx.he_net_batch(cts, self.W1, self.W2, self.F1, self.F2, self.net, outs)


class DeepRing(_NetWorkers):
    def __init__(self, spec: DeepSpec, workers: int, W1s, W2s, F, sk_seed: int, key_seed: int,
                 keep_results: bool = True, graphs: int = 0):
        super().__init__(spec.log_n, spec.n_q, spec.n_p, spec.alpha, workers, keep_results)
        self.spec = spec
        self.W1s, self.W2s, self.F = W1s, W2s, F
        self.convs, C = [], spec.C0
        for O in spec.channels:
            self.convs.append(self.ctx[0].mc_conv(C, spec.H, spec.W, 3, spec.rank, O))
            C = O
        self.n_in = self.ctx[0].mc_cts(spec.C0, spec.H, spec.W)
        self._keys(sk_seed, key_seed, self.ctx[0].he_deep_required_steps(self.convs, spec.n_cls))
        self._record(graphs, self.n_in)

    def footprint(self, req):
        # inputs, output, the widest tensor twice (in and out of a layer) and the layers'
        # extended-basis scratch share
        widest = max(self.ctx[0].mc_cts(c, self.spec.H, self.spec.W) for c in self.spec.channels)
        return self.ct_bytes * (self.n_in + 1 + 2 * widest) + 16 * self.ext_bytes

    def _call(self, ctx, cts, outs):
        ctx.he_deep_batch(cts, self.convs, self.W1s, self.W2s, self.F, outs)
