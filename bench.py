"""Benchmark: the encrypted FFConv layer at N = 2^15 on one GB300 (or N replicas).

One step = one encrypted FFConv layer (DP_SHIFT_EXT schedule: 24 hoisted rotations of each
input key-switched and multiplied by the tap plaintexts in the extended basis, one ModDown per
channel, ConvPack restore) over a batch of B encrypted 1 x 28 x 28 images (B = 64 by default,
the batched size of the layer workload; B = 1 latencies are reported beside it), RNS-BFV with
N = 2^15, 12 x 50-bit ciphertext primes, 3 x 60-bit special primes, key-switching digits of
3 primes.  Inputs are seeded synthetic images (pixels uniform in [0, 255]) and weights
(uniform in [-8, 8]) standing in for MNIST and trained weights.

The headline value is hoisted rotations per second over the whole job (B * 24 per step and
GPU); the layer latency is reported beside it.  `--impl reference` times the CPU oracle on a
bounded sample of the same work (the paper ships no implementation).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encrypted FFConv-layer latency (ms) & hoisted rotations/sec at N=2^15; HBM roofline %"
UNIT = "hoisted rotations/s"
LOG_N, N_Q, N_P, ALPHA = 15, 12, 3, 3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--pack", default="dp_shift_ext", choices=["dp_shift", "dp_shift_ext", "dp_dot"])
    ap.add_argument("--tap-arith", default="auto", choices=["auto", "chains", "columns", "products"],
                    help="force the fused tap kernel's arithmetic after autotuning")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-baseline-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the short network runs reported under 'also'")
    ap.add_argument("--serving-layers", action="store_true",
                    help="serving loop over single FFConv layers (28 x 28 at N = 2^14, 3 x 32 x 32 "
                         "at N = 2^15) instead of whole networks")
    ap.add_argument("--sweep", nargs="?", const="full", default=None, choices=["full", "short"],
                    help="batched primitive sweep (NTT, automorphism, plain and hoisted rotations "
                         "over B, N, L); 'short' = N=2^15, L=16, B in {16, 256}")
    ap.add_argument("--packing", action="store_true",
                    help="Table IX: the packing variants on WideNet's factorized second layer")
    ap.add_argument("--serving-rates", default="20,60,120,240",
                    help="offered request rates (per second) of --serving")
    ap.add_argument("--serving-count", type=int, default=0,
                    help="requests per rate of --serving (0: 3 s of arrivals, 60 .. 480)")
    ap.add_argument("--ntt", action="store_true",
                    help="forward and inverse NTT of 64 ciphertexts' c1 (64 x 12 limbs) at N=2^15, "
                         "default split and radix (the case the NTT profiles capture)")
    ap.add_argument("--single", action="store_true",
                    help="one-image latency of the 1x28x28 layer at N=8192, 3+1 primes, for the "
                         "DP_DOT, DP_SHIFT and DP_SHIFT_EXT schedules")
    ap.add_argument("--serving", action="store_true",
                    help="run the serving loop (mixed rings, Poisson arrivals) instead")
    ap.add_argument("--net", action="store_true",
                    help="time the three-layer network (batch --net-batch, N=2^14) instead")
    ap.add_argument("--net-batch", type=int, default=64)
    ap.add_argument("--deep", action="store_true",
                    help="time the deeper 3x32x32 network (factorized ranks vs unfactorized)")
    ap.add_argument("--deep-batch", type=int, default=16)
    ap.add_argument("--deep-ranks", default="8,16,32,0",
                    help="comma-separated ranks to time (0 = unfactorized)")
    return ap.parse_args()


def max_over_ranks(values, device):
    """Element-wise maximum of `values` over all ranks (the slowest replica sets the time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def check_line(line):
    """The bench line's contract keys and their types (raises ValueError on a malformed line)."""
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "dtype", "config", "e2e", "gpu_launches", "clocks"):
        if k not in line:
            raise ValueError(f"bench line without {k!r}")
    clk = line["clocks"]
    if not isinstance(clk, dict) or not {"sm_mhz", "sm_max_mhz", "reasons"} <= set(clk):
        raise ValueError(f"bench line clocks must be an object with sm_mhz, sm_max_mhz, reasons: {clk!r}")
    if not isinstance(line["e2e"], dict) or "value" not in line["e2e"]:
        raise ValueError("bench line e2e must be an object with a value")
    return line


def whole_job_rate(units_per_rank, world, ms_max):
    """Units processed by all replicas per second, timed by the slowest replica."""
    return world * units_per_rank / (ms_max / 1000.0)


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


# ---------------------------------------------------------------- CPU oracle sample

_ORACLE = {}


def _oracle_layer_setup():
    """Per-process, untimed set-up of the oracle's layer: the ring, the secret and the layer's
    24 Galois keys (seeds of rank 0's GPU arm), the weights."""
    from oracle import bfv, ffconv, params
    from paper_2102_03494_gb300 import workloads
    if _ORACLE:
        return _ORACLE
    prm = params.Params(log_n=LOG_N, n_q=N_Q, n_p=N_P, alpha=ALPHA)
    shape = workloads.MNIST_LAYER
    lay = ffconv.Layout(*shape.astuple(), pack="dp_shift_ext")
    s = bfv.keygen_secret(prm, 1000)
    steps = ffconv.required_steps(lay, prm.n)
    keys = {}
    for st in steps:
        g = bfv.galois_of(st, prm.n)
        keys[g] = bfv.galois_key(prm, s, g, 2000)
    W1, W2 = workloads.weights(0, shape)
    _ORACLE.update(prm=prm, shape=shape, lay=lay, s=s, keys=keys, W1=W1, W2=W2, n_rot=len(steps))
    return _ORACLE


def oracle_layer_step(i):
    """One image's encrypted FFConv layer by the oracle, under the GPU arm's schedule
    (DP_SHIFT_EXT at N = 2^15, 12 + 3 primes): image i of the GPU arm's batch, encrypted
    (untimed), then the layer timed.  Returns (seconds, hoisted rotations of the image)."""
    from oracle import bfv, encoder, ffconv
    from paper_2102_03494_gb300 import workloads
    o = _oracle_layer_setup()
    prm, lay = o["prm"], o["lay"]
    x = workloads.images(0, o["shape"], 64)[i % 64]
    ct = bfv.encrypt(prm, o["s"], encoder.encode(ffconv.input_slots(x, lay, prm.n), prm), 3000 + i % 64)
    t0 = time.perf_counter()
    ffconv.he_layer(prm, ct, o["W1"], o["W2"], lay, o["keys"])
    return time.perf_counter() - t0, o["n_rot"]


ORACLE_UNIT_DESC = ("the oracle's encrypted FFConv layer of one image under the same schedule "
                    "(DP_SHIFT_EXT: ModUp, 24 hoisted rotations key-switched in Q u P, 50 tap "
                    "plaintext products, ModDown per channel, ConvPack restore), N=2^15, L=12, K=3, "
                    "the GPU arm's inputs and seeds")


def cpu_baseline_child():
    """The single-core baseline, run in its own process (started after the timed end-to-end
    region, beside the GPU-bound extra runs on another host core): one image's layer, timed
    once."""
    dt, n = oracle_layer_step(0)
    print(json.dumps({"seconds": dt, "rotations": n}))


def start_cpu_baseline():
    """Starts cpu_baseline_child on one host core; returns the process (or None)."""
    try:
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
        return subprocess.Popen([sys.executable, os.path.abspath(__file__), "--cpu-baseline-child"],
                                stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
    except OSError:
        return None


def finish_cpu_baseline(proc, timeout=900):
    if proc is None:
        return {"error": "could not start the oracle process"}
    try:
        out, err = proc.communicate(timeout=timeout)
        rec = json.loads(out.strip().splitlines()[-1])
    except Exception as e:                 # noqa: BLE001 -- reported in the line
        proc.kill()
        return {"error": f"{type(e).__name__}: {e}"[:300]}
    return {"value": rec["rotations"] / rec["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "ms_per_image": 1000.0 * rec["seconds"],
            "sample": ORACLE_UNIT_DESC + "; one image, run once on one host core (key generation "
                      "and encryption untimed), beside the GPU-bound extra runs on another core"}


def copy_bandwidth(stream, nbytes=1 << 29):
    """Host <-> device copy rate (GB/s) of one large pinned copy each way, on `stream`."""
    import torch
    dev = torch.empty(nbytes // 8, dtype=torch.int64, device="cuda")
    host = torch.empty(nbytes // 8, dtype=torch.int64).pin_memory()
    out = []
    for h2d in (True, False):
        with torch.cuda.stream(stream):
            for _ in range(2):
                (dev.copy_(host, non_blocking=True) if h2d else host.copy_(dev, non_blocking=True))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(3):
                (dev.copy_(host, non_blocking=True) if h2d else host.copy_(dev, non_blocking=True))
            b.record(stream)
        torch.cuda.synchronize()
        out.append(3 * nbytes / (a.elapsed_time(b) / 1e3) / 1e9)
    return out[0], out[1]


def workload_name(args):
    return (f"FFConv layer 1x28x28 -> 5x5 s2 p1 (r=2) -> 1x1 (5 ch), {args.pack}, "
            "N=2^15, 12x50-bit q, 3x60-bit p, alpha=3")


def _reference_init():
    """Pool initializer: the untimed per-worker set-up (keys), before any step."""
    _oracle_layer_setup()


def _reference_step(i):
    return oracle_layer_step(i)


def run_reference(args):
    """The CPU oracle as it stands, on the GPU arm's unit: every step is one image's encrypted
    FFConv layer (DP_SHIFT_EXT, N = 2^15), the steps spread over the host's cores by a spawned
    process pool (no GPU is touched).  Each worker generates its keys before the warm-up; the
    warm-up runs one layer on every worker; the timed region is the wall time of the K steps.
    value = 24 K / wall, ms_per_step = wall / K."""
    import multiprocessing as mp
    rank, _, world = dist_env()
    if rank != 0:
        return
    try:
        avail = len(os.sched_getaffinity(0))
    except AttributeError:
        avail = os.cpu_count() or 1
    workers = max(1, min(16, avail, args.steps))
    with mp.get_context("spawn").Pool(workers, initializer=_reference_init) as pool:
        # at least one warm-up layer per worker (one wave: they run side by side)
        pool.map(_reference_step, range(max(args.warmup, workers)), chunksize=1)
        t0 = time.perf_counter()
        res = pool.map(_reference_step, range(args.steps), chunksize=1)
        wall = time.perf_counter() - t0
    rots = sum(n for _, n in res)
    value = rots / wall
    per_image = statistics.mean(dt for dt, _ in res)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": workload_name(args), "batch_per_gpu": args.batch,
                       "parallelism": f"replicas x{world} (rank 0 times the oracle)",
                       "same_config": True,
                       "sample": "each step: " + ORACLE_UNIT_DESC,
                       "ms_per_image": 1000.0 * per_image,
                       "workers": workers},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                             "sample": f"{args.steps} steps of {ORACLE_UNIT_DESC}, on {workers} host "
                                       f"cores side by side ({wall:.1f} s wall; "
                                       f"{1000.0 * per_image:.0f} ms per image per core)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            for name, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- our arm

def run(args):
    import numpy as np
    import torch

    from paper_2102_03494_gb300 import he, workloads

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    B = args.batch
    shape = workloads.MNIST_LAYER
    stream = torch.cuda.Stream()
    ctx = he.Context(log_n=LOG_N, n_q=N_Q, n_p=N_P, alpha=ALPHA, stream=stream)
    lay = ctx.layout(*shape.astuple(), pack=args.pack)
    steps = ctx.he_ffconv_required_steps(lay)
    n_rot = len(steps)                    # hoisted rotations per image (I_c = 1: no channel fold)
    N = 1 << LOG_N
    ct_bytes = 2 * N_Q * N * 8

    # client side, untimed: keys and encrypted inputs (single-channel image at slot h*I_w + w)
    sk = ctx.he_keygen_secret(1000 + rank)
    ctx.he_keygen_galois(sk, 2000 + rank, steps)
    W1, W2 = workloads.weights(0, shape)
    xs = workloads.images(rank, shape, B)
    cts = []
    for b, x in enumerate(xs):
        slots = np.zeros(N, dtype=np.int64)
        slots[: x.size] = x.reshape(-1)
        cts.append(ctx.he_encrypt(sk, slots, 3000 + b))
    outs = [ctx.new_ct() for _ in range(B * shape.O_c)]
    tuned = ctx.he_autotune(B)            # untimed: picks the NTT split and the tap kernel's
                                          # tile and arithmetic for this batch
    if args.tap_arith != "auto":
        ctx.he_tune_set(he.HE_TUNE_TAP_ARITH, ("chains", "columns", "products").index(args.tap_arith))
        tuned["tap_arith"] = args.tap_arith + " (forced)"
    torch.cuda.synchronize()

    def layer():
        ctx.he_ffconv_layer_batch(cts, W1, W2, lay, outs)

    for _ in range(args.warmup):
        layer()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    l0 = ctx.he_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.he_phase_times()                  # clear, then time every phase of the timed layers
    ctx.he_set_phase_timing(True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        layer()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    phases = ctx.he_phase_times()
    ctx.he_set_phase_timing(False)
    launches = ctx.he_launch_count() - l0
    ms = ev0.elapsed_time(ev1)
    ctx.he_check()                        # raises if a bounded device wait ran out
    sms = torch.cuda.get_device_properties(local).multi_processor_count

    # end to end through the same API with host buffers: every step copies its encrypted
    # inputs host -> device from pinned memory, runs the layer and copies every output
    # ciphertext device -> host.  Two buffer sets pipeline the steps: the H2D copy of step i + 1
    # and the D2H copy of step i - 1 run on copy streams while step i's layer runs.
    # one pinned host block per direction and one device block per buffer set, so that each
    # step's inputs and outputs move as one copy each
    h_in = torch.empty((B, 2, N_Q, N), dtype=torch.int64).pin_memory()
    for h, c in zip(h_in, cts):
        h.copy_(c)
    h_out = torch.empty((B * shape.O_c, 2, N_Q, N), dtype=torch.int64).pin_memory()
    blocks = [(ctx.new_ct(count=B), ctx.new_ct(count=B * shape.O_c)) for _ in range(2)]
    sets = [(list(bi), list(bo)) for bi, bo in blocks]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]      # inputs of set k on the device
    ev_used = [torch.cuda.Event(), torch.cuda.Event()]    # layer on set k finished
    ev_out = [torch.cuda.Event(), torch.cuda.Event()]     # outputs of set k copied out
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)

    def load(k):
        with torch.cuda.stream(up):
            up.wait_event(e0)
            up.wait_event(ev_used[k])                      # the layer two steps back is done
            blocks[k][0].copy_(h_in, non_blocking=True)
            ev_in[k].record(up)

    load(0)
    for i in range(args.steps):
        k = i & 1
        stream.wait_event(ev_in[k])
        stream.wait_event(ev_out[k])                       # outputs two steps back copied out
        ctx.he_ffconv_layer_batch(sets[k][0], W1, W2, lay, sets[k][1])
        ev_used[k].record(stream)
        # the next step's inputs: enqueued after the layer, so that the layer's own small
        # uploads are not queued behind this large copy on the host-to-device copy engine
        if i + 1 < args.steps:
            load(k ^ 1)
        with torch.cuda.stream(down):
            down.wait_event(ev_used[k])
            h_out.copy_(blocks[k][1], non_blocking=True)
            ev_out[k].record(down)
    stream.wait_event(ev_out[0])
    stream.wait_event(ev_out[1])
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1)
    h2d_gbs, d2h_gbs = copy_bandwidth(stream)
    # per-step latency distribution of the same layer (untimed for `value`): 50 steps, an
    # event pair each
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(50)]
    torch.cuda.synchronize()
    for a, b in evs:
        a.record(stream)
        layer()
        b.record(stream)
    torch.cuda.synchronize()
    lat = sorted(a.elapsed_time(b) for a, b in evs)
    lat_p50, lat_p99 = lat[len(lat) // 2], lat[min(len(lat) - 1, int(0.99 * len(lat)))]

    # the plain one-request-at-a-time form: the same layer on one image per call (outputs are
    # bit-identical to the batched call's; tests/test_gpu_layer.py checks it)
    one = [cts[0]]
    one_out = outs[: shape.O_c]
    for _ in range(3):
        ctx.he_ffconv_layer_batch(one, W1, W2, lay, one_out)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_single = max(8, min(64, args.steps))
    torch.cuda.synchronize()
    s0.record(stream)
    for _ in range(n_single):
        ctx.he_ffconv_layer_batch(one, W1, W2, lay, one_out)
    s1.record(stream)
    torch.cuda.synchronize()
    ms_single = s0.elapsed_time(s1) / n_single
    # the same single-image call with the weights resident (a layer plan: W1 plaintexts
    # encoded once, as a server holds them across requests)
    plan = ctx.he_ffconv_plan(W1, W2, lay)
    for _ in range(3):
        ctx.he_ffconv_layer_planned(plan, one, lay, one_out)
    torch.cuda.synchronize()
    s0.record(stream)
    for _ in range(n_single):
        ctx.he_ffconv_layer_planned(plan, one, lay, one_out)
    s1.record(stream)
    torch.cuda.synchronize()
    ms_single_planned = s0.elapsed_time(s1) / n_single
    # ... and captured into a CUDA graph: one submission per image, reading the bound input
    gid, _ = ctx.he_ffconv_graph_create(plan, one, lay, one_out)
    for _ in range(3):
        ctx.he_graph_launch(gid)
    torch.cuda.synchronize()
    s0.record(stream)
    for _ in range(n_single):
        ctx.he_graph_launch(gid)
    s1.record(stream)
    torch.cuda.synchronize()
    ms_single_graph = s0.elapsed_time(s1) / n_single
    ctx.he_graph_free(gid)
    ctx.he_ffconv_plan_free(plan)

    # the single-core oracle baseline runs in a child process from here on, beside the GPU-bound
    # work below; not beside the end-to-end region, whose pinned host copies it would slow
    cpu_proc = start_cpu_baseline() if world == 1 and not args.no_cpu_baseline else None
    roof = taps_roofline(phases, args, B, n_rot, sms, tuned["tap_arith"])
    if roof is not None:          # the measured multiply-accumulate rates, for context
        probe = ctx.he_probe_int_ops()
        clk_hz = measured_peaks()["sm_max_mhz"] * 1e6
        roof["probe"] = {"mul64_T_per_s": {k: probe[k] / 1e12
                                           for k in ("chain", "chain_wide", "columns", "karatsuba")},
                         "per_clock_per_sm": {k: probe[k] / (sms * clk_hz)
                                              for k in ("mad_lo", "mad_hi", "mad_wide")},
                         "read_gbs": ctx.he_probe_mem()}
    layer_bytes = layer_algorithmic_bytes(B, shape.O_c, n_rot)
    peaks = measured_peaks()

    if dist:
        ms, ms_e2e = max_over_ranks([ms, ms_e2e], "cuda")
    value = whole_job_rate(B * n_rot * args.steps, world, ms)
    e2e = whole_job_rate(B * n_rot * args.steps, world, ms_e2e)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": workload_name(args),
                       "batch_per_gpu": B, "layer_ms_per_batch": ms / args.steps,
                       "layer_ms_per_batch_p50_p99": [lat_p50, lat_p99],
                       "layer_ms_per_image": ms / args.steps / B, "hoisted_rotations_per_image": n_rot,
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (keys 755 MB + ModUp digits per step)",
                       "autotune": tuned},
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": B * ct_bytes,
                    "d2h_bytes_per_step": B * shape.O_c * ct_bytes, "ms_per_step": ms_e2e / args.steps,
                    "note": "pinned host buffers, one copy per direction and step; copies of "
                            "neighbouring steps overlap the layer (two buffer sets, two copy streams)",
                    "copy_gbs": {"h2d": h2d_gbs, "d2h": d2h_gbs,
                                 "d2h_ms_per_step": B * shape.O_c * ct_bytes / d2h_gbs / 1e6,
                                 "note": "one 512 MiB pinned copy each way, untimed: the end-to-end "
                                         "step is bound by max(layer, output copy)"}},
            "gpu_launches": launches, "clocks": clk, "roofline": roof,
            "phases_ms_per_step": {k: v[0] / args.steps for k, v in phases.items() if v[1]},
            "batching": {"one_at_a_time_ms_per_image": ms_single,
                         "one_at_a_time_weights_resident_ms_per_image": ms_single_planned,
                         "one_at_a_time_captured_graph_ms_per_image": ms_single_graph,
                         "batched_ms_per_image": ms / args.steps / B,
                         "factor": ms_single / (ms / args.steps / B),
                         "note": "same layer, same outputs; one image per call vs the batch"},
            "layer_hbm": {"algorithmic_bytes_per_step": layer_bytes,
                          "achieved_gbs": layer_bytes / (ms / args.steps / 1000.0) / 1e9,
                          "peak_gbs": peaks["hbm_gbs"],
                          "frac": layer_bytes / (ms / args.steps / 1000.0) / 1e9 / peaks["hbm_gbs"],
                          "note": "keys read once per batch + input and output ciphertexts; "
                                  "the layer is bound by 64-bit modular products, not HBM"}}
    if world == 1 and not args.no_extra:
        line["also"] = extra_workloads(cpu_proc)
    if cpu_proc is not None:
        line["cpu_baseline"] = finish_cpu_baseline(cpu_proc)
    print(json.dumps(check_line(line)))


def extra_workloads(cpu_proc=None):
    """Short runs of the other workloads (their own modes, in child processes on the same GPU),
    summarised beside the layer line; failures are reported, not raised.  The serving run,
    whose latencies depend on the host, starts only after the oracle child (cpu_proc) ended."""
    out = {}
    for key, flags in (("network_n14_b64", ["--net", "--steps", "3", "--warmup", "2"]),
                       ("deep_3x32x32_n15_b16", ["--deep", "--deep-ranks", "8", "--steps", "2",
                                                 "--warmup", "1"]),
                       ("single_request_n13", ["--single", "--steps", "50", "--warmup", "3"]),
                       ("sweep_n15_l16", ["--sweep", "short"]),
                       ("serving_mix", ["--serving", "--serving-rates", "60,120",
                                        "--serving-count", "120"])):
        if key == "serving_mix" and cpu_proc is not None:
            try:
                cpu_proc.wait(timeout=900)
            except subprocess.TimeoutExpired:
                pass
        try:
            res = subprocess.run([sys.executable, os.path.abspath(__file__)] + flags,
                                 capture_output=True, text=True, timeout=900)
            rec = json.loads(res.stdout.strip().splitlines()[-1])
        except Exception as e:             # noqa: BLE001 -- reported in the line
            out[key] = {"error": f"{type(e).__name__}: {e}"[:300]}
            continue
        if key in ("single_request_n13", "sweep_n15_l16"):
            out[key] = rec
            continue
        if key == "serving_mix":
            out[key] = {k: rec.get(k) for k in ("metric", "mix", "workload", "served", "rates")}
            continue
        keep = {k: rec[k] for k in ("metric", "value", "unit", "ms_per_step") if k in rec}
        keep["batch"] = rec.get("config", {}).get("batch_per_gpu")
        if "ops_per_image" in rec:
            keep["ops_per_image"] = rec["ops_per_image"]
        if "variants" in rec:
            keep["ops_per_image"] = rec["variants"][0]["ops_per_image"]
        keep["clocks"] = rec.get("clocks")
        out[key] = keep
    return out


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": d["hbm_gbs"], "sm_max_mhz": d.get("sm_max_mhz", 2070.0), "src": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "src": "fallback"}


# DRAM bytes (read + write) of one carry-chain tap launch at batch 64, from one ncu capture of
# the current kernel (the 64-bit add-with-carry residue products: dram__bytes_read.sum
# 3.545 GB + dram__bytes_write.sum 0.989 GB, one pass); cleared whenever the kernel changes
# until it is captured again.
TAPS_TRAFFIC = {("chains", 64): 3.544969984e9 + 0.989202176e9}


# 64 x 64 -> 128-bit products per second of the GPU's integer multiplier: SMs (152 on GB300)
# x 64 32-bit multiply-adds per clock x clock / 4.  A 64 x 64 -> 128-bit product is four
# 32 x 32 -> 64-bit partial products, and mad.wide.u32 forms one of them (both words) in a
# single multiply-add issue slot: the in-library probe (he_probe_int_ops) measures mad.wide.u32
# at 59 and mad.lo.u32 at 63 per clock and SM, mad.hi.u32 at 27 (half rate).
def mul64_peak_per_s(sm_mhz, sms=152):
    return sms * 64 / 4 * sm_mhz * 1e6


def taps_roofline(phases, args, B, n_rot, sms=152, arith="chains"):
    """Roofline of the dominant phase, the extended-basis tap MAC (the fused tap kernel; with
    the precomputed products also their preparation and the special-prime limbs' chain
    kernel), from its CUDA-event time inside the timed region.  Algorithmic work: per image,
    limb of Q u P and coefficient, 2 dnum products for the key inner product of each rotated
    tap and 2 r products for the plaintext product of every tap."""
    ms, spans = phases["taps"]
    if not spans or args.pack != "dp_shift_ext":
        return None
    N, LK, dnum, r, taps = 1 << LOG_N, N_Q + N_P, -(-N_Q // ALPHA), 2, 25
    products = B * N * LK * (n_rot * 2 * dnum + taps * 2 * r)
    sec = ms / 1000.0 / spans
    pk = measured_peaks()
    peak = mul64_peak_per_s(pk["sm_max_mhz"], sms) / 1e12
    achieved = products / sec / 1e12
    kernels = {"chains": "k_ks_mac_ext_bulk (carry chains)",
               "columns": "k_ks_mac_ext_bulk (30-bit columns)",
               "products": "k_pk_prep + k_tap_pk (q limbs) + k_ks_mac_ext_bulk (p limbs)"}
    return {"kernel": kernels.get(arith.split(" ")[0], arith), "bound": "alu",
            "achieved": achieved, "peak": peak, "unit": "T mul64/s", "frac": achieved / peak,
            "traffic": TAPS_TRAFFIC.get((arith.split(" ")[0], B)), "launch_us": sec * 1e6,
            "products_per_launch": products,
            "peak_note": f"{sms} SMs (device attribute) x 64 multiply-add issue slots per clock / 4 "
                         "mad.wide.u32 per 64x64->128-bit product x max SM clock of MEASURED_PEAKS "
                         f"({pk['src']}); derived, probe-checked (he_probe_int_ops)"}


def layer_algorithmic_bytes(B, O_c, n_rot):
    """Bytes a layer must move at least: its Galois keys once per batch, the input ciphertexts
    and the output ciphertexts (plaintexts are derived from the integer weights)."""
    N, L, LK, dnum = 1 << LOG_N, N_Q, N_Q + N_P, -(-N_Q // ALPHA)
    ct = 2 * L * N * 8
    keys = n_rot * dnum * 2 * LK * N * 8
    return keys + B * ct + B * O_c * ct


def run_serving(args):
    """Serving loop over whole networks: Poisson arrivals of mixed requests -- 60 % the 28 x 28
    three-layer network at N = 2^14 (6 + 2 primes; FFConv layer, combine, x^2, FC 845 -> 100,
    x^2, FC 100 -> 10), 40 % the 3 x 32 x 32 network at N = 2^15 (12 + 3 primes; 3 x 3
    convolutions 3 -> 64 -> 64 -> 128 at rank 8, x^2 after each, pooled classifier to 10) --
    with keys resident, footprint admission and continuous batching over two worker streams per
    ring, against the plain form (one request per call, in arrival order, one stream)."""
    import numpy as np
    import torch

    from paper_2102_03494_gb300 import serving, workloads

    shape = workloads.MNIST_LAYER
    n1 = shape.O_c * ((shape.I_h + 2 * shape.pad - shape.d) // shape.stride + 1) ** 2
    rng = np.random.default_rng(21)
    W1, W2 = workloads.weights(0, shape)
    F1 = rng.integers(-8, 9, (NET_M1, n1))
    F2 = rng.integers(-8, 9, (NET_M2, NET_M1))
    net = serving.NetRing(serving.NetSpec(NET_LOG_N, NET_N_Q, NET_N_P, NET_ALPHA, shape.astuple(),
                                          NET_M1, NET_M2),
                          workers=2, W1=W1, W2=W2, F1=F1, F2=F2, sk_seed=1, key_seed=11,
                          keep_results=False, graphs=8)
    chans, rank = (64, 64, 128), 8
    W1s, W2s, C = [], [], 3
    for O in chans:
        W1s.append(rng.integers(-8, 9, (rank, C, 3, 3)).astype(np.int32))
        W2s.append(rng.integers(-8, 9, (O, rank)).astype(np.int32))
        C = O
    F = rng.integers(-8, 9, (10, C)).astype(np.int32)
    deep = serving.DeepRing(serving.DeepSpec(LOG_N, N_Q, N_P, ALPHA, 3, 32, 32, chans, rank, 10),
                            workers=2, W1s=W1s, W2s=W2s, F=F, sk_seed=2, key_seed=12,
                            keep_results=False, graphs=8)
    rings = {"n14_net3": net, "n15_deep": deep}
    mix = {"n14_net3": 0.6, "n15_deep": 0.4}
    max_batch = 8

    def make_requests(rate, count, seed):
        reqs = serving.poisson_arrivals(seed=seed, rate=rate, count=count, mix=mix)
        for r in reqs:
            g = np.random.default_rng(r.rid + 1000 * seed)
            if r.ring == "n14_net3":
                x = g.integers(0, 256, (shape.I_h, shape.I_w))
                slots = np.zeros(1 << NET_LOG_N, dtype=np.int64)
                slots[: x.size] = x.reshape(-1)
                r.payload = net.encrypt(slots, 7000 + r.rid)
            else:
                x = g.integers(0, 256, (3, 32, 32))
                slots = np.zeros(1 << LOG_N, dtype=np.int64)
                for c in range(3):
                    slots[c * 1024: c * 1024 + 1024] = x[c].reshape(-1)
                r.payload = [deep.encrypt(slots, 7000 + r.rid)]
        torch.cuda.synchronize()
        return reqs

    def release(reqs):
        for r in reqs:
            r.payload = r.result = None

    # warm-up of every worker of every ring at the largest batch, both forms (the graphs were
    # recorded when the rings were built)
    warm = make_requests(1e9, 32, seed=99)
    for name, ring in rings.items():
        mine = [r for r in warm if r.ring == name][:max_batch]
        for use in (False, True):
            ring.use_graphs = use
            for w in range(ring.workers):
                ring.launch(w, mine)
        ring.run_alone(mine[0].payload)
    torch.cuda.synchronize()
    release(warm)

    def serve(rate, count, graphs):
        for ring in rings.values():
            ring.use_graphs = graphs
        reqs = make_requests(rate, count, seed=int(rate))
        sched = serving.Scheduler(rings, max_batch=max_batch, memory_budget=64 << 30,
                                  clock=time.perf_counter)
        done = sched.serve(reqs)
        torch.cuda.synchronize()
        release(reqs)
        return (serving.latency_stats(done),
                {name: serving.latency_stats([r for r in done if r.ring == name]) for name in rings})

    out = {"metric": "serving: mixed-ring encrypted network requests, continuous batching",
           "unit": "requests/s and ms", "mix": mix, "workers_per_ring": 2, "max_batch": max_batch,
           "workload": {"n14_net3": "1x28x28 -> FFConv 5x5 s2 (r=2) -> 5 ch -> combine -> x^2 -> "
                                    "FC 845->100 -> x^2 -> FC 100->10, N=2^14, 6+2 primes",
                        "n15_deep": "3x32x32 -> 3x3 conv 64 -> x^2 -> 64 -> x^2 -> 128 -> x^2 -> "
                                    "pooled FC 128->10, rank 8, N=2^15, 12+3 primes"},
           "served": "batches replayed as recorded CUDA graphs (one per worker and batch size)",
           "served_calls": "the same scheduler, batches run as library calls",
           "rates": []}
    for rate in [float(v) for v in args.serving_rates.split(",")]:
        count = args.serving_count or int(max(60, min(rate * 3, 480)))
        served_calls, _ = serve(rate, count, False)
        served, by_ring = serve(rate, count, True)
        # the plain form: one request per call in arrival order on one stream
        plain_reqs = make_requests(rate, count, seed=int(rate))
        t_free, lat = 0.0, []
        for r in plain_reqs:
            t0 = time.perf_counter()
            rings[r.ring].run_alone(r.payload)
            dt = time.perf_counter() - t0
            start = max(r.t_arrive, t_free)
            t_free = start + dt
            lat.append((t_free - r.t_arrive) * 1000.0)
        span = t_free - plain_reqs[0].t_arrive
        release(plain_reqs)
        plain = {"requests": count, "p50_ms": float(np.percentile(lat, 50)),
                 "p99_ms": float(np.percentile(lat, 99)), "requests_per_s": count / span}
        out["rates"].append({"offered_per_s": rate, "served": served, "served_by_ring": by_ring,
                             "served_calls": served_calls, "plain": plain,
                             "p99_factor": plain["p99_ms"] / served["p99_ms"]})
    print(json.dumps(out))


def run_serving_layers(args):
    """Serving loop over single layers: Poisson arrivals of mixed requests -- 60 % the 28 x 28 layer at N = 2^14
    (6 + 2 primes), 40 % a 3 x 32 x 32 layer (3 x 3 stride 1, r = 8 -> 64 channels) at
    N = 2^15 (12 + 3 primes) -- continuously batched over two worker streams per ring,
    against the plain form (one request per call, in arrival order, one stream)."""
    import numpy as np
    import torch

    from paper_2102_03494_gb300 import serving, workloads

    specs = {"n14_mnist": serving.RingSpec(14, 6, 2, 2, workloads.MNIST_LAYER.astuple()),
             "n15_cifar": serving.RingSpec(15, 12, 3, 3, (3, 32, 32, 3, 1, 1, 8, 64))}
    mix = {"n14_mnist": 0.6, "n15_cifar": 0.4}
    rings = {}
    for i, (name, sp) in enumerate(specs.items()):
        shape = workloads.LayerShape(*sp.shape)
        W1, W2 = workloads.weights(i, shape, lo=-8, hi=8)
        rings[name] = serving.GpuRing(sp, workers=2, W1=W1, W2=W2, sk_seed=1 + i, key_seed=11 + i,
                                      keep_results=False, graphs=8)

    def make_requests(rate, count, seed):
        reqs = serving.poisson_arrivals(seed=seed, rate=rate, count=count, mix=mix)
        for r in reqs:
            sp = specs[r.ring]
            shape = workloads.LayerShape(*sp.shape)
            x = workloads.image(r.rid + 1000 * seed, shape)
            N = 1 << sp.log_n
            hw = shape.I_h * shape.I_w
            B_c = hw if shape.I_c == 1 else 1 << (hw - 1).bit_length()
            slots = np.zeros(N, dtype=np.int64)
            for ci in range(shape.I_c):
                slots[ci * B_c: ci * B_c + hw] = x[ci].reshape(-1)
            r.payload = rings[r.ring].encrypt(slots, 7000 + r.rid)
        torch.cuda.synchronize()
        return reqs

    def release(reqs):
        for r in reqs:
            r.payload = r.result = None

    # warm-up of every worker of every ring at the largest batch (first launches), both forms
    warm = make_requests(1e9, 64, seed=99)
    for name, ring in rings.items():
        mine = [r for r in warm if r.ring == name][:8]
        for use in (False, True):
            ring.use_graphs = use
            for w in range(ring.workers):
                ring.launch(w, mine)
    torch.cuda.synchronize()
    out = {"metric": "serving: mixed-ring encrypted FFConv-layer requests, continuous batching",
           "unit": "requests/s and ms", "mix": mix, "workers_per_ring": 2, "max_batch": 8,
           "served": "batches run as captured CUDA graphs (one per worker and batch size)",
           "served_calls": "the same scheduler, batches run as library calls",
           "rates": []}

    def serve(rate, count, graphs):
        for ring in rings.values():
            ring.use_graphs = graphs
        reqs = make_requests(rate, count, seed=int(rate))
        sched = serving.Scheduler(rings, max_batch=8, memory_budget=64 << 30,
                                  clock=time.perf_counter)
        done = sched.serve(reqs)
        torch.cuda.synchronize()
        release(reqs)
        return serving.latency_stats(done)

    for rate in (100.0, 400.0, 800.0, 1600.0):
        count = int(min(rate * 1.5, 1200))
        served_calls = serve(rate, count, False)
        served = serve(rate, count, True)
        # the plain form: one request per call in arrival order on one stream
        plain_reqs = make_requests(rate, count, seed=int(rate))
        t_free, lat, t_first = 0.0, [], None
        for r in plain_reqs:
            t0 = time.perf_counter()
            rings[r.ring].run_alone(r.payload)
            dt = time.perf_counter() - t0
            start = max(r.t_arrive, t_free)
            t_free = start + dt
            lat.append((t_free - r.t_arrive) * 1000.0)
        span = t_free - plain_reqs[0].t_arrive
        release(plain_reqs)
        plain = {"requests": count, "p50_ms": float(np.percentile(lat, 50)),
                 "p99_ms": float(np.percentile(lat, 99)), "requests_per_s": count / span}
        out["rates"].append({"offered_per_s": rate, "served": served, "served_calls": served_calls,
                             "plain": plain, "p99_factor": plain["p99_ms"] / served["p99_ms"]})
    print(json.dumps(out))


NET_LOG_N, NET_N_Q, NET_N_P, NET_ALPHA, NET_M1, NET_M2 = 14, 6, 2, 2, 100, 10


def run_packing(args):
    """The packing variants of Table IX on its layer: WideNet's second convolution, factorized
    (83 x 13 x 13 input, 6 x 6 stride 2 pad 1 -> r = 20, then 1 x 1 -> 163 channels), one
    encrypted image at N = 2^14 (6 + 2 primes): DP-HI2C-CP (dp_dot, the paper's FFConv form),
    DP-DP (dp_dp, LoLa's form) and CP-HI2C-CP (cp_cp; the Im2Col columns come from the client
    here, so the homomorphic Im2Col that Table IX charges to it is not in the time)."""
    import numpy as np
    import torch

    from paper_2102_03494_gb300 import he

    torch.cuda.set_device(0)
    shape = (83, 13, 13, 6, 2, 1, 20, 163)
    I_c, I_h, I_w, d, st, pad, r, O_c = shape
    O = (I_h + 2 * pad - d) // st + 1
    stream = torch.cuda.Stream()
    ctx = he.Context(log_n=NET_LOG_N, n_q=NET_N_Q, n_p=NET_N_P, alpha=NET_ALPHA, stream=stream)
    N = 1 << NET_LOG_N
    rng = np.random.default_rng(31)
    x = rng.integers(0, 256, (I_c, I_h, I_w))
    W1 = rng.integers(-8, 9, (r, I_c, d, d)).astype(np.int32)
    W2 = rng.integers(-8, 9, (O_c, r)).astype(np.int32)
    sk = ctx.he_keygen_secret(41)
    lay_dp = ctx.layout(*shape, pack="dp_dp")
    ctx.he_keygen_galois(sk, 42, ctx.he_ffconv_required_steps(lay_dp))   # covers dp_dot's too
    dense = np.zeros(N, dtype=np.int64)
    dense[: x.size] = x.reshape(-1)
    ct_dense = ctx.he_encrypt(sk, dense, 43)
    cols = []
    for ci in range(I_c):
        for i in range(d):
            for j in range(d):
                v = np.zeros(N, dtype=np.int64)
                for oh in range(O):
                    for ow in range(O):
                        h, w = st * oh + i - pad, st * ow + j - pad
                        if 0 <= h < I_h and 0 <= w < I_w:
                            v[oh * O + ow] = x[ci, h, w]
                cols.append(ctx.he_encrypt(sk, v, 1000 + len(cols)))
    torch.cuda.synchronize()
    paper_s = {"dp_dot": 75.27, "dp_dp": 784.45, "cp_cp": 2560.49}
    rows = []
    for pack in ("dp_dot", "dp_dp", "cp_cp"):
        lay = ctx.layout(*shape, pack=pack)
        cts = cols if pack == "cp_cp" else [ct_dense]
        outs = [ctx.new_ct() for _ in range(O_c)]
        for _ in range(max(1, args.warmup)):
            ctx.he_ffconv_layer_batch(cts, W1, W2, lay, outs)
        torch.cuda.synchronize()
        ctx.he_reset_op_counts()
        reps = 2
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ctx.he_ffconv_layer_batch(cts, W1, W2, lay, outs)
        e1.record(stream)
        torch.cuda.synchronize()
        ops = {k: v // reps for k, v in ctx.he_op_counts().items()}
        rows.append({"packing": {"dp_dot": "DP-HI2C-CP", "dp_dp": "DP-DP", "cp_cp": "CP-HI2C-CP"}[pack],
                     "pack": pack, "ms_per_image": e0.elapsed_time(e1) / reps, "ops_per_image": ops,
                     "paper_cpu_s": paper_s[pack]})
    print(json.dumps({"metric": "FFConv packing variants on WideNet's factorized second layer (Table IX)",
                      "unit": "ms per image", "config": {
                          "layer": "83x13x13 -> 6x6 s2 p1 (r=20) -> 1x1 (163 ch)",
                          "ring": "N=2^14, 6x50-bit q, 2x60-bit p, alpha=2, t=65537",
                          "note": "cp_cp takes client-side Im2Col columns (2988 ciphertexts); the "
                                  "paper's CP-HI2C-CP time includes 2530 s of homomorphic Im2Col"},
                      "variants": rows}))


def run_net(args):
    """The three-layer network on a batch of encrypted 1 x 28 x 28 images: FFConv layer
    (5 x 5 stride 2, r = 2 -> 5 channels, extended-basis schedule), channel combine, x^2,
    fully connected 845 -> 100, x^2, fully connected 100 -> 10; N = 2^14, 6 x 50-bit q,
    2 x 60-bit p, alpha = 2.  One step = one batch through the whole network."""
    import numpy as np
    import torch

    from paper_2102_03494_gb300 import he, workloads

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B = args.net_batch
    shape = workloads.MNIST_LAYER
    stream = torch.cuda.Stream()
    ctx = he.Context(log_n=NET_LOG_N, n_q=NET_N_Q, n_p=NET_N_P, alpha=NET_ALPHA, stream=stream)
    lay = ctx.layout(*shape.astuple(), pack="dp_shift_ext")
    net = ctx.net(lay, NET_M1, NET_M2)
    steps = ctx.he_net_required_steps(net)
    N = 1 << NET_LOG_N
    ct_bytes = 2 * NET_N_Q * N * 8
    sk = ctx.he_keygen_secret(1000 + rank)
    ctx.he_keygen_galois(sk, 2000 + rank, steps)
    W1, W2 = workloads.weights(0, shape)
    rng = np.random.default_rng(5)
    n1 = shape.O_c * ((shape.I_h + 2 * shape.pad - shape.d) // shape.stride + 1) ** 2
    F1 = rng.integers(-8, 9, (NET_M1, n1))
    F2 = rng.integers(-8, 9, (NET_M2, NET_M1))
    xs = workloads.images(rank, shape, B)
    cts = []
    for b, x in enumerate(xs):
        slots = np.zeros(N, dtype=np.int64)
        slots[: x.size] = x.reshape(-1)
        cts.append(ctx.he_encrypt(sk, slots, 3000 + b))
    outs = [ctx.new_ct() for _ in range(B)]
    tuned = ctx.he_autotune(B)            # untimed
    torch.cuda.synchronize()

    def step():
        ctx.he_net_batch(cts, W1, W2, F1, F2, net, outs)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ctx.he_reset_op_counts()
    l0 = ctx.he_launch_count()
    ctx.he_phase_times()
    ctx.he_set_phase_timing(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    phases = ctx.he_phase_times()
    ctx.he_set_phase_timing(False)
    launches = ctx.he_launch_count() - l0
    ops = ctx.he_op_counts()
    ms = ev0.elapsed_time(ev1)

    h_in = [torch.empty((2, NET_N_Q, N), dtype=torch.int64).pin_memory() for _ in range(B)]
    for h, c in zip(h_in, cts):
        h.copy_(c)
    h_out = [torch.empty((2, NET_N_Q, N), dtype=torch.int64).pin_memory() for _ in range(B)]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            for h, c in zip(h_in, cts):
                c.copy_(h, non_blocking=True)
            step()
            for h, o in zip(h_out, outs):
                h.copy_(o, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1)
    if dist:
        ms, ms_e2e = max_over_ranks([ms, ms_e2e], "cuda")
    value = whole_job_rate(B * args.steps, world, ms)
    if rank != 0:
        return
    per_img = {k: v // (B * args.steps) for k, v in ops.items()}
    line = {"metric": "encrypted 3-layer network throughput (images/s) at N=2^14",
            "value": value, "unit": "images/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "1x28x28 -> FFConv 5x5 s2 p1 (r=2) -> 5 ch -> combine -> x^2 -> "
                                   "FC 845->100 -> x^2 -> FC 100->10, N=2^14, 6x50-bit q, "
                                   "2x60-bit p, alpha=2",
                       "batch_per_gpu": B, "ms_per_image": ms / args.steps / B,
                       "galois_keys": len(steps) - 1, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (Galois keys 0.9 GB per step)"},
            "ops_per_image": per_img,
            "e2e": {"value": whole_job_rate(B * args.steps, world, ms_e2e), "unit": "images/s",
                    "h2d_bytes_per_step": B * ct_bytes, "d2h_bytes_per_step": B * ct_bytes,
                    "ms_per_step": ms_e2e / args.steps},
            "gpu_launches": launches, "clocks": clk,
            "autotune": tuned,
            "phases_ms_per_step": {k: v[0] / args.steps for k, v in phases.items() if v[1]}}
    print(json.dumps(line))


def run_deep(args):
    """The deeper network on a batch of encrypted 3 x 32 x 32 images at N = 2^15 (12 + 3
    primes): three 3 x 3 convolutions 3 -> 64 -> 64 -> 128 channels, each factorized at rank
    r in {8, 16, 32} or unfactorized, x^2 after each, global sum pooling, 10 classes.  One step
    = one batch through the whole network; every variant is timed."""
    import numpy as np
    import torch

    from paper_2102_03494_gb300 import he

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    B = args.deep_batch
    stream = torch.cuda.Stream()
    ctx = he.Context(log_n=LOG_N, n_q=N_Q, n_p=N_P, alpha=ALPHA, stream=stream)
    chans, H, W, n_cls = (64, 64, 128), 32, 32, 10
    N = 1 << LOG_N

    def convs_for(r):
        out, C = [], 3
        for O in chans:
            out.append(ctx.mc_conv(C, H, W, 3, r, O))
            C = O
        return out

    steps = ctx.he_deep_required_steps(convs_for(8), n_cls)
    sk = ctx.he_keygen_secret(1000 + rank)
    ctx.he_keygen_galois(sk, 2000 + rank, steps)
    rng = np.random.default_rng(11)
    xs = rng.integers(0, 256, (B, 3, H, W))
    cts = []
    for b in range(B):
        v = np.zeros(N, dtype=np.int64)
        for c in range(3):
            v[c * 1024: c * 1024 + H * W] = xs[b, c].reshape(-1)
        cts.append(ctx.he_encrypt(sk, v, 3000 + b))
    outs = [ctx.new_ct() for _ in range(B)]
    tuned = ctx.he_autotune(B)            # untimed
    variants = []
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for r in [int(v) for v in args.deep_ranks.split(",")]:
        convs = convs_for(r)
        W1s, W2s, C = [], [], 3
        for O in chans:
            rr = r or O
            W1s.append(rng.integers(-8, 9, (rr, C, 3, 3)).astype(np.int32))
            W2s.append(rng.integers(-8, 9, (O, r)).astype(np.int32) if r else None)
            C = O
        F = rng.integers(-8, 9, (n_cls, C)).astype(np.int32)

        def step():
            ctx.he_deep_batch(cts, convs, W1s, W2s, F, outs)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        ctx.he_reset_op_counts()
        ctx.he_phase_times()
        ctx.he_set_phase_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        phases = ctx.he_phase_times()
        ctx.he_set_phase_timing(False)
        ms = e0.elapsed_time(e1) / args.steps
        ops = {k: v // (B * args.steps) for k, v in ctx.he_op_counts().items()}
        variants.append({"rank": r or "unfactorized", "images_per_s": B / (ms / 1000.0),
                         "ms_per_batch": ms, "ops_per_image": ops,
                         "phases_ms_per_batch": {k: v[0] / args.steps for k, v in phases.items() if v[1]}})
    clk = clocks.stop()
    if rank != 0:
        return
    unf = [v["ms_per_batch"] for v in variants if v["rank"] == "unfactorized"]
    for v in variants:
        if unf and v["rank"] != "unfactorized":
            v["speedup_vs_unfactorized"] = unf[0] / v["ms_per_batch"]
    best = variants[0]
    line = {"metric": "encrypted 3x32x32 network throughput (images/s) at N=2^15",
            "value": best["images_per_s"], "unit": "images/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": best["ms_per_batch"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "3x32x32 -> 3x3 conv 64 -> x^2 -> 3x3 conv 64 -> x^2 -> 3x3 conv "
                                   "128 -> x^2 -> sum pool -> FC 128->10, N=2^15, 12x50-bit q, "
                                   "3x60-bit p, alpha=3; value = rank 8",
                       "batch_per_gpu": B, "galois_keys": len(steps) - 1},
            "autotune": tuned,
            "clocks": clk, "variants": variants}
    print(json.dumps(line))


# ---------------------------------------------------------------- single request, N = 8192

def run_single(args):
    """The plain single-request layer: one encrypted 1 x 28 x 28 image (pixels uniform in
    [0, 255], seed 0), the 5 x 5 stride-2 pad-1 low-rank convolution to r = 2 channels and the
    1 x 1 restore to 5 channels (weights uniform in [-8, 8]), RNS-BFV N = 8192, t = 65537,
    3 x 50-bit q, one 60-bit special prime, digits of one prime; one image per call.  For each
    W1 schedule -- DP_DOT (the paper's DensePack: per output a plaintext product and a
    rotate-and-sum, Sec. 3.2 / Table I), DP_SHIFT and DP_SHIFT_EXT (hoisted filter taps) --
    the call's latency by CUDA events (warm-up, then --steps calls, an event pair each), the
    rotations per call, and the DP_SHIFT_EXT call with the weights resident (a layer plan)
    and replayed as a recorded CUDA graph."""
    import numpy as np
    import torch

    from paper_2102_03494_gb300 import he, workloads

    torch.cuda.set_device(0)
    shape = workloads.MNIST_LAYER
    stream = torch.cuda.Stream()
    ctx = he.Context(log_n=13, n_q=3, n_p=1, alpha=1, stream=stream)
    N = ctx.N
    sk = ctx.he_keygen_secret(1)
    x = workloads.image(0, shape)
    W1, W2 = workloads.weights(0, shape)
    slots = np.zeros(N, dtype=np.int64)
    slots[: x.size] = x.reshape(-1)
    ct = ctx.he_encrypt(sk, slots, 3)
    clocks = ClockSampler(0)
    clocks.start()
    res = {}

    def latency(fn, n):
        for _ in range(max(3, args.warmup)):
            fn()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(n)]
        torch.cuda.synchronize()
        for a, b in evs:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        ms = sorted(a.elapsed_time(b) for a, b in evs)
        return {"ms_mean": statistics.mean(ms), "ms_p50": ms[len(ms) // 2],
                "ms_p99": ms[min(len(ms) - 1, int(0.99 * len(ms)))], "calls": n}

    for pack in ("dp_dot", "dp_shift", "dp_shift_ext"):
        lay = ctx.layout(*shape.astuple(), pack=pack)
        ctx.he_keygen_galois(sk, 2, ctx.he_ffconv_required_steps(lay))
        outs = [ctx.new_ct() for _ in range(shape.O_c)]
        ctx.he_reset_op_counts()
        ctx.he_ffconv_layer_batch([ct], W1, W2, lay, outs)
        ops = ctx.he_op_counts()
        n = max(5, min(args.steps, 20 if pack == "dp_dot" else 200))
        res[pack] = dict(latency(lambda: ctx.he_ffconv_layer_batch([ct], W1, W2, lay, outs), n),
                         ops_per_call=ops)
        if pack == "dp_shift_ext":
            plan = ctx.he_ffconv_plan(W1, W2, lay)
            res[pack]["weights_resident"] = latency(
                lambda: ctx.he_ffconv_layer_planned(plan, [ct], lay, outs), n)
            gid, _ = ctx.he_ffconv_graph_create(plan, [ct], lay, outs)
            res[pack]["graph_replay"] = latency(lambda: ctx.he_graph_launch(gid), n)
            ctx.he_graph_free(gid)
            ctx.he_ffconv_plan_free(plan)
    ctx.he_check()
    clk = clocks.stop()
    print(json.dumps({"metric": "single-request encrypted FFConv layer latency (ms) at N=8192",
                      "unit": "ms", "higher_is_better": False, "dtype": "u64", "data": "synthetic",
                      "config": {"workload": "1x28x28 -> 5x5 s2 p1 (r=2) -> 1x1 (5 ch), N=8192, "
                                             "t=65537, 3x50-bit q + 1x60-bit p, alpha=1, batch 1"},
                      "schedules": res, "clocks": clk}))


# ---------------------------------------------------------------- NTT alone

def run_ntt(args):
    """Forward and inverse negacyclic NTT of 64 x 12 limbs at N = 2^15 (the c1 limbs of a
    batch-64 layer input), the context's default split and radix: one untimed pair first (the
    pair an ncu capture of `-k regex:k_ntt -c 4` sees), then 20 timed pairs by CUDA events;
    then 20 timed pairs on 128 x 12 limbs at the split and radix he_autotune(64) picks."""
    import torch

    from paper_2102_03494_gb300 import he

    torch.cuda.set_device(0)
    ctx = he.Context(log_n=LOG_N, n_q=N_Q, n_p=N_P, alpha=ALPHA)
    N, items, L = 1 << LOG_N, 64, N_Q
    moduli = ctx.he_get_moduli()[:L]
    with torch.cuda.stream(ctx.stream):
        X = torch.empty((items, L, N), dtype=torch.int64, device="cuda")
        for l, q in enumerate(moduli):
            X[:, l].random_(0, q)                       # uniform residues below q_l
    ctx.he_ntt(X, items, L)
    ctx.he_ntt(X, items, L, inverse=True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fwd, inv = [], []
    for _ in range(20):
        ev[0].record(ctx.stream)
        ctx.he_ntt(X, items, L)
        ev[1].record(ctx.stream)
        ctx.he_ntt(X, items, L, inverse=True)
        ev[2].record(ctx.stream)
        ev[2].synchronize()
        fwd.append(ev[0].elapsed_time(ev[1]))
        inv.append(ev[1].elapsed_time(ev[2]))
    bfly = items * L * (N // 2) * LOG_N
    f, i = statistics.median(fwd), statistics.median(inv)
    # then at the split and radix the autotuner picks for a batch of 64, on 128 x 12 limbs
    tuned = ctx.he_autotune(64)
    with torch.cuda.stream(ctx.stream):
        Y = torch.cat([X, X])
    fwd2, inv2 = [], []
    for rep in range(22):
        ev[0].record(ctx.stream)
        ctx.he_ntt(Y, 2 * items, L)
        ev[1].record(ctx.stream)
        ctx.he_ntt(Y, 2 * items, L, inverse=True)
        ev[2].record(ctx.stream)
        ev[2].synchronize()
        if rep >= 2:
            fwd2.append(ev[0].elapsed_time(ev[1]))
            inv2.append(ev[1].elapsed_time(ev[2]))
    ctx.he_check()
    f2, i2 = statistics.median(fwd2), statistics.median(inv2)
    print(json.dumps({"metric": "negacyclic NTT / inverse NTT at N=2^15, 50-bit primes",
                      "unit": "ms", "data": "synthetic (uniform residues)", "dtype": "u64",
                      "default_split_64x12": {"log2_n1": LOG_N // 2, "forward_ms": f,
                                              "inverse_ms": i,
                                              "forward_T_butterflies_per_s": bfly / f / 1e9,
                                              "inverse_T_butterflies_per_s": bfly / i / 1e9},
                      "autotuned_128x12": {"log2_n1": tuned["ntt_log2_n1"],
                                           "radix": tuned["ntt_radix"], "forward_ms": f2,
                                           "inverse_ms": i2,
                                           "forward_T_butterflies_per_s": 2 * bfly / f2 / 1e9,
                                           "inverse_T_butterflies_per_s": 2 * bfly / i2 / 1e9}}))


# ---------------------------------------------------------------- primitive sweep

# The primitive sweep's grid: ring sizes, ciphertext primes L -> (special primes K, digit
# width alpha = K), batch sizes and hoisted step counts.
SWEEP_LOG_N = (13, 14, 15, 16)
SWEEP_L = {3: 1, 8: 2, 16: 4, 24: 6}
SWEEP_B = (1, 16, 256, 1024)
SWEEP_H = (8, 24)
SWEEP_MAX_KEYS = 64
SWEEP_MEM_LIMIT = 150 << 30
L2_BYTES = 129 << 20


SWEEP_HOIST_OUT_BYTES = 16 << 30


def sweep_hoist_batch(log_n, L, h):
    """Ciphertexts per batched hoisted call in the sweep: as many whose h outputs fit 16 GiB,
    between 8 and 64 (the output sets are reused from call to call)."""
    ct = 2 * L * (1 << log_n) * 8
    return max(8, min(64, SWEEP_HOIST_OUT_BYTES // (h * ct)))


def sweep_point_bytes(log_n, L, K, B, h):
    """Device bytes a sweep point holds: the B input and B output ciphertexts, the hoisted
    outputs of one batched call (reused), the Galois keys and the rotation scratch."""
    N = 1 << log_n
    ct = 2 * L * N * 8
    dnum = -(-L // K)
    key = 16 * dnum * (L + K) * N
    n_keys = min(max(B, h), SWEEP_MAX_KEYS)
    scratch = min(B, 64) * (L + dnum * (L + K) + 2 * (L + K) + 2 * L) * N * 8
    hoist = min(B, sweep_hoist_batch(log_n, L, h)) * h * ct
    return 2 * B * ct + hoist + n_keys * key + scratch


def run_sweep(args):
    """Batched primitive sweep: negacyclic NTT and inverse NTT, the Galois automorphism, plain
    key-switched rotations (ciphertexts grouped by Galois key, one batched call per key) and
    hoisted rotations (h steps per ciphertext sharing one ModUp; ciphertexts grouped by step
    set, batched calls of up to 8 .. 64 of them), over batch sizes, ring sizes
    and prime counts.  Ciphertexts hold residues uniform modulo each prime; steps are uniform
    in [1, N/2); min(B, 64) distinct Galois keys (max(h, min(B, 64)) for the hoisted points),
    generated on the device, each ciphertext taking one of them uniformly.  Every op is timed
    by CUDA events on the library's stream: two warm-up calls, then enough repetitions for
    about 0.3 s (3 .. 20); points whose inputs are smaller than L2 flush it (a 256 MiB write,
    outside the timed events) before every repetition.  The ciphertext lists of every call are
    marshalled to the C ABI once per point, outside the timed calls.  Points above 150 GB are
    skipped."""
    import numpy as np
    import torch

    from paper_2102_03494_gb300 import he

    torch.cuda.set_device(0)
    short = args.sweep == "short"
    grid_n = (15,) if short else SWEEP_LOG_N
    grid_l = (16,) if short else tuple(SWEEP_L)
    grid_b = (16, 256) if short else SWEEP_B
    stream = torch.cuda.Stream()
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peaks = measured_peaks()
    clocks = ClockSampler(0)
    clocks.start()
    points = []

    def timed(fn, flush):
        for _ in range(2):
            fn()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        first = e0.elapsed_time(e1)
        reps = int(max(3, min(20, 300.0 / max(first, 1e-3))))
        total = 0.0
        for _ in range(reps):
            if flush:
                with torch.cuda.stream(stream):
                    flush_buf.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        return total / reps, reps

    for log_n in grid_n:
        N = 1 << log_n
        for L in grid_l:
            K = SWEEP_L[L]
            todo = [B for B in grid_b
                    if sweep_point_bytes(log_n, L, K, B, max(SWEEP_H)) <= SWEEP_MEM_LIMIT]
            for B in grid_b:
                if B not in todo:
                    points.append({"log_n": log_n, "L": L, "K": K, "B": B, "skipped":
                                   f"needs {sweep_point_bytes(log_n, L, K, B, max(SWEEP_H)) / 1e9:.0f} GB "
                                   "on the device, above the 150 GB bound"})
            if not todo:
                continue
            ctx = he.Context(log_n=log_n, n_q=L, n_p=K, alpha=K, stream=stream)
            rng = np.random.default_rng(1000 * log_n + L)
            n_keys = min(max(max(todo), max(SWEEP_H)), SWEEP_MAX_KEYS)
            steps = [int(x) for x in rng.choice(np.arange(1, N // 2), n_keys, replace=False)]
            sk = ctx.he_keygen_secret(7)
            ctx.he_keygen_galois(sk, 8, steps)
            ctx.he_autotune(min(max(todo), 64))
            moduli = ctx.he_get_moduli()[:L]
            dnum = -(-L // K)
            for B in todo:
                torch.cuda.synchronize()
                with torch.cuda.stream(stream):
                    X = torch.empty((B, 2, L, N), dtype=torch.int64, device="cuda")
                    for l, q in enumerate(moduli):
                        X[:, :, l, :].random_(0, q)       # uniform residues below q_l
                    Y = torch.empty_like(X)
                ins, outs = list(X), list(Y)
                ins_b, outs_b = ctx.ct_batch(ins), ctx.ct_batch(outs)   # marshalled once, untimed
                ct_bytes = 2 * L * N * 8
                flush = B * ct_bytes < 2 * L2_BYTES
                pt = {"log_n": log_n, "L": L, "K": K, "alpha": K, "B": B,
                      "l2": "flushed before every repetition" if flush else "inputs larger than L2"}
                # NTT / inverse NTT of all 2 B polynomials' limbs
                ms, reps = timed(lambda: ctx.he_ntt(X, 2 * B, L), flush)
                pt["ntt_limbs_per_s"] = 2 * B * L / (ms / 1e3)
                pt["ntt_butterflies_T_per_s"] = 2 * B * L * (N // 2) * log_n / (ms / 1e3) / 1e12
                ms, reps = timed(lambda: ctx.he_ntt(X, 2 * B, L, inverse=True), flush)
                pt["intt_limbs_per_s"] = 2 * B * L / (ms / 1e3)
                # automorphism: read and write every word once
                ms, reps = timed(lambda: ctx.he_automorphism(ins_b, steps[0], outs_b), flush)
                gbs = 2 * B * ct_bytes / (ms / 1e3) / 1e9
                pt["automorphism_gbs"] = gbs
                pt["automorphism_hbm_frac"] = gbs / peaks["hbm_gbs"]
                # plain rotations, grouped by key
                nk = min(B, SWEEP_MAX_KEYS)
                owner = rng.integers(0, nk, B)
                groups = [(steps[k], [i for i in range(B) if owner[i] == k]) for k in range(nk)]
                groups = [(st, ctx.ct_batch([ins[i] for i in idx]), ctx.ct_batch([outs[i] for i in idx]))
                          for st, idx in groups if idx]

                def plain():
                    for st, gi, go in groups:
                        ctx.he_rotate_batch(gi, st, go)

                ms, reps = timed(plain, flush)
                pt["rotations_per_s"] = B / (ms / 1e3)
                key_bytes = 16 * dnum * (L + K) * N
                pt["rotation_gbs_algorithmic"] = (2 * B * ct_bytes + len(groups) * key_bytes) / (ms / 1e3) / 1e9
                # hoisted: ciphertexts grouped by step set (one set of h steps per h of the
                # keys), one ModUp per ciphertext, batched calls of up to P ciphertexts of one
                # group, the P h output ciphertexts reused from call to call
                for h in SWEEP_H:
                    hk = min(max(B, h), SWEEP_MAX_KEYS)
                    sets = [[steps[int(k)] for k in rng.choice(hk, h, replace=False)]
                            for _ in range(max(1, hk // h))]
                    owner = rng.integers(0, len(sets), B)
                    P = min(B, sweep_hoist_batch(log_n, L, h))
                    calls = []
                    for g, st in enumerate(sets):
                        idx = [i for i in range(B) if owner[i] == g]
                        calls += [(st, [ins[i] for i in idx[j:j + P]])
                                  for j in range(0, len(idx), P)]
                    with torch.cuda.stream(stream):
                        pool = list(ctx.new_ct(count=P * h))
                    calls = [(st, ctx.ct_batch(cts), ctx.ct_batch(pool[:len(cts) * h]))
                             for st, cts in calls]

                    def hoisted():
                        for st, cts, po in calls:
                            ctx.he_rotate_hoisted_batch(cts, st, po)

                    ms, reps = timed(hoisted, flush)
                    pt[f"hoisted_h{h}_rotations_per_s"] = B * h / (ms / 1e3)
                    pt[f"hoisted_h{h}_calls"] = len(calls)
                    del pool
                ctx.he_check()
                points.append(pt)
                del X, Y, ins, outs
            ctx.close()
            torch.cuda.empty_cache()
    clk = clocks.stop()
    line = {"metric": "batched primitive sweep: NTT/INTT limbs/s, automorphism GB/s, plain and "
                      "hoisted key-switched rotations/s",
            "unit": "per point", "n_gpus": 1, "data": "synthetic (uniform residues)",
            "dtype": "u64", "grid": "short" if short else "full",
            "config": {"primes": "50-bit q, 60-bit p, alpha = K", "hbm_peak_gbs": peaks["hbm_gbs"],
                       "sms": sms},
            "points": points, "clocks": clk}
    print(json.dumps(line))


def main():
    args = parse()
    if args.cpu_baseline_child:
        cpu_baseline_child()
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.ntt:
        run_ntt(args)
        return
    if args.single:
        run_single(args)
        return
    if args.packing:
        run_packing(args)
        return
    if args.serving_layers:
        run_serving_layers(args)
        return
    if args.serving:
        run_serving(args)
        return
    if args.net:
        run_net(args)
        return
    if args.deep:
        run_deep(args)
        return
    run(args)


if __name__ == "__main__":
    main()
