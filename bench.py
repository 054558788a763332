"""Benchmark: the encrypted FFConv layer at N = 2^15 on one GB300 (or N replicas).

One step = one encrypted FFConv layer (DP_SHIFT schedule: 24 hoisted rotations of each input,
tap MACs, ConvPack restore) over a batch of B encrypted 1 x 28 x 28 images, RNS-BFV with
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
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--pack", default="dp_shift_ext", choices=["dp_shift", "dp_shift_ext", "dp_dot"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


# ---------------------------------------------------------------- CPU oracle sample

def oracle_sample(n_steps=2, seed=0):
    """Time the oracle's hoisted rotations of one ciphertext at the bench's ring (one ModUp,
    n_steps key switches).  Returns (seconds, rotations, description)."""
    import numpy as np
    from oracle import bfv, encoder, params
    prm = params.Params(log_n=LOG_N, n_q=N_Q, n_p=N_P, alpha=ALPHA)
    s = bfv.keygen_secret(prm, seed + 1)
    steps = [1, 28][:n_steps]
    keys = {bfv.galois_of(st, prm.n): bfv.galois_key(prm, s, bfv.galois_of(st, prm.n), seed + 2)
            for st in steps}
    v = np.random.default_rng(seed).integers(0, prm.t, prm.n)
    ct = bfv.encrypt(prm, s, encoder.encode(v, prm), seed + 3)
    t0 = time.perf_counter()
    bfv.rotate_hoisted(prm, ct, steps, keys)
    dt = time.perf_counter() - t0
    return dt, len(steps), f"oracle hoisted rotation of 1 ciphertext by {len(steps)} steps at N=2^15, L=12, K=3"


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    times, rots = [], 0
    for i in range(args.warmup + args.steps):
        dt, n, desc = oracle_sample(n_steps=1, seed=i)
        if i >= args.warmup:
            times.append(dt)
            rots += n
    total = sum(times)
    value = rots / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": "hoisted rotations of the FFConv layer input, N=2^15, L=12, K=3, alpha=3",
                       "ring": "N=32768, 12x50-bit q, 3x60-bit p", "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": desc.replace("by 2 steps", "by 1 step") + f", {args.steps} samples"},
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
                 "--format=csv,noheader,nounits", "-lms", "200"],
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
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        layer()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = ctx.he_launch_count() - l0
    ms = ev0.elapsed_time(ev1)

    # end to end through the same API with host buffers: H2D of the step's encrypted inputs
    # from pinned memory, the layer, D2H of every output ciphertext
    h_in = [torch.empty((2, N_Q, N), dtype=torch.int64).pin_memory() for _ in range(B)]
    for h, c in zip(h_in, cts):
        h.copy_(c)
    h_out = [torch.empty((2, N_Q, N), dtype=torch.int64).pin_memory() for _ in range(B * shape.O_c)]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            for h, c in zip(h_in, cts):
                c.copy_(h, non_blocking=True)
            layer()
            for h, o in zip(h_out, outs):
                h.copy_(o, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1)

    # roofline of the dominant kernel, timed alone on the same stream
    roof = kernel_roofline(ctx, stream, B)

    if dist:
        t = torch.tensor([ms, ms_e2e], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, ms_e2e = (float(v) for v in t.tolist())
    value = world * B * n_rot * args.steps / (ms / 1000.0)
    e2e = world * B * n_rot * args.steps / (ms_e2e / 1000.0)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"FFConv layer 1x28x28 -> 5x5 s2 p1 (r=2) -> 1x1 (5 ch), {args.pack}, "
                                   "N=2^15, 12x50-bit q, 3x60-bit p, alpha=3",
                       "batch_per_gpu": B, "layer_ms_per_batch": ms / args.steps,
                       "layer_ms_per_image": ms / args.steps / B, "hoisted_rotations_per_image": n_rot,
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (keys 377 MB + ModUp digits per step)"},
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": B * ct_bytes,
                    "d2h_bytes_per_step": B * shape.O_c * ct_bytes, "ms_per_step": ms_e2e / args.steps},
            "gpu_launches": launches, "clocks": clk, "roofline": roof}
    if world == 1 and not args.no_cpu_baseline:
        dt, n, desc = oracle_sample(n_steps=2)
        line["cpu_baseline"] = {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": desc}
    print(json.dumps(line))


def kernel_roofline(ctx, stream, B):
    """Average duration of the NTT launch pair the layer issues most (the ModDown transforms of
    B ciphertexts: 2 x 12 limbs forward), from CUDA events around repeated launches."""
    import torch
    N, L = 1 << LOG_N, N_Q
    items = 2 * B
    buf = torch.randint(0, 1 << 40, (items, L, N), dtype=torch.int64, device="cuda")
    reps = 20
    torch.cuda.synchronize()
    for _ in range(3):
        ctx.he_ntt(buf, items, L)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        ctx.he_ntt(buf, items, L)
    b.record(stream)
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1000.0 / reps
    limbs = items * L
    byts = limbs * N * 8 * 2           # each limb read and written once
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    gbs = byts / sec / 1e9
    return {"kernel": "ntt forward (column + row pass)", "bound": "hbm", "achieved": gbs,
            "peak": peak, "unit": "GB/s", "frac": gbs / peak, "traffic": None,
            "launch_us": sec * 1e6, "limbs_per_launch": limbs}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    run(args)


if __name__ == "__main__":
    main()
