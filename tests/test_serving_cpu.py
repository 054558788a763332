"""The serving scheduler's host logic with a fake executor and a fake clock (no GPU): every
request completes, admission never exceeds the memory budget, batches hold one ring and at
most max_batch requests, each ring is served oldest first, and requests that arrive while a
batch runs are batched into the next one."""
from paper_2102_03494_gb300.serving import Request, Scheduler, latency_stats, poisson_arrivals


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-4          # every poll advances time a little
        return self.t


class FakeRing:
    def __init__(self, name, workers, duration, footprint, clock, log):
        self.name, self.workers, self.duration, self.fp = name, workers, duration, footprint
        self.clock, self.log = clock, log

    def footprint(self, req):
        return self.fp

    def launch(self, worker, requests):
        self.log.append((self.name, worker, [r.rid for r in requests], self.clock.t))
        return self.clock.t + self.duration

    def done(self, handle):
        return self.clock.t >= handle

    def results(self, handle, requests):
        for r in requests:
            r.result = (self.name, r.rid)


def run(budget=10_000, max_batch=4):
    clock, log = Clock(), []
    rings = {"small": FakeRing("small", 2, 0.02, 100, clock, log),
             "large": FakeRing("large", 1, 0.05, 400, clock, log)}
    sched = Scheduler(rings, max_batch=max_batch, memory_budget=budget, clock=clock)
    peak = [0]
    orig = sched.step

    def step():
        busy = orig()
        peak[0] = max(peak[0], sched.in_use)
        return busy
    sched.step = step
    reqs = poisson_arrivals(seed=1, rate=300.0, count=200, mix={"small": 0.6, "large": 0.4})
    done = sched.serve(reqs)
    return done, log, peak[0], sched


def test_all_requests_complete_in_ring_order_and_batches_are_bounded():
    done, log, peak, sched = run()
    assert len(done) == 200 and all(r.result == (r.ring, r.rid) for r in done)
    assert sched.in_use == 0 and peak <= 10_000
    for ring, worker, rids, _ in log:
        assert 1 <= len(rids) <= 4
        assert all(next(r for r in done if r.rid == i).ring == ring for i in rids)
    for ring in ("small", "large"):
        starts = [(r.t_arrive, r.t_start) for r in done if r.ring == ring]
        starts.sort()
        assert all(a[1] <= b[1] for a, b in zip(starts, starts[1:]))   # oldest first


def test_budget_limits_admission():
    done, log, peak, sched = run(budget=800)        # two large or eight small at a time
    assert len(done) == 200 and peak <= 800


def test_continuous_batching_picks_up_late_arrivals():
    done, log, peak, sched = run()
    by_id = {r.rid: r for r in done}
    joined_late = 0
    for i, (ring, w, rids, t_launch) in enumerate(log):
        earlier = [x for x in log[:i] if x[0] == ring]
        if earlier:
            prev_launch = earlier[-1][3]
            joined_late += sum(1 for j in rids if by_id[j].t_arrive > prev_launch)
    assert joined_late > 0
    stats = latency_stats(done)
    assert stats["requests"] == 200 and stats["p99_ms"] >= stats["p50_ms"] > 0
