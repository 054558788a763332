"""The serving scheduler's host logic with a fake executor and a fake clock (no GPU): every
request completes, admission never exceeds the memory budget (a request larger than the
whole budget is refused), batches hold one ring and at most max_batch requests, no ring runs
more batches than it has workers, each ring is served oldest first, requests that arrive
while a batch runs are batched into the next one, and arrivals are seeded."""
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


def test_a_request_larger_than_the_budget_is_refused():
    import pytest
    clock, log = Clock(), []
    rings = {"large": FakeRing("large", 1, 0.05, 400, clock, log)}
    sched = Scheduler(rings, max_batch=4, memory_budget=300, clock=clock)
    with pytest.raises(ValueError):
        sched.submit(Request(rid=0, ring="large", t_arrive=0.0))


def test_no_ring_runs_more_batches_than_it_has_workers():
    done, log, peak, sched = run()
    durations = {"small": 0.02, "large": 0.05}
    workers = {"small": 2, "large": 1}
    for ring in ("small", "large"):
        spans = [(t, t + durations[ring]) for (r, w, rids, t) in log if r == ring]
        for t0, _ in spans:
            running = sum(1 for a, b in spans if a <= t0 < b)
            assert running <= workers[ring], (ring, t0, running)
        # each worker index is used by at most one batch at a time
        for w in range(workers[ring]):
            mine = sorted(t for (r, ww, rids, t) in log if r == ring and ww == w)
            assert all(b - a >= durations[ring] - 1e-9 for a, b in zip(mine, mine[1:]))


def test_poisson_arrivals_are_seeded_and_follow_the_mix():
    a = poisson_arrivals(seed=7, rate=100.0, count=2000, mix={"x": 0.6, "y": 0.4})
    b = poisson_arrivals(seed=7, rate=100.0, count=2000, mix={"x": 0.6, "y": 0.4})
    assert [(r.ring, r.t_arrive) for r in a] == [(r.ring, r.t_arrive) for r in b]
    share = sum(r.ring == "x" for r in a) / len(a)
    assert 0.55 < share < 0.65
    mean_gap = a[-1].t_arrive / len(a)
    assert 0.009 < mean_gap < 0.011                  # rate 100 per second
