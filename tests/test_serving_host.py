"""Host-side scheduling of the serving loop (no GPU): FIFO admission onto a
fixed set of workers, concurrency bounded by the workers, latency bookkeeping."""
import threading
import time

from paper_2606_20441_b300 import inputs, serving


class FakeExecutor:
    def __init__(self, service_s=0.02):
        self.service_s = service_s
        self.active = 0
        self.max_active = 0
        self.lock = threading.Lock()
        self.order = []

    def run(self, worker, inst):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
            self.order.append(inst.name)
        time.sleep(self.service_s)
        with self.lock:
            self.active -= 1
        return 0, float(len(inst.name)), 10.0, 1


def test_fifo_bounded_concurrency_and_latency():
    reqs = inputs.workload_serving(count=12, rate_hz=400.0, side_hi=5, steps_hi=6)
    ex = FakeExecutor()
    out = serving.Server(ex, n_workers=3).serve(reqs)
    assert [o.rid for o in out] == list(range(12))
    assert ex.max_active <= 3
    assert ex.order == [r.instance.name for r in sorted(reqs, key=lambda r: r.arrival_s)]
    for o in out:
        assert o.start_s >= o.arrival_s - 1e-3
        assert o.latency_s >= ex.service_s * 0.9
    s = serving.summarize(out)
    assert s["served"] == 12 and s["failed"] == 0 and s["p99_ms"] >= s["p50_ms"]


def test_failures_are_reported_not_retried():
    class Failing(FakeExecutor):
        def run(self, worker, inst):
            super().run(worker, inst)
            return 4, None, 0.0, 0
    reqs = inputs.workload_serving(count=4, rate_hz=1000.0, side_hi=4, steps_hi=5)
    out = serving.Server(Failing(0.001), n_workers=2).serve(reqs)
    s = serving.summarize(out)
    assert s["failed"] == 4 and s["served"] == 0


def test_requests_that_outgrow_a_large_share_run_alone():
    """With exclusive=True a request that outgrows a large share waits until
    every worker is idle (no new work starts meanwhile) and runs alone with the
    whole budget; its class then goes straight to the exclusive queue."""
    class Budget(FakeExecutor):
        def __init__(self, service_s):
            super().__init__(service_s)
            self.attempts = {}
            self.overlap = 0

        def _note(self, inst, kind):
            self.attempts.setdefault(inst.name, []).append(kind)

        def run(self, worker, inst):
            self._note(inst, "large" if worker >= 2 else "small")
            super().run(worker, inst)
            if inst.n_qubits > 20:
                return serving.PP_ERR_CAPACITY, None, 0.0, 0
            return 0, 1.0, 5.0, 1

        def run_exclusive(self, worker, inst):
            self._note(inst, "alone")
            with self.lock:
                self.overlap = max(self.overlap, self.active)
            super().run(worker, inst)
            return 0, 2.0, 50.0, 1

    def key(inst):
        return inst.n_qubits > 20

    reqs = inputs.workload_serving(count=12, rate_hz=800.0, side_hi=6, steps_hi=5)
    huge = [r for r in reqs if r.instance.n_qubits > 20]
    assert len(huge) >= 2
    ex = Budget(0.003)
    srv = serving.Server(ex, n_workers=2, n_large=1, route_key=key, exclusive=True)
    out = srv.serve(reqs)
    assert ex.overlap == 0
    s = serving.summarize(out)
    assert s["served"] == 12 and s["failed"] == 0
    by_rid = {o.rid: o for o in out}
    for r in huge:
        assert by_rid[r.rid].escalated and ex.attempts[r.instance.name][-1] == "alone"
    assert ex.attempts[huge[0].instance.name][0] != "alone"
    assert srv.exclusive_classes == {True}
    # the class is known now: later requests of it skip the smaller shares
    # (a backlog: everything present at once, the ordinary requests released
    # first), and the exclusive runs wait for the queued work, so every
    # ordinary request starts before the first exclusive run
    ex.attempts.clear()
    backlog = sorted(reqs, key=lambda r: r.instance.n_qubits > 20)
    again = [inputs.Request(100 + k, 0.0, r.instance) for k, r in enumerate(backlog)]
    size = {100 + k: r.instance.n_qubits for k, r in enumerate(backlog)}
    out2 = srv.serve(again)
    assert all(o.status == 0 for o in out2)
    for r in huge:
        assert ex.attempts[r.instance.name] == ["alone"]
    assert ex.overlap == 0
    first_alone = min(o.start_s for o in out2 if size[o.rid] > 20)
    assert all(o.start_s <= first_alone for o in out2 if size[o.rid] <= 20)
    # without exclusive the same requests fail on the large worker
    out3 = serving.Server(Budget(0.001), n_workers=2, n_large=1).serve(reqs)
    assert sum(o.status != 0 for o in out3) == len(huge)


def test_exclusive_failures_are_reported():
    class Never(FakeExecutor):
        def run(self, worker, inst):
            super().run(worker, inst)
            return serving.PP_ERR_CAPACITY, None, 0.0, 0

        def run_exclusive(self, worker, inst):
            super().run(worker, inst)
            return serving.PP_ERR_CAPACITY, None, 0.0, 0
    reqs = inputs.workload_serving(count=3, rate_hz=1000.0, side_hi=4, steps_hi=4)
    out = serving.Server(Never(0.001), n_workers=1, n_large=1, exclusive=True).serve(reqs)
    assert [o.status for o in out] == [serving.PP_ERR_CAPACITY] * 3
    try:
        serving.Server(FakeExecutor(), n_workers=1, exclusive=True)
    except ValueError:
        pass
    else:
        raise AssertionError("exclusive needs run_exclusive")


def test_capacity_failures_escalate_to_large_workers():
    """A request that outgrows a small worker's share is re-admitted to the
    large workers with its original arrival time and served there."""
    class Shares(FakeExecutor):
        def run(self, worker, inst):
            super().run(worker, inst)
            big = inst.n_qubits > 20
            if big and worker < 2:
                return serving.PP_ERR_CAPACITY, None, 0.0, 0
            return 0, 1.0, 5.0, 1
    reqs = inputs.workload_serving(count=10, rate_hz=500.0, side_hi=6, steps_hi=5)
    ex = Shares(0.002)
    out = serving.Server(ex, n_workers=2, n_large=1).serve(reqs)
    assert [o.rid for o in out] == list(range(10))
    by_rid = {r.rid: r for r in reqs}
    for o in out:
        big = by_rid[o.rid].instance.n_qubits > 20
        assert o.status == 0
        assert o.arrival_s <= o.start_s + 1e-3
        if big:
            assert o.worker == 2
        if o.escalated:
            assert big
    assert any(by_rid[o.rid].instance.n_qubits > 20 for o in out)
    s = serving.summarize(out)
    assert s["served"] == 10 and s["failed"] == 0


def test_large_worker_failures_are_final():
    class AlwaysFull(FakeExecutor):
        def run(self, worker, inst):
            super().run(worker, inst)
            return serving.PP_ERR_CAPACITY, None, 0.0, 0
    reqs = inputs.workload_serving(count=5, rate_hz=1000.0, side_hi=4, steps_hi=5)
    ex = AlwaysFull(0.001)
    out = serving.Server(ex, n_workers=2, n_large=1).serve(reqs)
    assert len(out) == 5 and all(o.status == serving.PP_ERR_CAPACITY for o in out)
    assert all(o.worker == 2 for o in out)
    # each request ran at most once on a small worker, then once on the large one
    assert len(ex.order) <= 10


def test_learned_routing_skips_small_workers():
    """Once a class has needed a large share, its later requests go straight to
    the large workers (each big request runs on a small worker at most once per
    class, not once per request)."""
    class Shares(FakeExecutor):
        def run(self, worker, inst):
            super().run(worker, inst)
            if inst.n_qubits > 20 and worker < 2:
                return serving.PP_ERR_CAPACITY, None, 0.0, 0
            return 0, 1.0, 5.0, 1
    reqs = inputs.workload_serving(count=24, rate_hz=100.0, side_hi=6, steps_hi=5)
    big = [r for r in reqs if r.instance.n_qubits > 20]
    assert len(big) >= 4
    ex = Shares(0.003)
    srv = serving.Server(ex, n_workers=2, n_large=1, route_key=lambda inst: inst.n_qubits > 20)
    out = srv.serve(reqs)
    assert all(o.status == 0 for o in out) and len(out) == 24
    # every run of a big request beyond the first few was on the large worker:
    # small-worker attempts are bounded by the requests in flight when the class
    # was first learned (at most the two small workers' worth)
    runs = len(ex.order)
    assert runs - len(reqs) <= 2
    assert srv.large_classes == {True}


class CancellableExecutor(FakeExecutor):
    """Runs until the request's service time passes or the server cancels it
    (the stand-in for pp_cancel stopping a propagation after a sub-layer)."""

    def __init__(self, service_s):
        super().__init__(service_s)
        self.stop = {}
        self.started = {}

    def run(self, worker, inst):
        ev = threading.Event()
        with self.lock:
            self.stop[worker] = ev
            self.started[inst.name] = time.perf_counter()
        cancelled = ev.wait(self.service_s)
        return (serving.PP_ERR_TIMEOUT, None, 0.0, 0) if cancelled else (0, 1.0, 10.0, 1)

    def cancel(self, worker):
        with self.lock:
            ev = self.stop.get(worker)
        if ev is not None:
            ev.set()


def test_cancel_running_and_queued_requests():
    """One worker: request 0 runs long and is cancelled mid-flight, request 1
    is cancelled while still queued; both end with PP_ERR_TIMEOUT, the worker
    goes on to serve the rest."""
    reqs = inputs.workload_serving(count=4, rate_hz=1e6, side_hi=4, steps_hi=5)
    ex = CancellableExecutor(service_s=2.0)
    srv = serving.Server(ex, n_workers=1)
    result = {}

    def run():
        result["out"] = srv.serve(reqs)

    th = threading.Thread(target=run)
    th.start()
    t0 = time.perf_counter()
    while reqs[0].instance.name not in ex.started and time.perf_counter() - t0 < 5:
        time.sleep(0.01)
    assert srv.cancel(reqs[1].rid)      # queued behind request 0
    assert srv.cancel(reqs[0].rid)      # running
    ex.service_s = 0.01                 # the rest finish quickly
    th.join(timeout=10)
    assert not th.is_alive()
    out = {o.rid: o for o in result["out"]}
    assert out[reqs[0].rid].status == serving.PP_ERR_TIMEOUT
    assert out[reqs[1].rid].status == serving.PP_ERR_TIMEOUT and out[reqs[1].rid].worker == -1
    assert out[reqs[2].rid].status == 0 and out[reqs[3].rid].status == 0
    assert time.perf_counter() - t0 < 2.0   # request 0 did not run its full service time
    assert not srv.cancel(reqs[2].rid)      # already finished


def test_largest_first_backlog_order():
    """With every request waiting at once and one worker, the largest-first
    backlog runs them by decreasing estimated cost (qubits x layers); FIFO runs
    them in arrival order."""
    reqs = inputs.workload_serving(count=8, rate_hz=1e6, side_hi=6, steps_hi=8, eps_set=(1e-3,), w_max=6)
    for backlog in ("fifo", "largest_first"):
        ex = FakeExecutor()
        out = serving.Server(ex, n_workers=1, backlog=backlog).serve(reqs, time_scale=0.0)
        assert all(o.status == 0 for o in out)
        by_name = {r.instance.name: r for r in reqs}
        ran = [by_name[n] for n in ex.order]
        if backlog == "fifo":
            assert ran == sorted(reqs, key=lambda r: r.arrival_s)
        else:
            # the first request may start before the others are released
            costs = [serving.estimated_cost(r.instance) for r in ran[1:]]
            assert costs == sorted(costs, reverse=True)
