"""Serving: continuous batching of propagation requests on one GPU.

Requests (an Instance each: lattice, depth, angles, noise, observable,
threshold) arrive over time.  Worker threads take them in arrival order as soon
as a worker is free, so requests that arrive while others run are admitted
immediately and their kernels overlap on the GPU: each worker drives its own
handles on its own CUDA stream, and the library's calls release the GIL.

Admission by HBM budget.  The number of live strings a request will reach is
not known before it runs, so the budget is divided up front into worker
shares: `n_small` workers with equal small shares and `n_large` workers that
split a large fraction of the budget.  A worker's handle (for the mask width of
its request) has its share as term capacity.  A request starts on whichever worker is free; if it outgrows a small
share (PP_ERR_CAPACITY) it is re-admitted, with its original arrival time, to
the queue that only the large workers serve first.  A request that outgrows a
large share is reported as failed, unless the server runs exclusive requests:
then it waits until no other request is queued, the GPU drains (no worker
takes new work meanwhile), and it runs alone with the whole budget.  Under a
backlog the exclusive runs thus come after the queued work, with one drain
instead of one per request.  With a `route_key` (a workload-class
function), a class that has needed a large share once sends its later requests
straight to the large workers, and one that has needed the whole budget
straight to the exclusive queue, so they do not first waste a smaller share's
time.  Keeping the term arrays of a request on the device between its layers
is the library's ordinary behaviour.

The executor is injectable so the scheduling logic can be exercised without a
GPU.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import Callable, List, Optional

import numpy as np

from . import inputs

PP_ERR_CAPACITY = 4
PP_ERR_TIMEOUT = 6    # cancelled (pp_cancel) or dropped from the queue by Server.cancel


@dataclasses.dataclass
class Outcome:
    rid: int
    arrival_s: float
    start_s: float
    done_s: float
    worker: int
    status: int
    expect: Optional[float]
    updates: float
    terms: int
    escalated: bool = False

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


class GpuExecutor:
    """Workers 0..n_small-1 hold small shares of the HBM budget, workers
    n_small..n_small+n_large-1 hold large ones.  Each worker has its own CUDA
    stream and one handle at a time, for the mask width of its current request
    (W = 1 up to 64 qubits, W = 2 up to 128), with the whole share as its term
    capacity.  Handles take their device memory from torch's caching
    allocator, so replacing a worker's handle when the mask width changes
    returns the memory to the cache instead of freeing it (a device free would
    stall every stream on the GPU)."""

    def __init__(self, n_small: int, hbm_budget_bytes: float, precision: int = 32,
                 n_large: int = 0, large_fraction: float = 0.5, tuner=None):
        import torch
        from . import pp
        self.pp = pp
        self.precision = precision
        self.n_small = n_small
        self.n_large = n_large
        self.tuner = tuner
        frac_small = 1.0 - (large_fraction if n_large > 0 else 0.0)
        self.shares = [hbm_budget_bytes * frac_small / n_small] * n_small
        self.shares += [hbm_budget_bytes * large_fraction / n_large] * n_large
        self.streams = [torch.cuda.Stream() for _ in self.shares]
        self.current: List[Optional[tuple]] = [None] * len(self.shares)   # (W, Handle)
        self.exclusive: Optional[tuple] = None     # (W, Handle) of the last exclusive run
        self._excl_worker: Optional[int] = None    # worker driving an exclusive run
        self._lock = threading.Lock()

    def capacity(self, worker: int, W: int) -> int:
        # two term arenas, two overflow areas of a quarter arena and per-bucket
        # counters: ~2.6 strings' worth of memory per term of capacity
        per_string = 16 * W + (4 if self.precision == 32 else 8)
        return int(self.shares[worker] / (2.6 * per_string))

    def _release_exclusive(self):
        """Closes the exclusive handle kept from the last exclusive run (its
        memory goes back to the device for the workers' shares)."""
        import torch
        with self._lock:
            if self.exclusive is not None:
                self.exclusive[1].close()
                self.exclusive = None
                torch.cuda.empty_cache()

    def handle(self, worker: int, W: int):
        if self.exclusive is not None:
            self._release_exclusive()
        cur = self.current[worker]
        if cur is not None and cur[0] == W:
            return cur[1]
        if cur is not None:
            cur[1].close()
        h = self.pp.Handle(64 * W, precision=self.precision, max_terms=self.capacity(worker, W),
                           torch_memory=True, stream=self.streams[worker].cuda_stream)
        self.current[worker] = (W, h)
        return h

    def _run_on(self, h, inst: "inputs.Instance", tune: bool = True):
        try:
            h.load_instance(inst)
            setting = self.tuner.apply(h, inst) if (tune and self.tuner is not None) else None
            h.run_instance(inst)
            e = h.pp_expect()
            s = h.pp_get_stats()
            if setting is not None:
                self.tuner.observe(inst, setting, s.updates, s.seconds)
            return self.pp.PP_OK, e, s.updates, s.n_terms
        except self.pp.PPError as ex:
            return ex.status, None, 0.0, 0

    def run(self, worker: int, inst: "inputs.Instance"):
        try:
            h = self.handle(worker, inputs.n_words(inst.n_qubits))
        except self.pp.PPError as ex:
            return ex.status, None, 0.0, 0
        return self._run_on(h, inst)

    def run_exclusive(self, worker: int, inst: "inputs.Instance"):
        """Runs `inst` alone with the whole budget as its capacity, on
        `worker`'s stream, with the library's default plan (no tuning trials
        on the largest requests).  The caller guarantees that no other worker
        is running.  The first exclusive run closes every worker's handle
        (their memory goes back to the device) and opens an exclusive handle;
        it stays open, at its grown capacity, for the exclusive runs that
        follow, and is closed when a worker next needs its own handle.  An
        allocation that torch refuses reaches the library as NULL
        (PP_ERR_NOMEM), never as a bad pointer."""
        import torch
        W = inputs.n_words(inst.n_qubits)
        if self.exclusive is None or self.exclusive[0] != W:
            self._release_exclusive()
            self._close_workers()
            # hand the released blocks back to the device: the library sizes its
            # growth from the device's free memory, which torch's cache hides
            torch.cuda.empty_cache()
            per_string = 16 * W + (4 if self.precision == 32 else 8)
            try:
                h = self.pp.Handle(64 * W, precision=self.precision,
                                   max_terms=int(sum(self.shares) / (2.6 * per_string)),
                                   torch_memory=True, stream=self.streams[worker].cuda_stream)
            except self.pp.PPError as ex:
                return ex.status, None, 0.0, 0
            self.exclusive = (W, h)
        h = self.exclusive[1]
        self._excl_worker = worker
        try:
            return self._run_on(h, inst, tune=False)
        finally:
            self._excl_worker = None

    def cancel(self, worker: int):
        """Stops the propagation running on `worker` (pp_cancel); its run()
        returns PP_ERR_TIMEOUT after the sub-layer in flight."""
        cur = self.current[worker]
        if self._excl_worker == worker and self.exclusive is not None:
            cur = self.exclusive
        if cur is not None:
            cur[1].pp_cancel()

    def _close_workers(self):
        for k, cur in enumerate(self.current):
            if cur is not None:
                cur[1].close()
            self.current[k] = None

    def close(self):
        """Closes every handle, the workers' and the exclusive one."""
        self._close_workers()
        self._release_exclusive()


def estimated_cost(inst: "inputs.Instance") -> float:
    """A size proxy for ordering a batch: qubits times layers (the live-string
    count grows with both)."""
    return float(inst.n_qubits) * float(inst.n_layers)


def batch_order(requests: List["inputs.Request"]) -> List["inputs.Request"]:
    """Largest-first order for requests that are all present at once, so the
    longest propagations start first and the short ones fill in around them."""
    return sorted(requests, key=lambda r: (r.arrival_s, -estimated_cost(r.instance), r.rid))


class Server:
    """Continuous batching: `n_workers` small-share workers and `n_large`
    large-share workers (indices after the small ones).  Large workers take
    re-admitted requests first, then ordinary ones.  `backlog` orders the
    ordinary requests that are waiting when a worker frees up: "fifo" (arrival
    order) or "largest_first" (the largest estimated cost first, ties by
    arrival: under a backlog the longest propagations start first and the short
    ones fill in around them, which shortens the span of a saturated stream;
    with an empty backlog both take the next arrival).  `exclusive` (needs an
    executor with run_exclusive) re-admits a request that outgrew a large
    share to an exclusive queue: once no other request is queued, no worker
    takes new work until every worker is idle, and it runs alone with the
    whole budget."""

    def __init__(self, executor, n_workers: int, n_large: int = 0,
                 clock: Callable[[], float] = time.perf_counter,
                 route_key: Optional[Callable] = None, backlog: str = "fifo",
                 exclusive: bool = False):
        if backlog not in ("fifo", "largest_first"):
            raise ValueError("backlog must be 'fifo' or 'largest_first'")
        if exclusive and not hasattr(executor, "run_exclusive"):
            raise ValueError("exclusive requests need an executor with run_exclusive")
        self.backlog = backlog
        self.executor = executor
        self.n_workers = n_workers
        self.n_large = n_large
        self.clock = clock
        self.route_key = route_key
        self.exclusive = exclusive
        self.large_classes: set = set()
        self.exclusive_classes: set = set()
        self.outcomes: List[Outcome] = []

    def _worker(self, w: int, large: bool):
        while True:
            alone = False
            with self._cv:
                while True:
                    if self._excl_running:
                        self._cv.wait()
                        continue
                    if self._exclusive and not self._fresh and not self._escalated:
                        # once no other request waits, drain: no new work
                        # until every worker is idle, then run it alone
                        if not self._running:
                            item = self._exclusive.popleft()
                            alone = True
                            self._excl_running = True
                            break
                        self._cv.wait()
                        continue
                    if large and self._escalated:
                        item = self._escalated.popleft()
                        break
                    if self._fresh:
                        if self.backlog == "largest_first" and len(self._fresh) > 1:
                            best = max(self._fresh, key=lambda it: (estimated_cost(it[0].instance), -it[1]))
                            self._fresh.remove(best)
                            item = best
                        else:
                            item = self._fresh.popleft()
                        break
                    if self._closed and self._pending == 0:
                        return
                    self._cv.wait()
            req, arrival, escalated = item
            start = self.clock()
            with self._cv:
                self._running[w] = req.rid
            if alone:
                status, e, upd, terms = self.executor.run_exclusive(w, req.instance)
            else:
                status, e, upd, terms = self.executor.run(w, req.instance)
            done = self.clock()
            with self._cv:
                self._running.pop(w, None)
                if alone:
                    self._excl_running = False
                if req.rid in self._cancelled:
                    status, e = PP_ERR_TIMEOUT, None
                retry = status == PP_ERR_CAPACITY and req.rid not in self._cancelled and not alone
                if retry and not large and self.n_large > 0:
                    self._escalated.append((req, arrival, True))
                    if self.route_key is not None:
                        self.large_classes.add(self.route_key(req.instance))
                elif retry and self.exclusive:
                    self._exclusive.append((req, arrival, True))
                    if self.route_key is not None:
                        self.exclusive_classes.add(self.route_key(req.instance))
                else:
                    self.outcomes.append(Outcome(req.rid, arrival, start, done, w, status, e, upd, terms,
                                                 escalated))
                    self._pending -= 1
                self._cv.notify_all()

    def cancel(self, rid: int) -> bool:
        """Cancels request `rid`: a queued request is dropped at once, one in
        flight is stopped by the executor after its current sub-layer.  Either
        way its outcome has status PP_ERR_TIMEOUT.  Returns False if the
        request already finished (or was never released)."""
        with self._cv:
            if any(o.rid == rid for o in self.outcomes):
                return False
            self._cancelled.add(rid)
            for q in (self._fresh, self._escalated, self._exclusive):
                for item in list(q):
                    if item[0].rid == rid:
                        q.remove(item)
                        now = self.clock()
                        self.outcomes.append(Outcome(rid, item[1], now, now, -1, PP_ERR_TIMEOUT, None, 0.0, 0,
                                                     item[2]))
                        self._pending -= 1
                        self._cv.notify_all()
                        return True
            for w, r in self._running.items():
                if r == rid:
                    self.executor.cancel(w)
                    return True
            return rid in self._released

    def serve(self, requests: List["inputs.Request"], time_scale: float = 1.0) -> List[Outcome]:
        """Releases each request at its arrival time (scaled), waits for all."""
        self._cv = threading.Condition()
        self._fresh: "collections.deque" = collections.deque()
        self._escalated: "collections.deque" = collections.deque()
        self._exclusive: "collections.deque" = collections.deque()
        self._excl_running = False
        self._running: dict = {}
        self._cancelled: set = set()
        self._released: set = set()
        self._closed = False
        self._pending = len(requests)
        self.outcomes = []
        workers = [threading.Thread(target=self._worker, args=(w, w >= self.n_workers), daemon=True)
                   for w in range(self.n_workers + self.n_large)]
        for t in workers:
            t.start()
        t0 = self.clock()
        for req in sorted(requests, key=lambda r: r.arrival_s):   # stable: ties keep the given order
            due = t0 + req.arrival_s * time_scale
            wait = due - self.clock()
            if wait > 0:
                time.sleep(wait)
            with self._cv:
                self._released.add(req.rid)
                if req.rid in self._cancelled:
                    now = self.clock()
                    self.outcomes.append(Outcome(req.rid, max(due, t0), now, now, -1, PP_ERR_TIMEOUT, None, 0.0,
                                                 0, False))
                    self._pending -= 1
                    self._cv.notify_all()
                    continue
                key = self.route_key(req.instance) if self.route_key is not None else None
                if self.exclusive and key is not None and key in self.exclusive_classes:
                    self._exclusive.append((req, max(due, t0), True))
                elif self.n_large > 0 and key is not None and key in self.large_classes:
                    self._escalated.append((req, max(due, t0), True))
                else:
                    self._fresh.append((req, max(due, t0), False))
                self._cv.notify_all()
        with self._cv:
            self._closed = True
            self._cv.notify_all()
        for t in workers:
            t.join()
        return sorted(self.outcomes, key=lambda o: o.rid)


def summarize(outcomes: List[Outcome], ok_status: int = 0) -> dict:
    ok = [o for o in outcomes if o.status == ok_status]
    lat = np.array([o.latency_s for o in ok]) if ok else np.zeros(1)
    span = (max(o.done_s for o in outcomes) - min(o.arrival_s for o in outcomes)) if outcomes else 0.0
    upd = sum(o.updates for o in ok)
    return {"requests": len(outcomes), "served": len(ok), "failed": len(outcomes) - len(ok),
            "escalated": sum(1 for o in outcomes if o.escalated),
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "updates_per_s": upd / span if span > 0 else 0.0, "span_s": span}
