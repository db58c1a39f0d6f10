"""Serving: continuous batching of propagation requests on one GPU.

Requests (an Instance each: lattice, depth, angles, noise, observable,
threshold) arrive over time.  Worker threads take them in arrival order as soon
as a worker is free, so requests that arrive while others run are admitted
immediately and their kernels overlap on the GPU: each worker drives its own
handles on its own CUDA stream, and the library's calls release the GIL.

Admission by HBM budget.  The number of live strings a request will reach is
not known before it runs, so the budget is divided up front into worker
shares: `n_small` workers with equal small shares and `n_large` workers that
split a large fraction of the budget.  Every worker owns one handle per mask
width (W = 1 up to 64 qubits, W = 2 up to 128) whose term capacity is its
share.  A request starts on whichever worker is free; if it outgrows a small
share (PP_ERR_CAPACITY) it is re-admitted, with its original arrival time, to
the queue that only the large workers serve first.  A request that outgrows a
large share is reported as failed.  Keeping the term arrays of a request on
the device between its layers is the library's ordinary behaviour.

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
    n_small..n_small+n_large-1 hold large ones; each worker has its own CUDA
    stream and one handle per mask width."""

    def __init__(self, n_small: int, hbm_budget_bytes: float, precision: int = 32,
                 n_large: int = 0, large_fraction: float = 0.5, tuner=None):
        import torch
        from . import pp
        self.pp = pp
        self.precision = precision
        self.n_small = n_small
        self.n_large = n_large
        self.tuner = tuner
        bytes_per = {1: 16 + (4 if precision == 32 else 8), 2: 32 + (4 if precision == 32 else 8)}
        frac_small = 1.0 - (large_fraction if n_large > 0 else 0.0)
        shares = [hbm_budget_bytes * frac_small / n_small] * n_small
        shares += [hbm_budget_bytes * large_fraction / n_large] * n_large
        self.handles = []
        self.streams = []
        for share in shares:
            st = torch.cuda.Stream()
            self.streams.append(st)
            hs = {}
            # per handle: two term arenas, two overflow areas of a quarter arena
            # and per-bucket counters, ~2.6 strings' worth per term of capacity;
            # the share is split between the W = 1 and W = 2 handles
            for W in (1, 2):
                cap = int(share / 2.0 / (2.6 * bytes_per[W]))
                hs[W] = pp.Handle(64 * W, precision=precision, max_terms=cap, stream=st.cuda_stream)
            self.handles.append(hs)

    def run(self, worker: int, inst: "inputs.Instance"):
        h = self.handles[worker][inputs.n_words(inst.n_qubits)]
        try:
            h.load_instance(inst)
            setting = self.tuner.apply(h, inst) if self.tuner is not None else None
            h.run_instance(inst)
            e = h.pp_expect()
            s = h.pp_get_stats()
            if setting is not None:
                self.tuner.observe(inst, setting, s.updates, s.seconds)
            return self.pp.PP_OK, e, s.updates, s.n_terms
        except self.pp.PPError as ex:
            return ex.status, None, 0.0, 0

    def close(self):
        for hs in self.handles:
            for h in hs.values():
                h.close()


class Server:
    """FIFO continuous batching: `n_workers` small-share workers and `n_large`
    large-share workers (indices after the small ones).  Large workers take
    re-admitted requests first, then ordinary ones."""

    def __init__(self, executor, n_workers: int, n_large: int = 0,
                 clock: Callable[[], float] = time.perf_counter):
        self.executor = executor
        self.n_workers = n_workers
        self.n_large = n_large
        self.clock = clock
        self.outcomes: List[Outcome] = []

    def _worker(self, w: int, large: bool):
        while True:
            with self._cv:
                while True:
                    if large and self._escalated:
                        item = self._escalated.popleft()
                        break
                    if self._fresh:
                        item = self._fresh.popleft()
                        break
                    if self._closed and self._pending == 0:
                        return
                    self._cv.wait()
            req, arrival, escalated = item
            start = self.clock()
            status, e, upd, terms = self.executor.run(w, req.instance)
            done = self.clock()
            with self._cv:
                if status == PP_ERR_CAPACITY and not large and self.n_large > 0:
                    self._escalated.append((req, arrival, True))
                else:
                    self.outcomes.append(Outcome(req.rid, arrival, start, done, w, status, e, upd, terms,
                                                 escalated))
                    self._pending -= 1
                self._cv.notify_all()

    def serve(self, requests: List["inputs.Request"], time_scale: float = 1.0) -> List[Outcome]:
        """Releases each request at its arrival time (scaled), waits for all."""
        self._cv = threading.Condition()
        self._fresh: "collections.deque" = collections.deque()
        self._escalated: "collections.deque" = collections.deque()
        self._closed = False
        self._pending = len(requests)
        self.outcomes = []
        workers = [threading.Thread(target=self._worker, args=(w, w >= self.n_workers), daemon=True)
                   for w in range(self.n_workers + self.n_large)]
        for t in workers:
            t.start()
        t0 = self.clock()
        for req in sorted(requests, key=lambda r: r.arrival_s):
            due = t0 + req.arrival_s * time_scale
            wait = due - self.clock()
            if wait > 0:
                time.sleep(wait)
            with self._cv:
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
