"""Serving: continuous batching of propagation requests on one GPU.

Requests (an Instance each: lattice, depth, angles, noise, observable,
threshold) arrive over time.  Worker threads take them in arrival order as soon
as a worker is free, so requests that arrive while others run are admitted
immediately and their kernels overlap on the GPU: each worker drives its own
handles on its own CUDA stream, and the library's calls release the GIL.

Admission by HBM budget: the budget is divided among the workers up front;
each worker owns one handle per mask width (W = 1 for up to 64 qubits, W = 2
up to 128), whose term capacity is its share of the budget.  A request whose
strings outgrow that capacity ends with PP_ERR_CAPACITY and is reported, not
retried on a smaller share.  Keeping the term arrays of a request on the
device between its layers is the library's ordinary behaviour.

The executor is injectable so the scheduling logic can be exercised without a
GPU.
"""
from __future__ import annotations

import dataclasses
import queue
import threading
import time
from typing import Callable, List, Optional

import numpy as np

from . import inputs


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

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


class GpuExecutor:
    """Runs a request on the worker's own handles (one per mask width)."""

    def __init__(self, n_workers: int, hbm_budget_bytes: float, precision: int = 32):
        import torch
        from . import pp
        self.pp = pp
        self.precision = precision
        bytes_per = {1: 16 + (4 if precision == 32 else 8), 2: 32 + (4 if precision == 32 else 8)}
        # per handle: two term arenas, two overflow areas of a quarter arena,
        # and per-bucket counters: ~2.6 strings' worth per term of capacity
        share = hbm_budget_bytes / n_workers / 2.0
        self.handles = []
        self.streams = []
        for w in range(n_workers):
            st = torch.cuda.Stream()
            self.streams.append(st)
            hs = {}
            for W in (1, 2):
                cap = int(share / (2.6 * bytes_per[W]))
                hs[W] = pp.Handle(64 * W, precision=precision, max_terms=cap, stream=st.cuda_stream)
            self.handles.append(hs)

    def run(self, worker: int, inst: "inputs.Instance"):
        h = self.handles[worker][inputs.n_words(inst.n_qubits)]
        try:
            h.load_instance(inst)
            h.run_instance(inst)
            e = h.pp_expect()
            s = h.pp_get_stats()
            return self.pp.PP_OK, e, s.updates, s.n_terms
        except self.pp.PPError as ex:
            return ex.status, None, 0.0, 0

    def close(self):
        for hs in self.handles:
            for h in hs.values():
                h.close()


class Server:
    """FIFO continuous batching over `n_workers` workers."""

    def __init__(self, executor, n_workers: int, clock: Callable[[], float] = time.perf_counter):
        self.executor = executor
        self.n_workers = n_workers
        self.clock = clock
        self.q: "queue.Queue" = queue.Queue()
        self.outcomes: List[Outcome] = []
        self._lock = threading.Lock()

    def _worker(self, w: int):
        while True:
            item = self.q.get()
            if item is None:
                return
            req, arrival = item
            start = self.clock()
            status, e, upd, terms = self.executor.run(w, req.instance)
            done = self.clock()
            with self._lock:
                self.outcomes.append(Outcome(req.rid, arrival, start, done, w, status, e, upd, terms))

    def serve(self, requests: List["inputs.Request"], time_scale: float = 1.0) -> List[Outcome]:
        """Releases each request at its arrival time (scaled), waits for all."""
        workers = [threading.Thread(target=self._worker, args=(w,), daemon=True) for w in range(self.n_workers)]
        for t in workers:
            t.start()
        t0 = self.clock()
        for req in sorted(requests, key=lambda r: r.arrival_s):
            due = t0 + req.arrival_s * time_scale
            wait = due - self.clock()
            if wait > 0:
                time.sleep(wait)
            self.q.put((req, max(due, t0)))
        for _ in workers:
            self.q.put(None)
        for t in workers:
            t.join()
        return sorted(self.outcomes, key=lambda o: o.rid)


def summarize(outcomes: List[Outcome], ok_status: int = 0) -> dict:
    ok = [o for o in outcomes if o.status == ok_status]
    lat = np.array([o.latency_s for o in ok]) if ok else np.zeros(1)
    span = (max(o.done_s for o in outcomes) - min(o.arrival_s for o in outcomes)) if outcomes else 0.0
    upd = sum(o.updates for o in ok)
    return {"requests": len(outcomes), "served": len(ok), "failed": len(outcomes) - len(ok),
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "updates_per_s": upd / span if span > 0 else 0.0, "span_s": span}
