"""Request loop: continuous batching of decomposition requests on one GPU.

Requests (a graph, a job (r,s), a mode) arrive at any time.  Worker threads,
each with its own CUDA stream, take waiting requests as soon as device memory
and a worker are free.  A worker drains every waiting request of the same job
(up to a byte cap) into one disjoint-union batch (nd_build_incidence_batch),
so small requests that arrive together share one launch per pass.  Requests
running on different workers overlap on the device.  Admission is by HBM
footprint: each request's incidence size is bounded from its degrees before
it is admitted, and the sum over running requests stays under the budget.

All computation runs in libnd; this module only schedules.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import nd


RELABEL_MIN_VERTICES = 1 << 16   # graphs from this size are renumbered by degree class in the build


def footprint_bytes(row_ptr: np.ndarray, col: np.ndarray, r: int) -> int:
    """Upper bound on the device bytes a request needs (graph copy, edge
    arrays, incidence, work items, two tau buffers and frontiers), at the
    build's peak: for (2,3) the incidence is written once and ranked into a
    second buffer, next to the CSR-slot arrays; for large (1,2) and (2,3)
    graphs the relabelled CSR sits next to the caller's copy, and a large
    (2,3) graph also sorts 8-byte keys (two buffers) and keeps edge-id maps.

    The incidence size is bounded by sum over edges of min(d_u, d_v) (common
    neighbours of an edge) for (2,3), and by that bound times the largest
    degree for (3,4)."""
    n = row_ptr.size - 1
    nnz = int(row_ptr[-1])
    deg = np.diff(row_ptr)
    base = 12 * (n + 1) + 8 * nnz + 16 * n
    copies = 1  # incidence buffers alive at the build's peak
    if r == 1:
        num_r, inc = n, nnz
        q = 1
        base += 8 * (n + 1) + 4 * nnz + 8 * n + 4 * n  # relabelled CSR, id maps, 16-bit copies
    else:
        u = np.repeat(np.arange(n), deg)
        up = u < col
        tri_bound = int(np.minimum(deg[u[up]], deg[col[up]]).astype(np.int64).sum())
        if r == 2:
            num_r, inc, q = nnz // 2, tri_bound, 2
            copies = 2
            base += 8 * (nnz // 2) + 4 * nnz + 4 * nnz + nnz // 4  # e_pos, 16-bit copies, reverse slots, frontier
            if n >= RELABEL_MIN_VERTICES:
                # relabelled CSR, sort keys and their ping-pong buffer, edge-id maps, vertex map
                base += 8 * (n + 1) + 4 * nnz + 16 * nnz + nnz // 2 + 8 * (nnz // 2) + 4 * n
        else:
            num_r = tri_bound // 3 + 1
            inc = tri_bound * int(deg.max() if n else 0) // 3
            q = 3
        base += 12 * (nnz // 2)
    return int(base + 8 * (num_r + 1) + copies * 4 * q * inc + 16 * num_r + 8 * num_r + num_r // 4 + (1 << 20))


@dataclass(eq=False)
class Request:
    row_ptr: np.ndarray
    col: np.ndarray
    r: int
    s: int
    mode: str = "and"           # "snd", "and" or "and_nn"
    rid: int = 0
    arrival: float = 0.0
    start: float = 0.0
    finish: float = 0.0
    result: np.ndarray | None = None
    iters: int = 0
    error: str | None = None
    footprint: int = 0
    batched_with: int = 1
    done: threading.Event = field(default_factory=threading.Event)


class Server:
    """Continuous-batching server.  submit() may be called from any thread
    while requests run; close() waits for everything submitted."""

    def __init__(self, budget_bytes: int, workers: int = 4, batch_bytes: int = 1 << 30,
                 max_batch: int = 64, device: int = 0, max_wait_s: float = 1.0):
        import torch
        self.torch = torch
        self.device = device
        self.max_wait_s = float(max_wait_s)
        self.budget = int(budget_bytes)
        self.batch_bytes = int(batch_bytes)
        self.max_batch = int(max_batch)
        self.used = 0
        self.queue: list[Request] = []
        self.cv = threading.Condition()
        self.closing = False
        self.next_id = 0
        self.completed: list[Request] = []
        nd.load()
        self.threads = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(workers)]
        for t in self.threads:
            t.start()

    # ------------------------------------------------------------- client
    def submit(self, row_ptr, col, r: int, s: int, mode: str = "and") -> Request:
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        req = Request(row_ptr, col, r, s, mode)
        req.footprint = footprint_bytes(row_ptr, col, r)
        with self.cv:
            if req.footprint > self.budget:
                req.error = "request exceeds the device budget"
                req.done.set()
                return req
            req.rid = self.next_id
            self.next_id += 1
            req.arrival = time.perf_counter()
            self.queue.append(req)
            self.cv.notify_all()
        return req

    def cancel(self, req: Request) -> bool:
        """Withdraw a request that is still waiting.  Returns True if it was
        removed (its error is then "cancelled" and it counts as done); False
        if a worker has already taken it (it runs to completion) or it has
        finished."""
        with self.cv:
            if req not in self.queue:
                return False
            self.queue.remove(req)
            req.error = "cancelled"
            req.finish = time.perf_counter()
            self.cv.notify_all()
        req.done.set()
        return True

    def close(self):
        with self.cv:
            self.closing = True
            self.cv.notify_all()
        for t in self.threads:
            t.join()

    # ------------------------------------------------------------- workers
    def _take(self, now: float | None = None) -> list[Request]:
        """Oldest admissible request, plus every waiting request of the same
        job and mode that fits the batch cap and the budget (FIFO within a
        job, so no request waits behind a later one of its own job).

        Aging: once the oldest waiting request has waited longer than
        max_wait_s without fitting, nothing else is admitted until it fits,
        so a stream of small requests cannot starve a large one."""
        if self.queue:
            oldest = self.queue[0]
            now = time.perf_counter() if now is None else now
            if now - oldest.arrival > self.max_wait_s and self.used + oldest.footprint > self.budget:
                return []
        for i, head in enumerate(self.queue):
            if self.used + head.footprint > self.budget:
                continue
            group = [head]
            total = head.footprint
            for other in self.queue[i + 1:]:
                if len(group) >= self.max_batch:
                    break
                if (other.r, other.s, other.mode) != (head.r, head.s, head.mode):
                    continue
                if total + other.footprint > self.batch_bytes or \
                        self.used + total + other.footprint > self.budget:
                    break
                group.append(other)
                total += other.footprint
            for g in group:
                self.queue.remove(g)
            self.used += total
            return group
        return []

    def _worker(self, wid: int):
        torch = self.torch
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(device=self.device)
        while True:
            with self.cv:
                group = []
                while not group:
                    if self.closing and not self.queue:
                        return
                    group = self._take()
                    if not group:
                        self.cv.wait(timeout=0.05)
            t0 = time.perf_counter()
            for g in group:
                g.start = t0
                g.batched_with = len(group)
            try:
                self._run(group, stream)
            except Exception as e:  # report, never kill the worker
                for g in group:
                    g.error = str(e)
            t1 = time.perf_counter()
            with self.cv:
                self.used -= sum(g.footprint for g in group)
                for g in group:
                    g.finish = t1
                    self.completed.append(g)
                self.cv.notify_all()
            for g in group:
                g.done.set()

    def _run(self, group: list[Request], stream):
        head = group[0]
        if len(group) == 1:
            inc = nd.build_incidence(head.row_ptr, head.col, head.r, head.s, stream=stream)
            offs = np.array([0, inc.num_r], dtype=np.int64)
        else:
            inc, offs = nd.build_incidence_batch([(g.row_ptr, g.col) for g in group], head.r, head.s,
                                                 stream=stream)
        try:
            if head.mode == "snd":
                tau, iters = inc.snd(stream=stream)
            else:
                tau, iters, _ = inc.and_(notify=(head.mode == "and"), stream=stream)
        finally:
            inc.free()
        for i, g in enumerate(group):
            g.result = tau[offs[i]:offs[i + 1]].copy()
            g.iters = iters


def latency_stats(reqs) -> dict:
    lat = np.array([r.finish - r.arrival for r in reqs if r.error is None])
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None, "count": 0}
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "count": int(lat.size)}


def poisson_arrivals(rate_per_s: float, count: int, seed: int) -> np.ndarray:
    """Arrival offsets (seconds) of a Poisson process."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
