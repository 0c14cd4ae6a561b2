"""Prediction-mode serving (Sec. 3: a query is one kernel's generated variants;
the answer is the variant the cost model predicts to be fastest).

Continuous batching: queries arriving while earlier batches are on the GPU
wait in a FIFO queue; whenever one of the pipelines (a model handle with its
own workspace, CUDA stream and pinned buffers, all sharing one resident
parameter block) is idle, the queued queries are packed into its next batch
up to its row capacity (admission by device memory: the capacity comes from
the pipeline's share of a device-memory budget and the library's workspace
size), copied host->device, ranked with one advisor_rank call and copied
back.  Each pipeline is driven by a host thread of its own, so that several
batches are in flight at once on different streams.  Every kernel of the
path computes each row and each kernel segment independently of the rest of
the batch, so a query's answer is the same alone and in any mix.

The host logic (Batcher, Server, the threaded executor) has no GPU
dependency and is tested on the CPU with fake executors.
"""
from __future__ import annotations

import collections
import dataclasses
import queue
import threading
import time

import numpy as np


@dataclasses.dataclass
class Query:
    qid: int
    desc: np.ndarray            # [n][16] int64
    arrival: float              # seconds (serving clock)
    admitted: float = -1.0
    done: float = -1.0
    best: int = -2
    score: float = float("nan")
    status: str = "queued"      # queued | running | done | rejected | cancelled

    @property
    def rows(self) -> int:
        return int(self.desc.shape[0])

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class Batcher:
    """FIFO admission into batches bounded by rows and queries."""

    def __init__(self, max_rows: int, max_queries: int):
        self.max_rows = int(max_rows)
        self.max_queries = int(max_queries)
        self.queue: collections.deque[Query] = collections.deque()
        self.rejected: list[Query] = []
        self.cancelled: list[Query] = []

    def submit(self, q: Query) -> bool:
        if q.rows < 1 or q.rows > self.max_rows:
            q.status = "rejected"          # can never fit a batch: refused at admission
            self.rejected.append(q)
            return False
        self.queue.append(q)
        return True

    def cancel(self, qid: int) -> bool:
        """Cancel a query that has not been admitted to a batch yet."""
        for q in self.queue:
            if q.qid == qid:
                self.queue.remove(q)
                q.status = "cancelled"
                self.cancelled.append(q)
                return True
        return False

    def next_batch(self) -> list[Query]:
        """Queued queries, oldest first, while they fit the row capacity.  A
        query that does not fit waits for the next batch (no overtaking)."""
        out, rows = [], 0
        while self.queue and len(out) < self.max_queries:
            q = self.queue[0]
            if rows + q.rows > self.max_rows:
                break
            out.append(self.queue.popleft())
            rows += q.rows
        return out

    def __len__(self):
        return len(self.queue)


def pack(batch: list[Query], desc_out: np.ndarray, off_out: np.ndarray) -> tuple[int, int]:
    """Concatenate the batch's descriptors and write segment offsets; returns
    (rows, kernels)."""
    n = 0
    off_out[0] = 0
    for i, q in enumerate(batch):
        desc_out[n:n + q.rows] = q.desc
        n += q.rows
        off_out[i + 1] = n
    return n, len(batch)


class Server:
    """Drives a Batcher and a set of executors (pipelines) on a serving clock.

    An executor provides: idle() -> bool, launch(batch) and poll() -> list of
    finished (batch, best[], score[]) results.  The GPU executor is
    GpuPipeline; tests use a fake one."""

    def __init__(self, batcher: Batcher, executors: list, clock=time.perf_counter):
        self.batcher = batcher
        self.executors = executors
        self.clock = clock
        self.finished: list[Query] = []
        # set by executors that finish batches on threads of their own, so that
        # the loop sleeps (releasing the interpreter lock) instead of spinning
        self.wake = threading.Event()
        for ex in executors:
            if hasattr(ex, "attach_wake"):
                ex.attach_wake(self.wake)

    def step(self, now: float) -> bool:
        """Collect finished batches and launch new ones; whether anything happened."""
        progressed = False
        for ex in self.executors:
            for batch, best, score in ex.poll():
                progressed = True
                t = self.clock() - self.t0
                for q, b, s in zip(batch, best, score):
                    q.best, q.score, q.done, q.status = int(b), float(s), t, "done"
                    self.finished.append(q)
        for ex in self.executors:
            if ex.idle() and len(self.batcher):
                batch = self.batcher.next_batch()
                if not batch:
                    break
                for q in batch:
                    q.admitted, q.status = now, "running"
                ex.launch(batch)
                progressed = True
        return progressed

    def run(self, queries: list[Query], cancel_at: dict | None = None, timeout_s: float = 60.0):
        """Open-loop replay: query i becomes visible at its arrival time."""
        self.t0 = self.clock()
        pending = sorted(queries, key=lambda q: q.arrival)
        i = 0
        cancel_at = dict(cancel_at or {})
        total = len(pending)
        while True:
            now = self.clock() - self.t0
            while i < total and pending[i].arrival <= now:
                self.batcher.submit(pending[i])
                i += 1
            for qid, t in list(cancel_at.items()):
                if now >= t:
                    self.batcher.cancel(qid)
                    del cancel_at[qid]
            progressed = self.step(now)
            settled = len(self.finished) + len(self.batcher.rejected) + len(self.batcher.cancelled)
            if i >= total and settled >= total:
                break
            if now > timeout_s:
                raise TimeoutError("serving replay did not finish in time")
            if not progressed:
                # nothing to do until the next arrival, a finished batch or a cancellation
                # (polled executors are checked again after at most 100 us)
                nxt = pending[i].arrival - now if i < total else 1e-3
                if cancel_at:
                    nxt = min(nxt, min(cancel_at.values()) - now)
                self.wake.wait(timeout=max(0.0, min(nxt, 1e-4)))
                self.wake.clear()
        return self.finished


class GpuPipeline:
    """One in-flight batch at a time on its own stream, with its own model
    handle (sharing the parameter block of `base`) and workspace."""

    def __init__(self, base, max_rows: int, max_queries: int, params, mu, sigma, precision="bf16",
                 eps=-1.0, eps32=0.0, host_io: bool = True):
        import ctypes

        import torch
        from . import advisor
        self.torch = torch
        self.model = advisor.Model(base.widths, max_rows, max_queries, device=base.device,
                                   param_block=base.param_block)
        self.model.set_params(params, mu, sigma)
        self.precision, self.eps, self.eps32 = precision, eps, eps32
        self.stream = torch.cuda.Stream(device=base.device)
        dev = base.device
        self.h_desc = torch.empty((max_rows, 16), dtype=torch.int64).pin_memory()
        self.h_off = torch.empty(max_queries + 1, dtype=torch.int64).pin_memory()
        self.h_best = torch.empty(max_queries, dtype=torch.int32).pin_memory()
        self.h_score = torch.empty(max_queries, dtype=torch.float64).pin_memory()
        # numpy views of the pinned buffers (packing and reading the answers)
        self.np_desc, self.np_off = self.h_desc.numpy(), self.h_off.numpy()
        self.np_best, self.np_score = self.h_best.numpy(), self.h_score.numpy()
        if not host_io:   # device copies of the batch's inputs and answers
            self.d_desc = torch.empty((max_rows, 16), dtype=torch.int64, device=dev)
            self.d_off = torch.empty(max_queries + 1, dtype=torch.int64, device=dev)
            self.d_best = torch.empty(max_queries, dtype=torch.int32, device=dev)
            self.d_score = torch.empty(max_queries, dtype=torch.float64, device=dev)
        self.event = torch.cuda.Event()
        # host_io: the kernels read the batch's descriptors and offsets from the pinned
        # host buffers and write the answers into pinned host memory (one library call
        # per batch instead of four copies around it: half the host time and half the
        # device time of a small batch); otherwise copies to and from device buffers.
        # The call goes straight to advisor_rank with the buffers' addresses (every
        # batch starts at their first element), so a batch costs no tensor views.
        self.host_io = host_io
        self._rank = advisor.lib().advisor_rank
        self._args = (self.model.handle, ctypes.c_void_p(self.h_desc.data_ptr()),
                      ctypes.c_void_p(self.h_off.data_ptr()), advisor._prec(precision), float(eps), float(eps32),
                      ctypes.c_void_p(self.h_best.data_ptr()), ctypes.c_void_p(self.h_score.data_ptr()),
                      ctypes.c_void_p(self.stream.cuda_stream))
        self._check = advisor._check
        self.batch = None
        self.nk = 0
        # batch timing: with `ref` set (an event recorded before the first timed batch),
        # every batch's start and end on this stream in ms after ref, read when the
        # batch has finished; its two events then go back to the pool
        self.ref = None
        self.intervals = []
        self._pool = []
        self._ev = None

    def idle(self) -> bool:
        return self.batch is None

    def _events(self):
        if self.ref is None:
            return None
        if self._pool:
            return self._pool.pop()
        torch = self.torch
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def launch(self, batch):
        n, k = pack(batch, self.np_desc, self.np_off)
        ev = self._events()
        if self.host_io:
            if ev:
                ev[0].record(self.stream)
            h, desc, off, prec, eps, eps32, best, score, stream = self._args
            self._check(self._rank(h, desc, n, off, k, prec, eps, eps32, best, score, None, None, stream),
                        "advisor_rank")
            if ev:
                ev[1].record(self.stream)
            self.event.record(self.stream)
            self._ev, self.batch, self.nk = ev, batch, k
            return
        torch = self.torch
        with torch.cuda.stream(self.stream):
            if ev:
                ev[0].record(self.stream)
            self.d_desc[:n].copy_(self.h_desc[:n], non_blocking=True)
            self.d_off[:k + 1].copy_(self.h_off[:k + 1], non_blocking=True)
            self.model.rank(self.d_desc[:n], self.d_off[:k + 1], self.precision, self.eps, self.eps32,
                            best=self.d_best[:k], best_score=self.d_score[:k], stream=self.stream)
            self.h_best[:k].copy_(self.d_best[:k], non_blocking=True)
            self.h_score[:k].copy_(self.d_score[:k], non_blocking=True)
            if ev:
                ev[1].record(self.stream)
            self.event.record(self.stream)
        self._ev, self.batch, self.nk = ev, batch, k

    def poll(self):
        if self.batch is None or not self.event.query():
            return []
        k = self.nk
        out = [(self.batch, self.np_best[:k].copy(), self.np_score[:k].copy())]
        if self._ev:
            a, b = self._ev
            self.intervals.append((self.ref.elapsed_time(a), self.ref.elapsed_time(b)))
            self._pool.append(self._ev)
        self._ev, self.batch = None, None
        return out


class ThreadedPipeline:
    """A pipeline driven by a worker thread of its own: launch() hands the
    batch to the worker, which packs it, enqueues the copies and the ranking
    on the pipeline's stream and waits for them; poll() returns what the
    worker finished.  The host work of different pipelines (packing,
    launches, waits; ctypes and torch release the interpreter lock) runs in
    parallel, so that one pipeline's batch is being enqueued while another's
    is on the GPU -- with one host thread, launching a small batch takes
    longer than the GPU takes to rank it, and the batches never overlap."""

    def __init__(self, pipe):
        self.pipe = pipe
        self.inbox: queue.Queue = queue.Queue(maxsize=1)
        self.results: collections.deque = collections.deque()
        self.busy = False
        self.wake: threading.Event | None = None
        self.error: BaseException | None = None
        self.thread = threading.Thread(target=self._work, daemon=True)
        self.thread.start()

    @property
    def intervals(self):
        return self.pipe.intervals

    @intervals.setter
    def intervals(self, v):
        self.pipe.intervals = v

    def idle(self) -> bool:
        return not self.busy

    def attach_wake(self, ev: threading.Event):
        self.wake = ev

    def launch(self, batch):
        self.busy = True
        self.inbox.put(batch)

    def _work(self):
        while True:
            batch = self.inbox.get()
            if batch is None:
                return
            try:
                self.pipe.launch(batch)
                self.pipe.event.synchronize()
                self.results.extend(self.pipe.poll())
            except BaseException as e:   # handed to the serving loop by poll()
                self.error = e
                self.results.append((batch, [-2] * len(batch), [float("nan")] * len(batch)))
            if self.wake is not None:
                self.wake.set()

    def poll(self):
        if self.error is not None:
            raise RuntimeError("serving pipeline failed") from self.error
        out = []
        while self.results:
            out.append(self.results.popleft())
        if out:
            self.busy = False
        return out

    def close(self):
        self.inbox.put(None)
        self.thread.join(timeout=10)


def latency_stats(finished: list[Query]) -> dict:
    lat = np.array([q.latency for q in finished if q.status == "done"]) * 1e3
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None, "n": 0}
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()), "n": int(lat.size)}


def make_queries(n_queries: int, rate_per_s: float, seed: int) -> list[Query]:
    """Poisson arrivals of queries of floor(2^U(2, 9)) variants (4..512) each,
    descriptors from the plain-method distribution."""
    from . import workloads
    sizes = workloads.make_query_sizes(n_queries, seed)
    arrivals = workloads.make_arrivals(n_queries, rate_per_s, seed)
    desc = workloads.make_descriptors(int(sizes.sum()), seed)
    out, pos = [], 0
    for i, (n, t) in enumerate(zip(sizes, arrivals)):
        out.append(Query(i, desc[pos:pos + n], float(t)))
        pos += n
    return out


def max_overlap(intervals) -> int:
    """Largest number of [start, end) intervals that contain a common instant."""
    ev = sorted([(a, 1) for a, _ in intervals] + [(b, -1) for _, b in intervals], key=lambda x: (x[0], x[1]))
    cur = best = 0
    for _, d in ev:
        cur += d
        best = max(best, cur)
    return best


def rows_for_budget(widths, budget_bytes: int, max_queries: int, lo: int = 512, hi: int = 1 << 20) -> int:
    """Admission by device memory: the largest batch (in variants) whose
    pipeline fits `budget_bytes` of device memory -- the library's workspace
    for that many rows (advisor_workspace_bytes) plus the pipeline's own
    device buffers (descriptors, offsets, answers).  Raises if not even `lo`
    rows (the largest query) fit."""
    from . import advisor

    def need(r):
        return advisor.workspace_bytes(widths, r, max_queries) + r * 128 + (max_queries + 1) * 8 + max_queries * 12

    if need(lo) > budget_bytes:
        raise ValueError(f"a device-memory budget of {budget_bytes} B does not fit a batch of {lo} variants")
    while lo < hi:   # need() grows with the rows
        mid = (lo + hi + 1) // 2
        if need(mid) <= budget_bytes:
            lo = mid
        else:
            hi = mid - 1
    return lo


def run_serving(base, params, mu, sigma, queries: list[Query], precision="bf16", eps=-1.0, eps32=0.0,
                pipelines: int = 3, max_rows: int = 8192, max_queries: int = 128, warmup: bool = True,
                memory_budget_bytes: int | None = None, threads: bool = True, host_io: bool = True):
    """Serve `queries` (open loop, real clock) with `pipelines` batches in
    flight; returns (finished queries, stats).  With memory_budget_bytes, each
    pipeline's row capacity (the admission bound of a batch) comes from its
    share of that device-memory budget instead of max_rows.  The stats report
    the largest number of batches whose copy-in .. copy-out intervals
    overlapped in device time (max_batches_in_flight)."""
    import torch
    if memory_budget_bytes is not None:
        max_rows = rows_for_budget(base.widths, memory_budget_bytes // pipelines, max_queries)
    pipes = [GpuPipeline(base, max_rows, max_queries, params, mu, sigma, precision, eps, eps32, host_io)
             for _ in range(pipelines)]
    if warmup:   # first launches (module load, attribute setup) outside the replay
        w = [Query(-1 - i, q.desc, 0.0) for i, q in enumerate(queries[:pipelines])]
        for p, qq in zip(pipes, w):
            p.launch([qq])
        torch.cuda.synchronize()
        for p in pipes:
            p.poll()
    ref = torch.cuda.Event(enable_timing=True)
    ref.record()
    for p in pipes:
        p.intervals = []
        p.ref = ref
    execs = [ThreadedPipeline(p) for p in pipes] if threads else pipes
    batcher = Batcher(max_rows, max_queries)
    srv = Server(batcher, execs)
    t0 = time.perf_counter()
    try:
        done = srv.run(queries)
    finally:
        if threads:
            for ex in execs:
                ex.close()
    wall = time.perf_counter() - t0
    torch.cuda.synchronize()
    iv = [x for p in pipes for x in p.intervals]
    st = latency_stats(done)
    st["batches"] = len(iv)
    st["max_batches_in_flight"] = max_overlap(iv)
    st["rows_per_batch_capacity"] = max_rows
    st["queries_per_s"] = len(done) / wall
    st["variants_per_s"] = sum(q.rows for q in done) / wall
    st["rejected"] = len(batcher.rejected)
    st["pipelines"] = pipelines
    st["host_threads"] = pipelines if threads else 1
    return done, st
