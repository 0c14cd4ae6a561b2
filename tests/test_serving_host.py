"""Host logic of the serving loop (no GPU): FIFO admission bounded by rows,
rejection of queries that can never fit, cancellation of queued queries,
back-pressure under a slow executor, and that every admitted query is
answered exactly once."""
import numpy as np

from paper_2301_03636_gb300 import serving


def q(qid, rows, t=0.0):
    return serving.Query(qid, np.full((rows, 16), qid, dtype=np.int64), t)


def test_batches_are_fifo_and_bounded():
    b = serving.Batcher(max_rows=100, max_queries=3)
    for i, r in enumerate([40, 50, 20, 5, 5]):
        assert b.submit(q(i, r))
    first = b.next_batch()
    assert [x.qid for x in first] == [0, 1]            # 40 + 50; 20 would overflow, no overtaking
    second = b.next_batch()
    assert [x.qid for x in second] == [2, 3, 4]
    assert b.next_batch() == []


def test_oversized_and_empty_queries_rejected():
    b = serving.Batcher(max_rows=64, max_queries=8)
    assert not b.submit(q(0, 65))
    assert not b.submit(serving.Query(1, np.zeros((0, 16), dtype=np.int64), 0.0))
    assert [x.status for x in b.rejected] == ["rejected", "rejected"]
    assert len(b) == 0


def test_cancel_only_before_admission():
    b = serving.Batcher(max_rows=100, max_queries=8)
    for i in range(4):
        b.submit(q(i, 10))
    assert b.cancel(2)
    batch = b.next_batch()
    assert [x.qid for x in batch] == [0, 1, 3]
    assert not b.cancel(0)                              # already admitted
    assert b.cancelled[0].status == "cancelled"


def test_pack_offsets():
    batch = [q(0, 3), q(1, 1), q(2, 4)]
    desc = np.zeros((10, 16), dtype=np.int64)
    off = np.zeros(4, dtype=np.int64)
    n, k = serving.pack(batch, desc, off)
    assert (n, k) == (8, 3) and off.tolist() == [0, 3, 4, 8]
    assert desc[3, 0] == 1 and desc[7, 0] == 2


class FakeExecutor:
    """Answers a batch after `delay` seconds of a fake clock: best = index of
    the row whose first field is smallest (all equal here -> 0)."""

    def __init__(self, clock, delay):
        self.clock, self.delay = clock, delay
        self.batch, self.t = None, 0.0
        self.launched = []

    def idle(self):
        return self.batch is None

    def launch(self, batch):
        self.batch, self.t = batch, self.clock()
        self.launched.append([x.qid for x in batch])

    def poll(self):
        if self.batch is None or self.clock() < self.t + self.delay:
            return []
        out = [(self.batch, np.zeros(len(self.batch), np.int32), np.arange(len(self.batch), dtype=np.float64))]
        self.batch = None
        return out


class FakeClock:
    def __init__(self, dt):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t


def test_server_continuous_batching_with_slow_executor():
    clock = FakeClock(1e-4)
    ex = [FakeExecutor(clock, 5e-3), FakeExecutor(clock, 5e-3)]
    b = serving.Batcher(max_rows=256, max_queries=16)
    srv = serving.Server(b, ex, clock=clock)
    rng = np.random.Generator(np.random.PCG64(0))
    arrivals = np.cumsum(rng.exponential(2e-4, size=200))       # faster than the executors drain
    sizes = rng.integers(4, 64, size=200)
    queries = [q(i, int(s), float(t)) for i, (s, t) in enumerate(zip(sizes, arrivals))]
    done = srv.run(queries, cancel_at={150: 0.0}, timeout_s=1e9)
    ids = sorted(x.qid for x in done)
    assert len(ids) == len(set(ids))                             # answered once
    assert set(ids) | {150} == set(range(200)) or set(ids) == set(range(200)) - {150}
    # both executors were used and batches carried several queries (back-pressure)
    assert ex[0].launched and ex[1].launched
    assert max(len(x) for x in ex[0].launched + ex[1].launched) > 1
    assert all(x.latency >= 0 for x in done)
    # FIFO across batches: admission order is arrival order
    order = [qid for e in (ex[0].launched, ex[1].launched) for batch in e for qid in batch]
    admitted = sorted(done, key=lambda x: (x.admitted, x.arrival))
    assert [x.qid for x in admitted] == sorted(x.qid for x in done)
    assert len(order) == len(done)


def test_max_overlap_counts_batches_in_flight():
    assert serving.max_overlap([]) == 0
    assert serving.max_overlap([(0, 1), (1, 2), (2, 3)]) == 1          # back to back: never two at once
    assert serving.max_overlap([(0, 5), (1, 2), (1.5, 3), (4, 6)]) == 3
    assert serving.max_overlap([(0, 10), (2, 3), (2, 3), (9, 11)]) == 3


def test_rows_for_budget_follows_the_workspace_size():
    """Admission by device memory: the row capacity is the largest batch whose
    workspace (the library's own size function) and buffers fit the budget."""
    from paper_2301_03636_gb300 import advisor
    widths, q = (32, 128, 128, 1), 128

    def need(r):
        return advisor.workspace_bytes(widths, r, q) + r * 128 + (q + 1) * 8 + q * 12

    for budget in (40 << 20, 64 << 20, 200 << 20):
        r = serving.rows_for_budget(widths, budget, q)
        assert need(r) <= budget < need(r + 1)
    try:
        serving.rows_for_budget(widths, 1 << 10, q)
        raise AssertionError("a budget smaller than one query must be refused")
    except ValueError:
        pass


def test_threaded_pipeline_runs_batches_on_its_worker():
    """The threaded executor: launch() returns at once, the worker runs the
    pipe's launch / wait / poll, poll() hands the results back and frees it."""
    import threading
    import time as _t

    class FakePipe:
        def __init__(self):
            self.intervals, self.threads, self.pending = [], set(), None

            class Ev:
                def synchronize(self_inner):
                    _t.sleep(0.01)
            self.event = Ev()

        def launch(self, batch):
            self.threads.add(threading.get_ident())
            self.pending = batch

        def poll(self):
            b, self.pending = self.pending, None
            return [(b, [q.rows - 1 for q in b], [float(q.qid) for q in b])]

    pipe = FakePipe()
    ex = serving.ThreadedPipeline(pipe)
    try:
        qs = [serving.Query(i, np.zeros((3 + i, 16), np.int64), 0.0) for i in range(3)]
        assert ex.idle()
        ex.launch(qs)
        assert not ex.idle()
        got = []
        for _ in range(500):
            got = ex.poll()
            if got:
                break
            _t.sleep(0.002)
        assert got and [b for b in got[0][1]] == [2, 3, 4] and ex.idle()
        assert pipe.threads == {ex.thread.ident}   # the GPU calls ran on the worker thread
    finally:
        ex.close()
    assert not ex.thread.is_alive()
