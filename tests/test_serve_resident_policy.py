"""Host policy of the resident serving loop (``serve.ResidentScheduler.step``) on the
CPU, against a stand-in for the C server: admission in arrival order, a request
whose graph has no free handle waits without holding up requests on other graphs,
a busy server (no free request slot) keeps the order, completions return handles
and count served edge·samples, and the queue bound and the sample limit shed."""
import collections
import threading
import types

from paper_2501_00675_gb300.serve import RequestSpec, ResidentScheduler


class FakeServer:
    """Stand-in for binding.ResidentServer: `slots` requests at once; poll reports a
    request complete once the test has marked it."""

    def __init__(self, slots):
        self.slots = slots
        self.running = {}
        self.finished = set()
        self.next = 1
        self.log = []

    def submit(self, handle, num_samples, seed, out):
        if len(self.running) >= self.slots:
            return None
        rid = self.next
        self.next += 1
        self.running[rid] = (handle, num_samples, seed)
        self.log.append((handle, num_samples, seed))
        return rid

    def poll(self, rid, allow_overflow=False):
        if rid in self.finished:
            del self.running[rid]
            self.finished.discard(rid)
            return 0.5
        return None


def make(handles_per_graph, edges, slots=8, max_queue=16, max_samples=1000):
    sch = ResidentScheduler.__new__(ResidentScheduler)
    sch.torch = None
    sch.cg = types.SimpleNamespace(CosError=RuntimeError)
    sch.info = [{"E": e} for e in edges]
    sch.free = collections.defaultdict(list)
    for gid, n in enumerate(handles_per_graph):
        for q in range(n):
            sch.free[gid].append((f"h{gid}.{q}", None))
    sch.srv = FakeServer(slots)
    sch.max_queue, sch.max_samples = max_queue, max_samples
    sch.queue, sch.inflight, sch.requests = collections.deque(), [], []
    sch._lock, sch._inbox, sch._rid = threading.Lock(), collections.deque(), 0
    sch.shed, sch.units_done = 0, 0.0
    return sch


def test_waiting_graph_does_not_block_others():
    sch = make([1, 1], [10, 20])
    a = sch.submit(RequestSpec(0, 100, 1))
    b = sch.submit(RequestSpec(0, 200, 2))   # graph 0's only handle is taken by a
    c = sch.submit(RequestSpec(1, 300, 3))
    assert sch.step()
    assert [a.status, b.status, c.status] == ["running", "queued", "running"]
    assert [x[2] for x in sch.srv.log] == [1, 3]
    sch.srv.finished.add(a._sid)
    sch.step()                                # a completes, b takes the handle
    assert a.status == "done" and a.mean == 0.5 and b.status == "running"
    assert sch.units_done == 10 * 100
    sch.srv.finished.update([b._sid, c._sid])
    sch.step()
    assert b.status == c.status == "done"
    assert sch.units_done == 10 * 100 + 10 * 200 + 20 * 300
    assert not sch.step()


def test_busy_server_keeps_arrival_order():
    sch = make([3, 3], [1, 1], slots=2)
    reqs = [sch.submit(RequestSpec(q % 2, 10 + q, q)) for q in range(5)]
    sch.step()
    assert [r.status for r in reqs] == ["running", "running", "queued", "queued", "queued"]
    assert [r.spec.seed for r in sch.queue] == [2, 3, 4]
    sch.srv.finished.add(reqs[0]._sid)
    sch.step()
    assert reqs[2].status == "running" and [r.spec.seed for r in sch.queue] == [3, 4]


def test_shedding():
    sch = make([1], [1], slots=1, max_queue=2, max_samples=1000)
    big = sch.submit(RequestSpec(0, 5000, 0))        # more samples than a handle holds
    rs = [sch.submit(RequestSpec(0, 10, q)) for q in range(1, 5)]
    sch.step()
    assert big.status == "shed"
    # the first two enter the queue (bound 2) and one of them starts; the rest are shed
    assert [r.status for r in rs] == ["running", "queued", "shed", "shed"]
    assert sch.shed == 3


def test_held_work_cap_keeps_age_order():
    """The server is handed requests oldest first while the work it holds (edges x
    samples of unfinished requests) stays within the cap; the first request always
    fits, a request waiting for the cap holds back every younger one, and a finished
    request frees its share."""
    sch = make([4, 4], [10, 10], slots=8)
    sch.max_inflight, sch.max_inflight_work = 8, 10 * 500
    big = sch.submit(RequestSpec(0, 900, 1))          # larger than the cap: runs alone
    small = [sch.submit(RequestSpec(1, 100, 2 + q)) for q in range(5)]
    sch.step()
    assert big.status == "running" and all(r.status == "queued" for r in small)
    sch.srv.finished.add(big._sid)
    sch.step()                                        # big done: four of 100 (4000 <= 5000) start
    assert big.status == "done"
    assert [r.status for r in small] == ["running"] * 4 + ["queued"]
    sch.max_inflight = 2                              # the count cap binds as well
    sch.srv.finished.update([small[0]._sid, small[1]._sid, small[2]._sid])
    sch.step()
    assert small[4].status == "running" and sum(r.status == "running" for r in small) == 2
