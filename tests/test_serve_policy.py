"""Host-side policy of the serving loop (no GPU): FIFO admission under a device
memory budget, bounded queue with load shedding, memory release, latency summary."""
import numpy as np

from paper_2501_00675_gb300.serve import AdmissionController, Request, RequestSpec, latency_summary


def _req(i, need):
    return Request(RequestSpec(0, 100, i), need, float(i), i)


def test_fifo_admission_respects_budget_and_order():
    ac = AdmissionController(budget_bytes=100, max_queue=10)
    reqs = [_req(i, n) for i, n in enumerate([40, 40, 30, 10, 90])]
    for r in reqs:
        assert ac.offer(r)
    first = ac.admit(max_n=10)
    assert [r.rid for r in first] == [0, 1]          # 40 + 40; 30 does not fit -> head of line waits
    assert ac.in_use == 80 and ac.peak == 80
    assert ac.admit(10) == []
    ac.release(first[0])
    nxt = ac.admit(10)
    assert [r.rid for r in nxt] == [2, 3]             # 40 + 30 + 10 = 80; 90 waits at the head
    assert ac.in_use == 80
    for r in (first[1], nxt[0], nxt[1]):
        ac.release(r)
    assert [r.rid for r in ac.admit(10)] == [4]
    assert ac.peak <= 100


def test_shedding_and_max_batch():
    ac = AdmissionController(budget_bytes=100, max_queue=3)
    assert not ac.offer(_req(0, 101))                 # can never fit
    assert all(ac.offer(_req(i, 1)) for i in range(1, 4))
    assert not ac.offer(_req(4, 1))                   # queue full
    assert ac.shed == 2
    assert len(ac.admit(max_n=2)) == 2 and len(ac.queue) == 1


def test_random_stream_never_exceeds_budget():
    rng = np.random.default_rng(0)
    ac = AdmissionController(budget_bytes=1000, max_queue=50)
    running = []
    for step in range(2000):
        if rng.random() < 0.6:
            ac.offer(_req(step, int(rng.integers(1, 400))))
        running += ac.admit(int(rng.integers(1, 5)))
        assert ac.in_use <= 1000
        if running and rng.random() < 0.5:
            ac.release(running.pop(int(rng.integers(0, len(running)))))
    assert ac.peak <= 1000 and ac.admitted > 100


def test_latency_summary():
    rs = []
    for i in range(100):
        r = _req(i, 1)
        r.status = "done"
        r.t_submit = 0.0
        r.t_done = (i + 1) / 1000.0
        rs.append(r)
    s = latency_summary(rs)
    assert s["completed"] == 100
    assert abs(s["p50_ms"] - 50.5) < 1e-6 and 99 < s["p99_ms"] <= 100


def test_reclaim_and_resource_veto():
    ac = AdmissionController(budget_bytes=100, max_queue=10)
    for i in range(3):
        ac.offer(_req(i, 50))
    idle = [30, 30]                                   # memory held by idle handles, reclaimable

    def reclaim(n):
        freed = 0
        while freed < n and idle:
            freed += idle.pop()
        return freed

    ac.in_use = 60                                    # two idle handles charged
    got = ac.admit(10, cost=lambda r: 40, reclaim=reclaim)
    assert [r.rid for r in got] == [0, 1] and ac.in_use == 80 and idle == []
    assert ac.admit(10, cost=lambda r: 40, reclaim=reclaim) == []     # nothing left to reclaim
    ac.release(nbytes=40)
    blocked = ac.admit(10, cost=lambda r: 10, can_run=lambda r: False)
    assert blocked == [] and len(ac.queue) == 1       # vetoed head stays queued
    seen = []
    assert [r.rid for r in ac.admit(10, cost=lambda r: 10, on_admit=seen.append)] == [2]
    assert [r.rid for r in seen] == [2] and ac.peak <= 100
