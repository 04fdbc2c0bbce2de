"""Host logic of the continuous-batching scheduler, with a fake executor (no GPU)."""
import time

import numpy as np

from paper_2406_09144_gb300.serve import Request, Scheduler, estimate_bytes, summarize


class FakeExecutor:
    """Each call takes `dur` seconds of wall time; records concurrency."""

    def __init__(self, dur=0.004):
        self.dur = dur
        self.busy_until = {}
        self.live = set()
        self.max_live = 0
        self.order = []

    def admit(self, r):
        self.order.append(r.rid)
        self.live.add(r.rid)
        self.max_live = max(self.max_live, len(self.live))
        self.busy_until[r.rid] = time.perf_counter()
        return r

    def ready(self, r):
        return time.perf_counter() >= self.busy_until[r.rid]

    def issue(self, r):
        self.busy_until[r.rid] = time.perf_counter() + self.dur

    def finish(self, r):
        r.result = np.full(3, r.rid, dtype=np.float32)
        self.live.discard(r.rid)


def _req(i, nx, arrival, ncalls=3):
    return Request(rid=i, kind="psf" if i % 2 else "major", uvw=np.zeros((1000, 3)),
                   freqs=np.array([1e9]), weights=None, nx=nx, ny=nx, pixsize=1e-5,
                   sky=np.zeros((1, 1, nx, nx), np.float32), ncalls=ncalls, arrival=arrival)


def test_admission_respects_budget_slots_and_fifo():
    reqs = [_req(i, 256 if i % 3 else 1024, arrival=0.002 * i) for i in range(24)]
    budget = estimate_bytes(_req(0, 1024, 0)) * 2 + estimate_bytes(_req(1, 256, 0))
    ex = FakeExecutor()
    sch = Scheduler(ex, budget, max_active=4)
    t0 = time.perf_counter()
    done = sch.run(reqs)
    wall = time.perf_counter() - t0
    assert sch.peak_bytes <= budget
    assert ex.max_live <= 4 and sch.peak_active >= 2
    assert ex.order == sorted(ex.order)  # FIFO admission
    for r in done:
        assert r.result is not None and r.result[0] == r.rid
        assert r.arrival <= r.t_admit <= r.t_done
    s = summarize(done, wall)
    assert s["requests"] == 24 and s["p99_ms"] >= s["p50_ms"] > 0


def test_jobs_arriving_later_join_while_others_run():
    reqs = [_req(0, 256, 0.0, ncalls=10), _req(1, 256, 0.01, ncalls=2)]
    sch = Scheduler(FakeExecutor(0.005), 10 ** 12, max_active=4)
    sch.run(reqs)
    ev = [(e[0], e[1]) for e in sch.log]
    # job 1 is admitted before job 0 finishes: continuous batching, not a queue
    assert ev.index(("admit", 1)) < ev.index(("done", 0))
    assert reqs[1].t_done < reqs[0].t_done


def test_request_larger_than_budget_is_refused():
    import pytest
    with pytest.raises(ValueError):
        Scheduler(FakeExecutor(), 1000, 2).run([_req(0, 256, 0.0)])


def test_capture_gate_keeps_cleanup_apart_from_captures():
    """Plan and graph destruction (device-synchronising) never overlaps a graph capture: the
    exclusive section waits for captures in progress and holds new captures back."""
    import threading
    import time as _time
    from paper_2406_09144_gb300.serve import CaptureGate

    gate = CaptureGate()
    log = []
    lock = threading.Lock()

    def note(x):
        with lock:
            log.append(x)

    def capture(i, hold):
        with gate.capture():
            note(("cap+", i))
            _time.sleep(hold)
            note(("cap-", i))

    def cleanup():
        with gate.exclusive():
            note(("free+", 0))
            _time.sleep(0.05)
            note(("free-", 0))

    a = threading.Thread(target=capture, args=(1, 0.2))
    b = threading.Thread(target=capture, args=(2, 0.2))
    a.start()
    b.start()
    _time.sleep(0.05)  # both captures are in progress
    c = threading.Thread(target=cleanup)
    c.start()
    _time.sleep(0.05)  # cleanup is now waiting; a new capture must wait behind it
    d = threading.Thread(target=capture, args=(3, 0.01))
    d.start()
    for t in (a, b, c, d):
        t.join(5)
    active = 0
    freeing = False
    for kind, _ in log:
        if kind == "cap+":
            assert not freeing
            active += 1
        elif kind == "cap-":
            active -= 1
        elif kind == "free+":
            assert active == 0
            freeing = True
        else:
            freeing = False
    assert [k for k, i in log if i == 3] == ["cap+", "cap-"]
    assert log.index(("cap+", 3)) > log.index(("free-", 0))
    # two captures ran concurrently
    assert log.index(("cap+", 2)) < log.index(("cap-", 1)) or log.index(("cap+", 1)) < log.index(("cap-", 2))
