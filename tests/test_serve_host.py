"""Host logic of the serving loop, on CPU: admission in arrival order under the
memory budget and the slot count, failures reported through each request's
future, and a slot that cannot start failing the queue instead of hanging it.
The device work is replaced by a stub; the GPU tests run the real solves."""
import threading
import time

import numpy as np
import pytest

pytest.importorskip("torch")
from paper_2405_11168_gb300 import serve  # noqa: E402


class StubServer(serve.Server):
    """Server whose requests take a given time and size instead of running solves."""

    def __init__(self, *a, fail_start=False, **kw):
        self.fail_start = fail_start
        self.log = []
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0
        super().__init__(*a, device="cuda:0", **kw)

    def request_bytes(self, req):
        return req.tag["bytes"]

    def _start_slot(self):
        if self.fail_start:
            raise RuntimeError("no device")
        return None

    def _run(self, req, stream):
        with self.lock:
            self.log.append(req.tag["id"])
            self.active += 1
            self.max_active = max(self.max_active, self.active)
        try:
            time.sleep(req.tag.get("sleep", 0.02))
            if req.tag.get("fail"):
                raise ValueError(f"request {req.tag['id']} failed")
            return serve.Result(tag=req.tag, sig_eff=np.zeros((1, 6)), iters=[1], errs=[0.0], status=[0])
        finally:
            with self.lock:
                self.active -= 1


def _req(i, nbytes, **kw):
    return serve.Request(ids=np.zeros((4, 4, 4), np.uint8), table=np.zeros((1, 6, 6)), loads=[np.zeros(6)],
                         tag=dict(id=i, bytes=nbytes, **kw))


@pytest.mark.timeout(60)
def test_admission_in_order_within_budget_and_slots():
    srv = StubServer(budget_bytes=100, slots=3)
    sizes = [60, 30, 30, 50, 10, 90, 20, 40]
    futs = [srv.submit(_req(i, b)) for i, b in enumerate(sizes)]
    res = [f.result(timeout=30) for f in futs]
    srv.close()
    assert [r.tag["id"] for r in res] == list(range(len(sizes)))
    assert all(r.bytes == b for r, b in zip(res, sizes))
    assert srv.log == list(range(len(sizes)))          # admitted in arrival order
    assert srv.max_used <= 100 and srv.max_running <= 3 and srv.max_active <= 3
    assert srv.max_running >= 2                          # requests that fit together did overlap
    assert srv.used == 0 and srv.running == 0


@pytest.mark.timeout(60)
def test_failure_reaches_its_future_and_others_complete():
    srv = StubServer(budget_bytes=100, slots=2)
    futs = [srv.submit(_req(i, 40, fail=(i == 1))) for i in range(4)]
    with pytest.raises(ValueError, match="request 1 failed"):
        futs[1].result(timeout=30)
    assert [futs[i].result(timeout=30).tag["id"] for i in (0, 2, 3)] == [0, 2, 3]
    srv.close()
    assert srv.used == 0


@pytest.mark.timeout(60)
def test_request_above_budget_is_refused():
    srv = StubServer(budget_bytes=100, slots=1)
    with pytest.raises(ValueError):
        srv.submit(_req(0, 101))
    srv.close()
    with pytest.raises(RuntimeError):
        srv.submit(_req(1, 10))


@pytest.mark.timeout(60)
def test_slot_that_cannot_start_fails_pending_requests():
    srv = StubServer(budget_bytes=100, slots=2, fail_start=True)
    for t in srv._workers:
        t.join(timeout=10)
    with pytest.raises(RuntimeError):
        f = srv.submit(_req(0, 10))     # the queue is closed once a slot fails
        f.result(timeout=10)
