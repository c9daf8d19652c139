"""Host logic of the open-loop serving driver (ccs.serve_stream): output
slots of a ring are reused only after the request that held them has been
collected, results come back in submission order, and a failed collection
is raised on the submitting thread.  A fake server stands in for the
library (no GPU)."""
import threading
import time

import pytest

from paper_1508_01256_gb300 import ccs


class _Info:
    def __init__(self, ticket):
        self.ticket = ticket


class FakeServer:
    """Tickets complete in order, `delay_s` after the collector asks."""

    def __init__(self, delay_s=0.0005, fail_at=None):
        self.delay_s = delay_s
        self.fail_at = fail_at
        self.submitted = []
        self.collected = set()
        self.lock = threading.Lock()

    def submit(self, *req):
        with self.lock:
            self.submitted.append(req)
            return len(self.submitted) - 1

    def wait(self, ticket, timeout_ms):
        time.sleep(self.delay_s)
        if ticket == self.fail_at:
            return None
        with self.lock:
            self.collected.add(ticket)
        return _Info(ticket)


def test_ring_slots_are_reused_only_after_collection():
    srv = FakeServer()
    ring, count = 4, 40
    violations = []

    def request_of(q):
        # request q takes slot q % ring: request q - ring must be collected
        if q >= ring and (q - ring) not in srv.collected:
            violations.append(q)
        return (q, q % ring)

    infos, waited = ccs.serve_stream(srv, request_of, count, [0.0] * count, ring)
    assert not violations
    assert [i.ticket for i in infos] == list(range(count))
    assert [r[0] for r in srv.submitted] == list(range(count))
    # every arrival is at t = 0, so the submitter runs ahead of the collector
    # and has to wait for slots
    assert waited > 0


def test_no_waits_when_the_ring_covers_the_stream():
    srv = FakeServer(delay_s=0.0)
    infos, waited = ccs.serve_stream(srv, lambda q: (q,), 16, [0.0] * 16, ring=16)
    assert waited == 0 and len(infos) == 16


def test_arrival_times_are_respected():
    srv = FakeServer(delay_s=0.0)
    arrivals = [0.0, 0.02, 0.04]
    stamps = []

    def request_of(q):
        stamps.append(time.perf_counter())
        return (q,)

    t0 = time.perf_counter()
    ccs.serve_stream(srv, request_of, 3, arrivals, ring=8)
    for at, ts in zip(arrivals, stamps):
        assert ts - t0 >= at - 1e-3


def test_a_failed_collection_is_raised():
    srv = FakeServer(fail_at=5)
    with pytest.raises(RuntimeError, match="request 5"):
        ccs.serve_stream(srv, lambda q: (q,), 20, [0.0] * 20, ring=4, timeout_ms=2000)
