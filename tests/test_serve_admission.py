"""Admission logic of the serving engine on the CPU (no GPU, no library
calls): the device-facing parts (gauge upload, batch and lattice-group
sessions, CUDA streams and memory counters) are replaced by fakes that
finish each request after a short delay, so the engine's budget accounting,
eviction and waiting can be driven through tight budgets.

The case that matters: a small field's idle session keeps memory while a
request on the largest field waits for room.  The engine must evict the
idle field to admit it (before the fix it waited forever), and a request
that cannot fit even into an empty device must raise instead of hanging."""
import threading
import time

import numpy as np
import pytest

import paper_1111_0125_gb300.serve as serve
from paper_1111_0125_gb300.serve import Request

pytestmark = []

GAUGE = {"a": 100, "b": 400, "c": 250}      # field bytes by key
SESSION = {"a": 30, "b": 120, "c": 80}      # session bytes by key


class FakeGauge:
    def __init__(self, dims, links, sloppy=None, recon=None, stream=None):
        self.key = links
        self.vh = int(np.prod(dims)) // 2
        self.handle = 1
        self.closed = False

    def close(self):
        self.closed = True


class FakeSession:
    live = 0

    def __init__(self, engine, entry, device, priority=0):
        self.engine, self.entry = engine, entry
        self.bytes = SESSION[entry.key]
        self.lib_bytes = self.bytes
        self.inbox, self.busy = [], {}
        self.lock = threading.Lock()
        FakeSession.live += 1
        self.alive = True

    def load(self):
        with self.lock:
            return len(self.inbox) + len(self.busy)

    def free_slots(self):
        return self.engine.slots - self.load()

    def submit(self, req):
        with self.lock:
            self.inbox.append(req)
        threading.Timer(0.01, self._finish, args=(req,)).start()

    def _finish(self, req):
        with self.lock:
            self.inbox.remove(req)
        self.engine._complete(req, 0, {"iters": 1, "updates": 1, "true_res": 0.0}, None)
        self.engine._wake()

    def close(self):
        assert self.load() == 0
        FakeSession.live -= 1
        self.alive = False


@pytest.fixture
def fake_engine(monkeypatch):
    monkeypatch.setattr(serve, "Gauge", FakeGauge)
    monkeypatch.setattr(serve, "_Session", FakeSession)
    monkeypatch.setattr(serve, "gauge_bytes", lambda dims, sloppy, recon: GAUGE[_key_of(dims)])
    monkeypatch.setattr(serve, "session_bytes", lambda gauge, slots, sloppy: SESSION[gauge.key])

    class Cuda:
        @staticmethod
        def memory_allocated(device=None):
            return 0

        @staticmethod
        def set_device(device):
            pass

        @staticmethod
        def Stream(device=None, priority=0):
            return None

    class Host:
        def __init__(self, a):
            self.a = a

        def pin_memory(self):
            return self

    class FakeTorch:
        cuda = Cuda

        @staticmethod
        def from_numpy(a):
            return Host(a)

    monkeypatch.setattr(serve, "torch", FakeTorch)

    def make(budget, **kw):
        gauges = {k: (_dims_of(k), k) for k in GAUGE}
        return serve.ServeEngine(gauges, {k: np.zeros((1, 3), complex) for k in GAUGE},
                                 hbm_budget=budget, slots=2, max_sessions_per_gauge=1, **kw)
    return make


DIMS = {"a": (2, 2, 2, 2), "b": (4, 4, 4, 4), "c": (4, 2, 2, 2)}


def _dims_of(k):
    return DIMS[k]


def _key_of(dims):
    return next(k for k, d in DIMS.items() if d == tuple(dims))


def _reqs(keys):
    return [Request(i, 0.0, k, k, 0.1, 1e-10) for i, k in enumerate(keys)]


def test_idle_field_is_evicted_to_admit_a_session(fake_engine):
    # room for the largest field and its session, nothing more
    eng = fake_engine(GAUGE["b"] + SESSION["b"])
    res = eng.run(_reqs(["a", "b", "c", "a", "b"]), realtime=False)
    assert [r.rid for r in res] == [0, 1, 2, 3, 4]
    assert eng.peak_used <= eng.budget
    eng.close()
    assert eng.used == 0 and FakeSession.live == 0


def test_request_beyond_the_budget_raises(fake_engine):
    eng = fake_engine(GAUGE["b"] + SESSION["b"] - 1)
    t0 = time.time()
    with pytest.raises(RuntimeError, match="cannot be admitted"):
        eng.run(_reqs(["b"]), realtime=False)
    assert time.time() - t0 < 30
    eng.close()
