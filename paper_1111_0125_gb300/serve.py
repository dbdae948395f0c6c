"""Serving loop: a stream of solve requests with continuous batching.

Requests (lattice, gauge field, mass, tolerance, source) arrive over time.
Each resident gauge field has batch sessions (``stg_batch_*``): a session
holds the device state of up to `slots` systems and advances all of them by
one chunk of CG iterations per step; between steps finished systems leave
and newly arrived requests take their slots, so requests that arrive while
others are on the GPU join the running batch instead of waiting for it to
drain.  Every session runs on its own CUDA stream in its own host thread
(the C calls release the GIL), so sessions of different gauge fields and
lattices overlap on the device.

Admission is by an HBM budget: a gauge field is uploaded (at most
`max_resident` at a time, least recently used idle one evicted) and a
session created only while the budget allows; otherwise the request waits
until memory frees.  The count charges a gauge field with the library's
resident bytes for its handle (FP64 and sloppy links, tile-major copies,
workspace scalars) and a session with its batch state plus the source and
solution buffers of every slot, so everything a request causes on the device
is counted before it is admitted and released when its session closes.
`peak_used` is the largest count seen; `peak_measured` the largest device
usage measured during the run (live torch allocations of the engine plus the
library's bytes of every live handle and session).  Latency is measured per
request from its arrival to the moment its solution is back in host memory.

With `group_max_vh` > 0, requests on lattices of at most that many sites per
parity go to lattice-group sessions (``stg_lgroup_*``) instead: systems of
different small lattices and gauge fields share one session and iterate in
lock-step, four launches per iteration for all of them, on one stream and
one host thread.  A gauge field stays resident while any of its requests is
in a group.

With `priority_by_size`, sessions of smaller lattices run on higher-priority
CUDA streams, so their short kernels are scheduled ahead of the long
kernels of large lattices (shortest job first at the level of thread
blocks); the largest lattice keeps the default priority.

This module only schedules: every solve runs in the CUDA library through the
C ABI.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time

import numpy as np
import torch

from . import (STG_FP32, STG_OK, stg_batch_add, stg_batch_bytes, stg_batch_create,
               stg_batch_destroy, stg_batch_step, stg_cg_params_default, stg_gauge_bytes,
               stg_lgroup_add, stg_lgroup_bytes, stg_lgroup_create, stg_lgroup_destroy,
               stg_lgroup_step)
from .fields import Gauge


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the stream
    gauge_key: object       # key into the gauge table
    source_key: object      # key into the source table
    mass: float
    tol: float


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    done: float
    status: int
    iters: int
    updates: int
    true_res: float
    x: np.ndarray | None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def gauge_bytes(dims, sloppy: int = STG_FP32, recon: int = 12) -> int:
    """Device bytes a handle keeps resident (the library's own count: FP64
    links, sloppy links and their tile-major copies) plus its workspace
    scalars."""
    return stg_gauge_bytes(dims, sloppy, recon) + 4096


def session_bytes(gauge, slots: int, sloppy: int) -> int:
    """Device bytes of one batch session: the library's count of its state
    plus a complex128 source and solution buffer (48 bytes per site each)
    for every slot."""
    return stg_batch_bytes(gauge.handle, slots, sloppy) + 2 * slots * gauge.vh * 48


class _Session:
    """One batch session on one resident gauge field, driven by a thread."""

    def __init__(self, engine, entry, device, priority=0):
        self.engine = engine
        self.entry = entry
        self.stream = torch.cuda.Stream(device=device, priority=priority)
        params = stg_cg_params_default(entry.gauge.handle)
        params.sloppy = engine.sloppy
        params.check_every = engine.chunk
        self.handle = stg_batch_create(entry.gauge.handle, engine.slots, params, self.stream)
        self.lib_bytes = stg_batch_bytes(entry.gauge.handle, engine.slots, engine.sloppy)
        self.vh = entry.gauge.vh
        # batch state plus one source and one solution buffer per slot
        self.bytes = session_bytes(entry.gauge, engine.slots, engine.sloppy)
        self.device = device
        self.busy = {}            # slot -> (request, source buffer, solution buffer)
        self.inbox = collections.deque()
        self.cv = threading.Condition()
        self.stop = False
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def load(self) -> int:
        with self.cv:
            return len(self.busy) + len(self.inbox)

    def free_slots(self) -> int:
        return self.engine.slots - self.load()

    def submit(self, req: Request):
        with self.cv:
            self.inbox.append(req)
            self.cv.notify()

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify()
        self.thread.join()
        stg_batch_destroy(self.handle)

    def _admit(self, req: Request):
        host = self.engine.sources[req.source_key]
        with torch.cuda.stream(self.stream):
            # buffers live until the system is reported done (stream-ordered
            # caching allocator on the session stream)
            src = torch.empty((self.vh, 3), dtype=torch.complex128, device=self.device)
            src.copy_(host, non_blocking=True)
            x = torch.zeros_like(src)
        self.engine._sample_memory()
        slot = stg_batch_add(self.handle, src, x, req.mass, req.tol)
        self.busy[slot] = (req, src, x)

    def _run(self):
        torch.cuda.set_device(self.engine.device)
        eng = self.engine
        while True:
            with self.cv:
                while not self.stop and not self.inbox and not self.busy:
                    self.cv.wait()
                if self.stop and not self.busy and not self.inbox:
                    return
                new = []
                while self.inbox and len(self.busy) + len(new) < eng.slots:
                    new.append(self.inbox.popleft())
            for req in new:
                self._admit(req)
            done, _ = stg_batch_step(self.handle, eng.slots)
            for slot, status, st in done:
                req, src, x = self.busy.pop(slot)
                with torch.cuda.stream(self.stream):
                    xh = x.to("cpu", non_blocking=True)
                self.stream.synchronize()
                # release the slot's device buffers now, before the next
                # admission allocates its own (the budget counts one pair per slot)
                del src, x
                eng._complete(req, status, st, xh.numpy() if eng.keep_solutions else None)
            if done:
                eng._wake()


def group_bytes(slots: int, max_vh: int, sloppy: int) -> int:
    """Device bytes of one lattice-group session: the library's count plus a
    complex128 source and solution buffer of max_vh sites for every slot."""
    return stg_lgroup_bytes(slots, max_vh, sloppy) + 2 * slots * max_vh * 48


class _GroupSession(_Session):
    """A lattice-group session: its slots take requests on any resident
    gauge field of at most max_vh sites per parity."""

    def __init__(self, engine, device, priority=0):
        self.engine = engine
        self.entry = None
        self.stream = torch.cuda.Stream(device=device, priority=priority)
        params = stg_cg_params_default(None)
        params.sloppy = engine.sloppy
        params.delta = engine.group_delta
        params.check_every = engine.chunk
        self.max_vh = engine.group_max_vh
        self.nslots = engine.group_slots
        self.handle = stg_lgroup_create(self.nslots, self.max_vh, engine.sloppy, engine.recon,
                                        params, self.stream)
        self.lib_bytes = stg_lgroup_bytes(self.nslots, self.max_vh, engine.sloppy)
        self.bytes = group_bytes(self.nslots, self.max_vh, engine.sloppy)
        self.device = device
        self.busy = {}
        self.inbox = collections.deque()
        self.cv = threading.Condition()
        self.stop = False
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def free_slots(self) -> int:
        return self.nslots - self.load()

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify()
        self.thread.join()
        stg_lgroup_destroy(self.handle)

    def _admit(self, item):
        req, entry = item
        host = self.engine.sources[req.source_key]
        vh = entry.gauge.vh
        with torch.cuda.stream(self.stream):
            src = torch.empty((vh, 3), dtype=torch.complex128, device=self.device)
            src.copy_(host, non_blocking=True)
            x = torch.zeros_like(src)
        self.engine._sample_memory()
        slot = stg_lgroup_add(self.handle, entry.gauge.handle, src, x, req.mass, req.tol)
        self.busy[slot] = (item, src, x)

    def _run(self):
        torch.cuda.set_device(self.engine.device)
        eng = self.engine
        while True:
            with self.cv:
                while not self.stop and not self.inbox and not self.busy:
                    self.cv.wait()
                if self.stop and not self.busy and not self.inbox:
                    return
                new = []
                while self.inbox and len(self.busy) + len(new) < self.nslots:
                    new.append(self.inbox.popleft())
            for item in new:
                self._admit(item)
            done, _ = stg_lgroup_step(self.handle, self.nslots)
            for slot, status, st in done:
                (req, entry), src, x = self.busy.pop(slot)
                with torch.cuda.stream(self.stream):
                    xh = x.to("cpu", non_blocking=True)
                self.stream.synchronize()
                del src, x
                with eng.lock:
                    entry.in_groups -= 1
                eng._complete(req, status, st, xh.numpy() if eng.keep_solutions else None)
            if done:
                eng._wake()


@dataclasses.dataclass
class _GaugeEntry:
    key: object
    gauge: Gauge
    bytes: int
    sessions: list
    last_used: float
    in_groups: int = 0      # requests of this field inside lattice-group sessions


class ServeEngine:
    """Continuous-batching solve server on one GPU.

    gauges:  key -> (dims, canonical host links)
    sources: key -> canonical host source (complex128 [Vh][3]); pinned on entry
    """

    def __init__(self, gauges: dict, sources: dict, hbm_budget: float = 120e9, slots: int = 4,
                 max_sessions_per_gauge: int = 2, max_resident: int = 8, sloppy: int = STG_FP32,
                 recon: int = 12, chunk: int = 16, keep_solutions: bool = False, device: int = 0,
                 priority_by_size: bool = True, group_max_vh: int = 0, group_slots: int = 8,
                 max_groups: int = 2, group_delta: float | None = None):
        self.gauge_src = gauges
        self.sources = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
                        for k, v in sources.items()}
        self.budget = float(hbm_budget)
        self.slots = int(slots)
        self.max_sessions = int(max_sessions_per_gauge)
        self.max_resident = int(max_resident)
        self.sloppy = sloppy
        self.recon = recon
        self.chunk = chunk
        self.keep_solutions = keep_solutions
        self.device = device
        self.priority_by_size = priority_by_size
        self.group_max_vh = int(group_max_vh)
        self.group_slots = int(group_slots)
        self.max_groups = int(max_groups)
        # the library's per-precision default reliable-update threshold
        self.group_delta = (group_delta if group_delta is not None else
                            0.1 if sloppy == 0 else 0.05 if sloppy == STG_FP32 else 0.25)
        self.groups: list = []
        vols = sorted({int(np.prod(d)) for d, _ in gauges.values()})
        # stream priority per lattice volume: 0 for the largest, one step
        # higher (more negative) per distinct larger volume
        self._prio = {v: -(len(vols) - 1 - k) for k, v in enumerate(vols)}
        self.used = 0.0
        self.peak_used = 0.0
        self.peak_measured = 0.0
        self._alloc_base = torch.cuda.memory_allocated(device)
        self.resident: dict = {}
        self.results: list = []
        self.lock = threading.Lock()
        self.event = threading.Event()
        self.t0 = None
        torch.cuda.set_device(device)
        self.upload_stream = torch.cuda.Stream(device=device)

    # -- bookkeeping called from session threads --------------------------
    def _complete(self, req, status, st, x):
        t = time.perf_counter() - self.t0
        with self.lock:
            self.results.append(Result(req.rid, req.arrival, t, status, st["iters"],
                                       st["updates"], st["true_res"], x))

    def _wake(self):
        self.event.set()

    def _lib_bytes(self) -> int:
        n = 0
        for e in list(self.resident.values()):
            n += e.bytes
            n += sum(s.lib_bytes for s in list(e.sessions))
        n += sum(s.lib_bytes for s in list(self.groups))
        return n

    def _sample_memory(self):
        """Device bytes in use now: the engine's live torch tensors (request
        buffers) plus the library's bytes of every live handle and session."""
        live = torch.cuda.memory_allocated(self.device) - self._alloc_base
        m = live + self._lib_bytes()
        if m > self.peak_measured:
            self.peak_measured = float(m)
        if self.used > self.peak_used:
            self.peak_used = float(self.used)

    # -- placement ----------------------------------------------------------
    def _idle_gauges(self, keep=None):
        return [g for g in self.resident.values()
                if g is not keep and all(s.load() == 0 for s in g.sessions) and g.in_groups == 0]

    def _make_room(self, need, keep=None, slots_for_gauge=False) -> bool:
        """Evict idle gauge fields (least recently used first, never `keep`)
        and close idle lattice-group sessions until `need` more bytes fit the
        budget (and, for a new field, the resident count allows one more).
        False if nothing idle is left to free."""
        while (self.used + need > self.budget or
               (slots_for_gauge and len(self.resident) >= self.max_resident)):
            idle = self._idle_gauges(keep)
            if idle:
                self._evict(min(idle, key=lambda g: g.last_used))
                continue
            idle_groups = [g for g in self.groups if g.load() == 0]
            if idle_groups and self.used + need > self.budget:
                g = idle_groups[0]
                g.close()
                self.used -= g.bytes
                self.groups.remove(g)
                continue
            return False
        return True

    def _busy(self) -> int:
        n = sum(s.load() for e in self.resident.values() for s in e.sessions)
        return n + sum(g.load() for g in self.groups)

    def _gauge(self, key):
        e = self.resident.get(key)
        if e is not None:
            return e
        dims, links = self.gauge_src[key]
        need = gauge_bytes(dims, self.sloppy, self.recon)
        # evict idle gauges while over the resident count or the budget
        if not self._make_room(need, slots_for_gauge=True):
            return None
        g = Gauge(dims, links, sloppy=self.sloppy, recon=self.recon, stream=self.upload_stream)
        e = _GaugeEntry(key, g, need, [], time.perf_counter())
        self.resident[key] = e
        self.used += need
        self._sample_memory()
        return e

    def _evict(self, e):
        for s in e.sessions:
            s.close()
            self.used -= s.bytes
        e.gauge.close()
        self.used -= e.bytes
        del self.resident[e.key]

    def _place_group(self, req, e) -> bool:
        open_g = [s for s in self.groups if s.free_slots() > 0]
        if not open_g and len(self.groups) < self.max_groups:
            need = group_bytes(self.group_slots, self.group_max_vh, self.sloppy)
            if self.used + need <= self.budget or self._make_room(need, keep=e):
                prio = min(self._prio.values()) if self.priority_by_size else 0
                g = _GroupSession(self, self.device, prio)
                self.used += g.bytes
                self.groups.append(g)
                self._sample_memory()
                open_g = [g]
        if not open_g:
            return False
        with self.lock:
            e.in_groups += 1
        min(open_g, key=lambda s: s.load()).submit((req, e))
        return True

    def _place(self, req) -> bool:
        e = self._gauge(req.gauge_key)
        if e is None:
            return False
        e.last_used = time.perf_counter()
        if self.group_max_vh > 0 and e.gauge.vh <= self.group_max_vh:
            return self._place_group(req, e)
        open_s = [s for s in e.sessions if s.free_slots() > 0]
        if open_s:
            min(open_s, key=lambda s: s.load()).submit(req)
            return True
        if len(e.sessions) < self.max_sessions:
            need = session_bytes(e.gauge, self.slots, self.sloppy)
            if self.used + need <= self.budget or self._make_room(need, keep=e):
                prio = 0
                if self.priority_by_size:
                    prio = self._prio.get(int(np.prod(self.gauge_src[e.key][0])), 0)
                s = _Session(self, e, self.device, prio)
                self.used += s.bytes
                e.sessions.append(s)
                self._sample_memory()
                s.submit(req)
                return True
        return False

    # -- the stream -----------------------------------------------------------
    def run(self, requests, realtime: bool = True):
        """Serve `requests` (sorted by arrival).  realtime=False submits every
        request at once (saturation run).  Returns the results by rid."""
        torch.cuda.set_device(self.device)
        self.results = []
        pending = collections.deque()
        todo = collections.deque(sorted(requests, key=lambda r: r.arrival))
        self.t0 = time.perf_counter()
        n = len(todo)
        stall_since, last_finished = None, -1
        while True:
            now = time.perf_counter() - self.t0
            while todo and (not realtime or todo[0].arrival <= now):
                r = todo.popleft()
                if not realtime:
                    r.arrival = now
                pending.append(r)
            still = collections.deque()
            while pending:
                r = pending.popleft()
                if not self._place(r):
                    still.append(r)
            pending = still
            self._sample_memory()
            with self.lock:
                finished = len(self.results)
            if finished == n:
                break
            if pending and self._busy() == 0 and finished == last_finished:
                # nothing runs and nothing idle is left to evict: for a few
                # seconds no request could be placed (its field and session
                # alone exceed the budget)
                if stall_since is None:
                    stall_since = time.perf_counter()
                elif time.perf_counter() - stall_since > 5.0:
                    raise RuntimeError(f"request {pending[0].rid} cannot be admitted within the "
                                       f"HBM budget of {self.budget:.0f} bytes")
            else:
                stall_since = None
            last_finished = finished
            wait = 0.05
            if todo and realtime:
                wait = min(wait, max(0.0, todo[0].arrival - (time.perf_counter() - self.t0)))
            self.event.wait(wait)
            self.event.clear()
        return sorted(self.results, key=lambda r: r.rid)

    def close(self):
        for g in self.groups:
            g.close()
            self.used -= g.bytes
        self.groups = []
        for e in list(self.resident.values()):
            self._evict(e)


def summarize(results, makespan=None) -> dict:
    lat = np.array([r.latency for r in results])
    span = makespan if makespan is not None else max(r.done for r in results) - min(
        r.arrival for r in results)
    ok = sum(1 for r in results if r.status == STG_OK)
    return {"requests": len(results), "ok": ok, "solves_per_s": len(results) / span,
            "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "mean_ms": 1e3 * float(lat.mean()), "makespan_s": span}
