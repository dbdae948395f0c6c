"""Serving loop: requests of several lattices and gauge fields, more requests
than batch slots (so systems join running batches), checked against the same
requests solved alone and against the oracle's A; the HBM budget checked
against measured device usage."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1111_0125_gb300 as stg
from paper_1111_0125_gb300.serve import Request, ServeEngine, gauge_bytes, session_bytes

pytestmark = pytest.mark.gpu

LATTICES = {"a": ((4, 4, 4, 4), "haar", 0), "b": ((8, 8, 8, 8), "exp", 1),
            "c": ((6, 4, 10, 12), "exp", 2)}


def _tables():
    gauges, sources = {}, {}
    for key, (dims, kind, seed) in LATTICES.items():
        gauges[key] = (dims, gen.gauge_field(dims, kind, seed=seed, eps=0.5))
        for j in range(2):
            sources[(key, j)] = gen.source(dims, seed=100 + 10 * seed + j)
    return gauges, sources


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    keys = list(LATTICES)
    reqs = []
    for rid in range(n):
        key = keys[rid % len(keys)]
        reqs.append(Request(rid, 0.0, key, (key, int(rng.integers(2))),
                            float(np.exp(rng.uniform(np.log(0.05), np.log(0.3)))),
                            float(rng.choice([1e-8, 1e-10]))))
    return reqs


def _check(results, reqs, gauges, sources):
    assert len(results) == len(reqs)
    alone = {}
    for key, (dims, links) in gauges.items():
        alone[key] = stg.Gauge(dims, links, sloppy=stg.STG_FP32, recon=12)
    try:
        for res, req in zip(results, reqs):
            assert res.rid == req.rid and res.status == stg.STG_OK
            dims, links = gauges[req.gauge_key]
            b = sources[req.source_key]
            r = b - oracle.apply_A(dims, links, req.mass, res.x)
            assert np.linalg.norm(r) <= req.tol * np.linalg.norm(b), req
            g = alone[req.gauge_key]
            x1, _ = g.cg_solve(torch.from_numpy(b).cuda(), req.mass, req.tol)
            x1 = x1.cpu().numpy()
            kappa = (req.mass ** 2 + 64) / req.mass ** 2
            assert np.linalg.norm(res.x - x1) <= kappa * req.tol * np.linalg.norm(x1)
    finally:
        for g in alone.values():
            g.close()


def test_mixed_stream_matches_solving_alone():
    gauges, sources = _tables()
    reqs = _requests(24, seed=5)
    eng = ServeEngine(gauges, sources, slots=4, max_sessions_per_gauge=2, keep_solutions=True)
    try:
        results = eng.run(reqs, realtime=False)
    finally:
        eng.close()
    _check(results, reqs, gauges, sources)


def test_one_resident_field_evicts_and_waits():
    """Room for one gauge field at a time: requests of other lattices wait
    until the resident field's sessions drain, then it is evicted and theirs
    is uploaded; every request still gets the answer it gets alone."""
    gauges, sources = _tables()
    reqs = _requests(9, seed=6)
    eng = ServeEngine(gauges, sources, slots=2, max_sessions_per_gauge=1, max_resident=1,
                      keep_solutions=True)
    try:
        results = eng.run(reqs, realtime=False)
        assert len(eng.resident) <= 1
        assert eng.used <= eng.budget
    finally:
        eng.close()
    _check(results, reqs, gauges, sources)


def test_small_budget_holds_on_the_device():
    """An HBM budget with room for one gauge field and one session of the
    largest lattice: requests queue until memory frees, every one is served,
    and neither the engine's count nor the device usage measured during the
    run (its live torch buffers plus the library's bytes of every live handle
    and session) ever exceeds the budget."""
    gauges, sources = _tables()
    biggest = max(gauges, key=lambda k: int(np.prod(gauges[k][0])))
    dims, links = gauges[biggest]
    with stg.Gauge(dims, links, sloppy=stg.STG_FP32, recon=12) as g:
        need = gauge_bytes(dims, stg.STG_FP32, 12) + session_bytes(g, 2, stg.STG_FP32)
    budget = need + 4096
    reqs = _requests(12, seed=8)
    eng = ServeEngine(gauges, sources, hbm_budget=budget, slots=2, max_sessions_per_gauge=1,
                      keep_solutions=True)
    try:
        results = eng.run(reqs, realtime=False)
        assert 0 < eng.peak_used <= budget
        assert 0 < eng.peak_measured <= budget
        # what was measured is what was counted (allocator rounding aside)
        assert eng.peak_measured <= eng.peak_used + 64 * 1024
    finally:
        eng.close()
    _check(results, reqs, gauges, sources)


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("sloppy", [stg.STG_FP32, stg.STG_FX16])
def test_library_byte_counts_match_device_memory(sloppy):
    """The byte counts the budget relies on (stg_gauge_bytes, stg_batch_bytes)
    against the drop of the device's free memory when the handle and the
    session are created (each allocation rounded up to 2 MiB pages)."""
    dims = (16, 16, 16, 32)
    U = gen.gauge_field(dims, "exp", seed=1, eps=0.5)
    with stg.Gauge(dims, U, sloppy=sloppy, recon=12) as warm:   # loads the kernels once
        b = stg.stg_batch_create(warm.handle, 4, warm.params())
        stg.stg_batch_destroy(b)
    page = 2 << 20
    f0 = _free_bytes()
    with stg.Gauge(dims, U, sloppy=sloppy, recon=12) as g:
        f1 = _free_bytes()
        want = stg.stg_gauge_bytes(dims, sloppy, 12)
        assert want - page <= f0 - f1 <= want + 4 * page, (f0 - f1, want)
        b = stg.stg_batch_create(g.handle, 4, g.params())
        try:
            f2 = _free_bytes()
            want_b = stg.stg_batch_bytes(g.handle, 4, sloppy)
            assert want_b - page <= f1 - f2 <= want_b + 14 * page, (f1 - f2, want_b)
        finally:
            stg.stg_batch_destroy(b)


def test_batch_session_join_while_running():
    """A system added to a session that is already iterating converges to the
    same answer as alone (continuous batching at the C ABI)."""
    dims = (8, 8, 8, 8)
    U = gen.gauge_field(dims, "exp", seed=1, eps=0.5)
    bs = gen.source(dims, seed=3, nrhs=3)
    masses, tol = [0.02, 0.3, 0.2], 1e-10   # system 0 is the slowest
    with stg.Gauge(dims, U, sloppy=stg.STG_FP32, recon=12) as g:
        p = g.params(check_every=8)
        b = stg.stg_batch_create(g.handle, 2, p)
        try:
            src = [torch.from_numpy(v).cuda() for v in bs]
            xs = [torch.zeros_like(v) for v in src]
            s0 = stg.stg_batch_add(b, src[0], xs[0], masses[0], tol)
            stg.stg_batch_step(b)   # system 0 runs alone for a chunk
            s1 = stg.stg_batch_add(b, src[1], xs[1], masses[1], tol)
            assert s1 != s0
            done, added, steps = [], False, 0
            while len(done) < 3 and steps < 100000:
                fin, nact = stg.stg_batch_step(b)
                steps += 1
                done += fin
                if not added and any(f[0] == s1 for f in fin):
                    # the freed slot takes a third system while system 0 runs
                    assert not any(f[0] == s0 for f in done)
                    assert stg.stg_batch_add(b, src[2], xs[2], masses[2], tol) == s1
                    added = True
            assert added and len(done) == 3 and all(st == stg.STG_OK for _, st, _ in done)
        finally:
            stg.stg_batch_destroy(b)
        for k in range(3):
            r = bs[k] - oracle.apply_A(dims, U, masses[k], xs[k].cpu().numpy())
            assert np.linalg.norm(r) <= tol * np.linalg.norm(bs[k])


def test_small_lattices_served_through_lattice_groups():
    """Requests on the two small lattices go to lattice-group sessions
    (systems of different lattices and gauge fields in lock-step), the rest
    to per-field batch sessions; every result is the one the request gets
    alone, within the budget."""
    gauges, sources = _tables()
    reqs = _requests(24, seed=9)
    eng = ServeEngine(gauges, sources, slots=2, max_sessions_per_gauge=1, keep_solutions=True,
                      group_max_vh=int(np.prod((6, 4, 10, 12))) // 2, group_slots=4, max_groups=2)
    try:
        results = eng.run(reqs, realtime=False)
        assert len(eng.groups) >= 1
        assert eng.peak_measured <= eng.budget
    finally:
        eng.close()
    _check(results, reqs, gauges, sources)
