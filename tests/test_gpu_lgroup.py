"""Lattice-group CG session (stg_lgroup_*): systems on lattices of different
sizes iterate in lock-step, four launches per iteration for the whole group.
Each solution is checked with the oracle's A (true residual <= tol) and
against the same system solved alone (within kappa * tol, kappa = (m^2 +
64) / m^2 bounding the condition number)."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1111_0125_gb300 as stg
from paper_1111_0125_gb300 import Gauge

pytestmark = pytest.mark.gpu

# (dims, link kind, seed, mass, tol)
SYSTEMS = [((4, 4, 4, 4), "haar", 0, 0.1, 1e-10),
           ((8, 8, 8, 8), "exp", 1, 0.05, 1e-10),
           ((6, 4, 10, 12), "exp", 2, 0.2, 1e-8),
           ((12, 12, 12, 24), "exp", 3, 0.03, 1e-10),
           ((4, 4, 4, 8), "exp", 4, 0.02, 1e-10)]


def _vh(dims):
    return int(np.prod(dims)) // 2


def _check(dims, U, mass, tol, b, x, x_alone):
    r = b - oracle.apply_A(dims, U, mass, x)
    assert np.linalg.norm(r) <= tol * np.linalg.norm(b), (dims, mass)
    kappa = (mass ** 2 + 64) / mass ** 2
    assert np.linalg.norm(x - x_alone) <= kappa * tol * np.linalg.norm(x_alone), (dims, mass)


def _run(group, max_done=16, limit=200000):
    done, steps = [], 0
    while True:
        fin, nact = stg.stg_lgroup_step(group, max_done)
        done += fin
        steps += 1
        if nact == 0 or steps > limit:
            return done


@pytest.mark.parametrize("sloppy", [stg.STG_FP32, stg.STG_FX16])
def test_lattices_of_different_sizes_in_one_group(sloppy):
    gauges, Us, bs = [], [], []
    try:
        for dims, kind, seed, mass, tol in SYSTEMS:
            U = gen.gauge_field(dims, kind, seed=seed, eps=0.5)
            Us.append(U)
            bs.append(gen.source(dims, seed=100 + seed))
            gauges.append(Gauge(dims, U, sloppy=sloppy, recon=12))
        max_vh = max(_vh(s[0]) for s in SYSTEMS)
        grp = stg.stg_lgroup_create(len(SYSTEMS), max_vh, sloppy, 12,
                                    gauges[0].params(sloppy=sloppy, check_every=8))
        try:
            src = [torch.from_numpy(b).cuda() for b in bs]
            xs = [torch.zeros_like(v) for v in src]
            slots = [stg.stg_lgroup_add(grp, g.handle, s, x, spec[3], spec[4])
                     for g, s, x, spec in zip(gauges, src, xs, SYSTEMS)]
            assert sorted(slots) == list(range(len(SYSTEMS)))
            done = _run(grp)
        finally:
            stg.stg_lgroup_destroy(grp)
        assert sorted(d[0] for d in done) == sorted(slots)
        assert all(st == stg.STG_OK for _, st, _ in done)
        for k, (dims, kind, seed, mass, tol) in enumerate(SYSTEMS):
            x_alone, _ = gauges[k].cg_solve(src[k], mass, tol)
            _check(dims, Us[k], mass, tol, bs[k], xs[k].cpu().numpy(), x_alone.cpu().numpy())
            st = next(d[2] for d in done if d[0] == slots[k])
            assert st["iters"] > 0 and st["true_res"] <= tol
    finally:
        for g in gauges:
            g.close()


def test_system_joins_a_running_group():
    """A slot freed by a finished system takes a new system of another
    lattice while the slowest system keeps iterating."""
    specs = [((8, 8, 8, 8), 1, 0.02), ((4, 4, 4, 4), 2, 0.5), ((6, 4, 10, 12), 3, 0.2)]
    gauges, Us, bs = [], [], []
    try:
        for dims, seed, _ in specs:
            U = gen.gauge_field(dims, "exp", seed=seed, eps=0.5)
            Us.append(U)
            bs.append(gen.source(dims, seed=50 + seed))
            gauges.append(Gauge(dims, U, sloppy=stg.STG_FP32, recon=12))
        grp = stg.stg_lgroup_create(2, max(_vh(s[0]) for s in specs), stg.STG_FP32, 12,
                                    gauges[0].params(check_every=8))
        try:
            src = [torch.from_numpy(b).cuda() for b in bs]
            xs = [torch.zeros_like(v) for v in src]
            s0 = stg.stg_lgroup_add(grp, gauges[0].handle, src[0], xs[0], specs[0][2], 1e-10)
            s1 = stg.stg_lgroup_add(grp, gauges[1].handle, src[1], xs[1], specs[1][2], 1e-10)
            done, added, steps = [], False, 0
            while len(done) < 3 and steps < 100000:
                fin, _ = stg.stg_lgroup_step(grp)
                steps += 1
                done += fin
                if not added and any(f[0] == s1 for f in fin):
                    assert not any(f[0] == s0 for f in done)
                    assert stg.stg_lgroup_add(grp, gauges[2].handle, src[2], xs[2], specs[2][2],
                                              1e-10) == s1
                    added = True
        finally:
            stg.stg_lgroup_destroy(grp)
        assert added and len(done) == 3 and all(st == stg.STG_OK for _, st, _ in done)
        for k, (dims, _, mass) in enumerate(specs):
            x_alone, _ = gauges[k].cg_solve(src[k], mass, 1e-10)
            _check(dims, Us[k], mass, 1e-10, bs[k], xs[k].cpu().numpy(), x_alone.cpu().numpy())
    finally:
        for g in gauges:
            g.close()


def test_group_argument_checks():
    dims = (4, 4, 4, 4)
    U = gen.gauge_field(dims, "haar", seed=0)
    b = torch.from_numpy(gen.source(dims, seed=1)).cuda()
    x = torch.zeros_like(b)
    with pytest.raises(stg.StgError) as e:
        stg.stg_lgroup_create(17, 128, stg.STG_FP32, 12)
    assert e.value.status == stg.STG_ERR_INVALID_ARG
    grp = stg.stg_lgroup_create(2, 64, stg.STG_FP32, 12)   # 4^4 has Vh = 128 > 64
    try:
        with Gauge(dims, U, sloppy=stg.STG_FP32, recon=12) as g:
            with pytest.raises(stg.StgError) as e:
                stg.stg_lgroup_add(grp, g.handle, b, x, 0.1, 1e-10)
            assert e.value.status == stg.STG_ERR_INVALID_ARG
        with Gauge((4, 2, 2, 2), gen.gauge_field((4, 2, 2, 2), "haar", seed=0),
                   sloppy=stg.STG_FP32, recon=18) as g18:
            b2 = torch.from_numpy(gen.source((4, 2, 2, 2), seed=1)).cuda()
            with pytest.raises(stg.StgError) as e:
                stg.stg_lgroup_add(grp, g18.handle, b2, torch.zeros_like(b2), 0.1, 1e-10)
            assert e.value.status == stg.STG_ERR_UNSUPPORTED
        fin, nact = stg.stg_lgroup_step(grp)
        assert fin == [] and nact == 0
    finally:
        stg.stg_lgroup_destroy(grp)
