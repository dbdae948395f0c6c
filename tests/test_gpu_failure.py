"""Failure detection on the GPU without a fault.

The staged FX16 Dslash waits on shared-memory stage barriers for its bulk
copies; every such wait gives up after about a second.  Here the kernel is
told to withhold one fill (STG_FX16_TEST_DROP_FILL=1), so that wait runs
out: the kernel records the timeout, lets its other copies land and returns;
the CG stops on the device flag and the solver returns STG_ERR_TIMEOUT.  The
context stays usable: a second handle solves the same system afterwards.
"""
import time

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1111_0125_gb300 as stg
from paper_1111_0125_gb300 import Gauge

pytestmark = pytest.mark.gpu


def test_stage_wait_timeout_is_reported_and_the_context_recovers(monkeypatch):
    dims, mass, tol = (12, 12, 12, 24), 0.05, 1e-10   # 21 tiles of 1024 sites
    U = gen.gauge_field(dims, "exp", seed=4, eps=0.5)
    b = gen.source(dims, seed=5)
    monkeypatch.setenv("STG_FX16_GRID", "4")          # every CTA walks >= 5 tiles
    monkeypatch.setenv("STG_FX16_TEST_DROP_FILL", "1")
    with Gauge(dims, U, sloppy=stg.STG_FX16, recon=12) as g:
        t0 = time.time()
        with pytest.raises(stg.StgError) as err:
            g.cg_solve(torch.from_numpy(b).cuda(), mass, tol)
        assert err.value.status == stg.STG_ERR_TIMEOUT
        assert time.time() - t0 < 60
    torch.cuda.synchronize()
    monkeypatch.delenv("STG_FX16_TEST_DROP_FILL")
    with Gauge(dims, U, sloppy=stg.STG_FX16, recon=12) as g:
        x, st = g.cg_solve(torch.from_numpy(b).cuda(), mass, tol)
    r = b - oracle.apply_A(dims, U, mass, x.cpu().numpy())
    assert np.linalg.norm(r) <= tol * np.linalg.norm(b)
