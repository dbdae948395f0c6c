"""stg_apply_A_dot_noalloc against stg_apply_A_dot, through the C ABI.

The no-allocation variant serves callers that may not allocate device
memory (latency-bound loops that cannot take cudaMalloc's device-wide
synchronisation, hosts whose device memory belongs to another allocator or a
fixed budget).  It must give what the allocating entry point gives, on
repeated calls that reuse the shared static scratch.  This file sorts last so
that a run stopping at its first failure has run every other test already.
"""
import numpy as np
import pytest
import torch

import gen
import paper_1111_0125_gb300 as stg

pytestmark = pytest.mark.gpu

TOL = {stg.STG_FP64: 1e-12, stg.STG_FP32: 1e-6, stg.STG_FP16: 2e-3}


def _rel(a, b):
    # complex128 fields: the norm covers real and imaginary parts
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.mark.parametrize("dims,prec,recon", [
    ((6, 4, 10, 12), stg.STG_FP64, 18),
    ((8, 8, 8, 16), stg.STG_FP32, 12),
    ((12, 12, 12, 24), stg.STG_FP16, 12),
])
def test_noalloc_matches_allocating_entry_point(dims, prec, recon):
    U = gen.gauge_field(dims, "exp", seed=4, eps=0.5)
    b = torch.from_numpy(gen.source(dims, seed=6)).cuda()
    mass = 0.07
    with stg.Gauge(dims, U, sloppy=prec, recon=recon) as g:
        f = g.pack(b, prec)
        ref_out, ref_dot = g.apply_A_dot(f, mass, prec)
        ref = g.unpack(ref_out, prec)
        for _ in range(2):  # two calls in a row share the static scratch
            out = g.new_field(prec)
            dot = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            stg.stg_apply_A_dot_noalloc(g.handle, mass, f, out, dot, prec)
            torch.cuda.synchronize()
            assert _rel(g.unpack(out, prec), ref) <= TOL[prec]
            assert abs(dot.item() - ref_dot.item()) <= TOL[prec] * abs(ref_dot.item())


def test_noalloc_rejects_lattice_beyond_scratch():
    dims = (32, 32, 32, 48)  # FP64 intermediate alone needs 37.7 MB > 32 MiB
    with stg.Gauge(dims, gen.unit_gauge(dims), sloppy=stg.STG_FP64) as g:
        f = g.new_field(stg.STG_FP64)
        out = g.new_field(stg.STG_FP64)
        dot = torch.zeros(1, dtype=torch.float64, device="cuda")
        with pytest.raises(stg.StgError) as e:
            stg.stg_apply_A_dot_noalloc(g.handle, 0.1, f, out, dot, stg.STG_FP64)
        assert e.value.status == stg.STG_ERR_INVALID_ARG
        assert "scratch" in str(e.value)
