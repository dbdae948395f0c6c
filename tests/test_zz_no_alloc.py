"""stg_apply_A_dot_noalloc against stg_apply_A_dot, through the C ABI.

The no-allocation variant serves callers that may not allocate device
memory (latency-bound loops that cannot take cudaMalloc's device-wide
synchronisation, hosts whose device memory belongs to another allocator or a
fixed budget).  It launches the same kernels in the same order as the
allocating entry point, so its output field and its d^dag A d must be
bitwise those of stg_apply_A_dot, on repeated calls that reuse the shared
static scratch.  It must also leave the device's free memory unchanged on a
handle that has never allocated its workspace.  This file sorts last so that
a run stopping at its first failure has run every other test already.
"""
import pytest
import torch

import gen
import paper_1111_0125_gb300 as stg

pytestmark = pytest.mark.gpu

CASES = [
    ((6, 4, 10, 12), stg.STG_FP64, 18),
    ((24, 24, 24, 48), stg.STG_FP64, 12),   # FP64 at the scratch limit
    ((8, 8, 8, 16), stg.STG_FP32, 12),
    ((12, 12, 12, 24), stg.STG_FP16, 12),
    ((12, 12, 12, 24), stg.STG_BF16, 12),
    ((12, 12, 12, 24), stg.STG_FX16, 12),   # staged kernel, 21 tiles (ragged last)
    ((8, 8, 8, 16), stg.STG_FX16, 18),      # register-fed packed kernel
]


def _noalloc(g, f, mass, prec):
    out = g.new_field(prec)
    dot = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stg.stg_apply_A_dot_noalloc(g.handle, mass, f, out, dot, prec)
    return out, dot


@pytest.mark.parametrize("dims,prec,recon", CASES)
def test_noalloc_is_bitwise_the_allocating_entry_point(dims, prec, recon):
    U = gen.gauge_field(dims, "exp", seed=4, eps=0.5)
    b = torch.from_numpy(gen.source(dims, seed=6)).cuda()
    mass = 0.07
    # a first handle loads every kernel this path launches (lazy module
    # loading may take device memory on a kernel's first launch)
    with stg.Gauge(dims, U, sloppy=prec, recon=recon) as warm:
        fw = warm.pack(b, prec)
        _noalloc(warm, fw, mass, prec)
        warm.apply_A_dot(fw, mass, prec)
        torch.cuda.synchronize()
    with stg.Gauge(dims, U, sloppy=prec, recon=recon) as g:
        f = g.pack(b, prec)
        outs = [g.new_field(prec) for _ in range(2)]
        dots = [torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
                for _ in range(2)]
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for out, dot in zip(outs, dots):  # two calls in a row share the static scratch
            stg.stg_apply_A_dot_noalloc(g.handle, mass, f, out, dot, prec)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        # a fresh handle has no workspace yet: any allocation on the path
        # would show here
        assert free1 == free0, (free0, free1)
        # the reference creates the handle's workspace only now
        ref_out, ref_dot = g.apply_A_dot(f, mass, prec)
        torch.cuda.synchronize()
        for out, dot in zip(outs, dots):
            assert torch.equal(out, ref_out)
            assert dot.item() == ref_dot.item()


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
