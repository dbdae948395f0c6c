"""t-slab decomposition (Sec. 3.3, Table 1) on one device, through the C ABI.

- The Dslash on P slabs equals the oracle's Eq. 5 for every precision and
  reconstruction, P from 1 (self-exchange) to one slab of two time slices
  per rank, both parities; the two edge slices of every slab (where the
  ghost fields and ghost links are read) are also checked on their own.
- FP64, FP32, BF16 and FP16 / 18-real are bitwise equal to stg_dslash on
  the whole lattice: the same arithmetic in the same order, only the source
  of the neighbour data differs (FX16 and FP16 with 12-real links run the
  staged two-site kernel there).
- COPY, DIRECT and the overlapped schedule give bitwise the same output and
  the same d^dag A d.
- apply_A_dot against the oracle's A and its inner product.
- The CG on the slabs (FP64; FP32 and FX16 inner iterations with reliable
  updates): true residual with the oracle's A <= tol, and the solution
  within kappa_hat tol of the oracle's.
"""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1111_0125_gb300 as stg
from paper_1111_0125_gb300 import Gauge

pytestmark = pytest.mark.gpu

TOL = {stg.STG_FP64: 1e-12, stg.STG_FP32: 1e-6, stg.STG_FP16: 2e-3, stg.STG_FX16: 1e-4,
       stg.STG_BF16: 1e-2}
MODES = [(stg.STG_SLAB_COPY, 0), (stg.STG_SLAB_DIRECT, 0), (stg.STG_SLAB_COPY, 1),
         (stg.STG_SLAB_DIRECT, 1)]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    oracle.build()
    yield
    torch.cuda.synchronize()


class Slabs:
    def __init__(self, dims, U, nslabs, prec=stg.STG_FP64, recon=18, mode=stg.STG_SLAB_COPY,
                 overlap=0):
        self.h = stg.stg_slabs_create(dims, U, nslabs, prec, recon)
        stg.stg_slabs_set_exchange(self.h, mode, overlap)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        stg.stg_slabs_destroy(self.h)

    def dslash(self, chi, parity):
        inp = _to_dev(chi)
        out = torch.zeros_like(inp)
        stg.stg_slabs_load(self.h, 0, inp)
        stg.stg_slabs_dslash(self.h, parity, 0, 1)
        stg.stg_slabs_store(self.h, 1, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    def apply_A_dot(self, chi, mass):
        inp = _to_dev(chi)
        out = torch.zeros_like(inp)
        dot = torch.zeros(1, dtype=torch.float64, device="cuda")
        stg.stg_slabs_load(self.h, 0, inp)
        stg.stg_slabs_apply_A_dot(self.h, mass, 0, 1, dot)
        stg.stg_slabs_store(self.h, 1, out)
        torch.cuda.synchronize()
        return out.cpu().numpy(), float(dot.item())


def _edge_rows(dims, nslabs):
    """Checkerboard indices of every slab's first and last time slice."""
    lx, ly, lz, lt = dims
    st, lts = lx * ly * lz // 2, lt // nslabs
    rows = []
    for r in range(nslabs):
        for t in (r * lts, r * lts + lts - 1):
            rows.append(np.arange(t * st, (t + 1) * st))
    return np.concatenate(rows)


# (dims, slab counts): Lt / P even; P = Lt / 2 gives slabs of two slices
CASES = [((4, 4, 4, 8), [1, 2, 4]), ((6, 4, 10, 12), [3, 6]), ((4, 6, 2, 16), [8])]
PRECS = [(stg.STG_FP64, 18), (stg.STG_FP64, 12), (stg.STG_FP32, 18), (stg.STG_FP32, 12),
         (stg.STG_FP16, 18), (stg.STG_FP16, 12), (stg.STG_FX16, 18), (stg.STG_FX16, 12),
         (stg.STG_BF16, 18), (stg.STG_BF16, 12)]


@pytest.mark.parametrize("dims,counts", CASES)
@pytest.mark.parametrize("prec,recon", PRECS)
def test_slab_dslash_matches_oracle(dims, counts, prec, recon):
    U = gen.gauge_field(dims, "haar", seed=sum(dims) + 3)
    edges = {P: _edge_rows(dims, P) for P in counts}
    for parity in (0, 1):
        chi = gen.source(dims, seed=11 + parity)
        ref = oracle.dslash(dims, U, chi, parity)
        whole = None
        if prec != stg.STG_FX16 and not (prec == stg.STG_FP16 and recon == 12):
            with Gauge(dims, U, sloppy=prec, recon=recon) as g:
                whole = g.unpack(g.dslash(g.pack(_to_dev(chi), prec), parity, prec), prec)
                whole = whole.cpu().numpy()
        for P in counts:
            with Slabs(dims, U, P, prec, recon) as s:
                out = s.dslash(chi, parity)
            assert rel(out, ref) < TOL[prec], (P, parity)
            e = edges[P]
            assert rel(out[e], ref[e]) < TOL[prec], (P, parity, "edge slices")
            if whole is not None:
                assert np.array_equal(out, whole), (P, parity, "bitwise vs stg_dslash")


@pytest.mark.parametrize("prec,recon", [(stg.STG_FP64, 18), (stg.STG_FP32, 12), (stg.STG_FX16, 12)])
def test_slab_exchange_modes_agree_bitwise(prec, recon):
    dims, P, mass = (6, 4, 10, 12), 3, 0.2
    U = gen.gauge_field(dims, "exp", seed=5, eps=0.5)
    chi = gen.source(dims, seed=9)
    outs = []
    for mode, overlap in MODES:
        with Slabs(dims, U, P, prec, recon, mode, overlap) as s:
            d = s.dslash(chi, 1)
            q, dot = s.apply_A_dot(chi, mass)
        outs.append((d, q, dot))
    for d, q, dot in outs[1:]:
        assert np.array_equal(d, outs[0][0])
        assert np.array_equal(q, outs[0][1])
        assert dot == outs[0][2]


@pytest.mark.parametrize("prec,recon", [(stg.STG_FP64, 18), (stg.STG_FP64, 12), (stg.STG_FP32, 12),
                                        (stg.STG_FX16, 12)])
@pytest.mark.parametrize("P", [1, 2, 4])
def test_slab_apply_A_dot_matches_oracle(prec, recon, P):
    dims, mass = (4, 6, 2, 16), 0.15
    U = gen.gauge_field(dims, "exp", seed=2, eps=0.6)
    chi = gen.source(dims, seed=21)
    ref = oracle.apply_A(dims, U, mass, chi)
    ref_dot = float(np.vdot(chi, ref).real)
    with Slabs(dims, U, P, prec, recon, stg.STG_SLAB_DIRECT, 1) as s:
        q, dot = s.apply_A_dot(chi, mass)
    tol = TOL[prec] * 10
    assert rel(q, ref) < tol
    assert abs(dot - ref_dot) / abs(ref_dot) < tol


@pytest.mark.parametrize("dims,P,mode", [((4, 4, 4, 8), 2, stg.STG_SLAB_COPY),
                                         ((6, 4, 10, 12), 3, stg.STG_SLAB_DIRECT),
                                         ((8, 8, 8, 16), 8, stg.STG_SLAB_COPY)])
def test_slab_cg_matches_oracle(dims, P, mode):
    mass, tol = 0.1, 1e-10
    U = gen.gauge_field(dims, "exp", seed=1, eps=0.4)
    b = gen.source(dims, seed=3)
    x_ref, info = oracle.cg(dims, U, mass, b, tol=tol)
    with Slabs(dims, U, P, stg.STG_FP64, 18, mode, 1) as s:
        bd = _to_dev(b)
        xd = torch.zeros_like(bd)
        stats = stg.stg_slabs_cg_solve(s.h, bd, xd, mass, tol)
        x = xd.cpu().numpy()
    res = np.linalg.norm(b - oracle.apply_A(dims, U, mass, x)) / np.linalg.norm(b)
    assert res <= tol * 1.01, stats
    kappa = (mass ** 2 + 64.0) / mass ** 2
    assert rel(x, x_ref) <= kappa * tol
    assert abs(stats["iters"] - info["iters"]) <= max(3, info["iters"] // 20), (stats, info)
    assert stats["true_res"] <= tol


@pytest.mark.parametrize("prec,recon,P", [(stg.STG_FP32, 12, 2), (stg.STG_FX16, 12, 3),
                                          (stg.STG_FP32, 18, 1)])
def test_slab_mixed_cg_matches_oracle(prec, recon, P):
    """Inner iterations in FP32 / FX16 on the slabs, reliable updates with the
    FP64 links (Sec. 3.2), to the FP64 true residual."""
    dims, mass, tol = (6, 4, 10, 12), 0.05, 1e-10
    U = gen.gauge_field(dims, "exp", seed=4, eps=0.5)
    b = gen.source(dims, seed=8)
    x_ref, info = oracle.cg(dims, U, mass, b, tol=tol)
    with Slabs(dims, U, P, prec, recon, stg.STG_SLAB_DIRECT, 0) as s:
        bd = _to_dev(b)
        xd = torch.zeros_like(bd)
        stats = stg.stg_slabs_cg_solve(s.h, bd, xd, mass, tol)
        x = xd.cpu().numpy()
    res = np.linalg.norm(b - oracle.apply_A(dims, U, mass, x)) / np.linalg.norm(b)
    assert res <= tol * 1.01, stats
    kappa = (mass ** 2 + 64.0) / mass ** 2
    assert rel(x, x_ref) <= kappa * tol
    assert stats["updates"] >= 2 and stats["sloppy_iters"] == stats["iters"]
    assert stats["iters"] < 3 * info["iters"], (stats, info)


def test_slab_cg_unsupported_precision_and_profile():
    dims = (4, 4, 4, 8)
    U = gen.gauge_field(dims, "haar", seed=0)
    b = _to_dev(gen.source(dims, seed=1))
    x = torch.zeros_like(b)
    with Slabs(dims, U, 2, stg.STG_FP16, 12) as s:
        with pytest.raises(stg.StgError) as e:
            stg.stg_slabs_cg_solve(s.h, b, x, 0.1, 1e-8)
        assert e.value.status == stg.STG_ERR_UNSUPPORTED
        for mode in (stg.STG_SLAB_COPY, stg.STG_SLAB_DIRECT):
            stg.stg_slabs_set_exchange(s.h, mode, 0)
            t = stg.stg_slabs_profile(s.h, 3)
            assert all(v >= 0.0 for v in t.values())
            assert t["compute_ms"] > 0.0 and t["total_ms"] > 0.0
            if mode == stg.STG_SLAB_DIRECT:
                assert t["exchange_ms"] == 0.0
