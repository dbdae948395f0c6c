"""Parity at the workloads' full sizes, in the launch configuration bench.py
times.

* 32^3 x 64, exp(i 0.6 H) links, m = 0.005: Dslash outputs at sampled sites
  (random plus every boundary class) against the oracle evaluated site by
  site, for FP16/12 (the bench's inner precision), FX16/12, FP32/12 and
  FP64/18; the bench's mixed CG solve (FP16 and FX16 inner) to 1e-10 checked
  with the oracle's A on the whole lattice (a property that holds at any
  size).
* 16^3 x 32, exp(i 0.4 H), m = 0.01: mixed FP32 CG and plain FP64 CG both
  reach a 1e-10 true residual (oracle's A) and agree within kappa * tol.
* 24^3 x 48, exp(i 0.5 H): sampled Dslash parity; the 16-system Dslash of
  the batched workload (sources seed 1 onward, FP32 and FX16 / 12-real) on
  the autotuner's kernel and on both (re, im) FP32x2 shapes, every system at
  sampled sites against the oracle.
"""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1111_0125_gb300 as stg

pytestmark = pytest.mark.gpu

TOL = {stg.STG_FP64: 1e-12, stg.STG_FP32: 1e-6, stg.STG_FP16: 2e-3, stg.STG_FX16: 1e-4}
_cache = {}


def _gauge(dims, eps):
    key = (dims, eps)
    if key not in _cache:
        _cache.clear()
        _cache[key] = gen.gauge_field(dims, "exp", seed=0, eps=eps)
    return _cache[key]


def _sample_sites(dims, parity, n, seed):
    """n random checkerboard indices plus sites on every face and corner."""
    lx, ly, lz, lt = dims
    vh = lx * ly * lz * lt // 2
    rng = np.random.default_rng(seed)
    picks = set(rng.choice(vh, size=n, replace=False).tolist())
    for t in (0, lt - 1):
        for z in (0, lz - 1):
            for y in (0, ly - 1):
                for x in (0, 1, lx - 2, lx - 1):
                    if (x + y + z + t) % 2 == parity:
                        picks.add((x + lx * (y + ly * (z + lz * t))) >> 1)
    return np.array(sorted(picks), dtype=np.int64)


def _rel_rows(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dims,eps", [((32, 32, 32, 64), 0.6), ((24, 24, 24, 48), 0.5)])
@pytest.mark.parametrize("prec,recon", [(stg.STG_FP16, 12), (stg.STG_FX16, 12), (stg.STG_FP32, 12),
                                        (stg.STG_FP64, 18)])
def test_dslash_sampled_sites(dims, eps, prec, recon):
    U = _gauge(dims, eps)
    chi = gen.source(dims, seed=1)
    with stg.Gauge(dims, U, sloppy=prec, recon=recon) as g:
        f = g.pack(torch.from_numpy(chi).cuda(), prec)
        chi_r = g.unpack(f, prec).cpu().numpy()  # the input as the kernel sees it
        for parity in (0, 1):
            out = g.unpack(g.dslash(f, parity, prec), prec).cpu().numpy()
            sites = _sample_sites(dims, parity, 4096, seed=parity + 3)
            want = oracle.dslash_sites(dims, U, chi_r, parity, sites)
            assert _rel_rows(out[sites], want) < TOL[prec], (prec, recon, parity)


@pytest.mark.parametrize("prec", [stg.STG_FP32, stg.STG_FX16])
@pytest.mark.parametrize("shape", [None, "14", "15"])
def test_mrhs_dslash_sampled_sites_24x48(monkeypatch, prec, shape):
    dims, n = (24, 24, 24, 48), 16
    if shape is not None:
        monkeypatch.setenv("STG_MRHS_SHAPE", shape)
    U = _gauge(dims, 0.5)
    chis = gen.source(dims, seed=1, nrhs=n)
    with stg.Gauge(dims, U, sloppy=prec, recon=12) as g:
        fb = stg.stg_field_bytes(g.handle, prec)
        buf = torch.empty(n * fb, dtype=torch.uint8, device="cuda")
        for k in range(n):
            stg.stg_pack_field(g.handle, prec, torch.from_numpy(chis[k]).cuda(), buf[k * fb:(k + 1) * fb])
        out = torch.empty_like(buf)
        stg.stg_dslash_mrhs(g.handle, 1, n, buf, out, prec)
        nb, tps = stg.stg_mrhs_tuning(g.handle, prec, n)
        if shape is not None:
            assert (nb, tps) == ({"14": 2, "15": 4}[shape], -2)
        sites = _sample_sites(dims, 1, 1024, seed=7)
        for k in range(n):
            chi_r = g.unpack(buf[k * fb:(k + 1) * fb], prec).cpu().numpy()
            got = g.unpack(out[k * fb:(k + 1) * fb], prec).cpu().numpy()
            want = oracle.dslash_sites(dims, U, chi_r, 1, sites)
            assert _rel_rows(got[sites], want) < TOL[prec], (prec, shape, k)


@pytest.mark.parametrize("prec", [stg.STG_FP16, stg.STG_FX16])
def test_bench_workload_mixed_cg_32x64(prec):
    """The bench's solve: FP16/12 inner iterations (and FX16/12 beside it)
    with the library's default updates, m = 0.005, tol = 1e-10, source
    seed 1."""
    dims, mass, tol = (32, 32, 32, 64), 0.005, 1e-10
    U = _gauge(dims, 0.6)
    b = gen.source(dims, seed=1)
    with stg.Gauge(dims, U, sloppy=prec, recon=12) as g:
        x, st = g.cg_solve(torch.from_numpy(b).cuda(), mass, tol, g.params(timing=1))
    x = x.cpu().numpy()
    r = b - oracle.apply_A(dims, U, mass, x)
    tr = np.linalg.norm(r) / np.linalg.norm(b)
    assert tr <= tol, tr
    assert abs(tr - st["true_res"]) <= 1e-3 * tol + 1e-3 * tr
    assert st["updates"] >= 2 and st["sloppy_iters"] == st["iters"]
    assert st["t_iter_ms"] > 0 and st["timed_iters"] > 0


def test_c2_mixed_vs_fp64_16x32():
    dims, mass, tol = (16, 16, 16, 32), 0.01, 1e-10
    U = gen.gauge_field(dims, "exp", seed=0, eps=0.4)
    b = gen.source(dims, seed=1)
    with stg.Gauge(dims, U, sloppy=stg.STG_FP32, recon=18) as g:
        bd = torch.from_numpy(b).cuda()
        xm, sm = g.cg_solve(bd, mass, tol, g.params(policy=stg.STG_CG_RELIABLE))
        xd, sd = g.cg_solve(bd, mass, tol, g.params(policy=stg.STG_CG_PLAIN))
    for x in (xm.cpu().numpy(), xd.cpu().numpy()):
        r = b - oracle.apply_A(dims, U, mass, x)
        assert np.linalg.norm(r) <= tol * np.linalg.norm(b)
    kappa = (mass ** 2 + 64) / mass ** 2
    diff = np.linalg.norm(xm.cpu().numpy() - xd.cpu().numpy()) / np.linalg.norm(xd.cpu().numpy())
    assert diff <= kappa * tol
    # every inner iteration ran in FP32; the FP64 work is the updates only.
    # (The share of low-precision iterations, 99.8% in Sec. 3.1, is measured
    # by bench.py, not pinned: it depends on the system's iteration count.)
    assert sm["sloppy_iters"] == sm["iters"] and sd["sloppy_iters"] == 0
    assert 0 < sm["updates"] < sm["iters"]


@pytest.mark.parametrize("prec", [stg.STG_FP16, stg.STG_FX16, stg.STG_FP32])
def test_dot_reduction_against_exact_sum_32x64(prec):
    """d^dag A d of stg_apply_A_dot at 32^3 x 64 (the reduction of the CG's
    alpha, and the same grid_sum_ff code as its |r|^2) against the exact sum.
    Per site the kernel forms Re d^dag q in FP32 from the values as stored;
    sites are summed in compensated FP32 pairs and the grid total in FP64.
    Products of two FP32 values are exact in FP64, so math.fsum over them is
    the exactly rounded sum.  The per-site FP32 rounding (relative 2^-24 per
    term, random in sign) leaves about 2^-24 / sqrt(n) of the sum of |terms|
    over n = 3 Vh terms; the bound asserted is 2^-30 of that sum."""
    import math
    dims, mass = (32, 32, 32, 64), 0.005
    U = _gauge(dims, 0.6)
    chi = gen.source(dims, seed=1)
    with stg.Gauge(dims, U, sloppy=prec, recon=12) as g:
        f = g.pack(torch.from_numpy(chi).cuda(), prec)
        out, dot = g.apply_A_dot(f, mass, prec)
        d = g.unpack(f, prec).cpu().numpy()
        q = g.unpack(out, prec).cpu().numpy()
        got = dot.item()
    prods = np.concatenate([(d.real * q.real).ravel(), (d.imag * q.imag).ravel()])
    exact = math.fsum(prods.tolist())
    scale = math.fsum(np.abs(prods).tolist())
    assert exact > 0
    assert abs(got - exact) <= 2.0 ** -30 * scale, (got, exact, (got - exact) / scale)
