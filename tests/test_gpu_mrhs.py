"""Multi-right-hand-side Dslash, A and batched CG against the oracle and
against the single-system path, through the C ABI."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1111_0125_gb300 as stg

pytestmark = pytest.mark.gpu

TOL = {stg.STG_FP32: 1e-6, stg.STG_FX16: 1e-4}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _pack_batch(g, fields, prec):
    """n canonical [Vh][3] arrays -> one buffer of n consecutive device fields."""
    fb = stg.stg_field_bytes(g.handle, prec)
    buf = torch.empty(len(fields) * fb, dtype=torch.uint8, device="cuda")
    for k, f in enumerate(fields):
        stg.stg_pack_field(g.handle, prec, torch.from_numpy(f).cuda(), buf[k * fb:(k + 1) * fb])
    return buf, fb


def _unpack_batch(g, buf, fb, n, prec):
    out = []
    for k in range(n):
        c = torch.empty((g.vh, 3), dtype=torch.complex128, device="cuda")
        stg.stg_unpack_field(g.handle, prec, buf[k * fb:(k + 1) * fb], c)
        out.append(c.cpu().numpy())
    return out


@pytest.mark.parametrize("dims", [(6, 4, 10, 12), (8, 8, 8, 8)])
@pytest.mark.parametrize("prec,recon", [(stg.STG_FP32, 12), (stg.STG_FP32, 18),
                                        (stg.STG_FX16, 12), (stg.STG_FX16, 18)])
@pytest.mark.parametrize("n", [1, 3, 9])
def test_dslash_mrhs_matches_oracle_and_single(dims, prec, recon, n):
    U = gen.gauge_field(dims, "haar", seed=5)
    chis = list(gen.source(dims, seed=2, nrhs=n))
    with stg.Gauge(dims, U, sloppy=prec, recon=recon) as g:
        buf, fb = _pack_batch(g, chis, prec)
        for parity in (0, 1):
            out = torch.empty_like(buf)
            stg.stg_dslash_mrhs(g.handle, parity, n, buf, out, prec)
            got = _unpack_batch(g, out, fb, n, prec)
            ins = _unpack_batch(g, buf, fb, n, prec)   # inputs as stored
            for k in range(n):
                want = oracle.dslash(dims, U, ins[k], parity)
                assert rel(got[k], want) < TOL[prec], (k, parity)
                single = g.unpack(g.dslash(buf[k * fb:(k + 1) * fb], parity, prec), prec)
                single = single.cpu().numpy()
                # same products; the compiler may contract them into FMAs
                # differently in the two kernels, so agreement is to rounding
                assert rel(got[k], single) < TOL[prec]
        nb, tps = stg.stg_mrhs_tuning(g.handle, prec, n)
        if tps == 0:  # staged kernel (12-real only)
            assert recon == 12 and nb in (2, 4, 8)
        elif tps == -1:  # staged, two sites per thread (FX16 / 12-real only)
            assert prec == stg.STG_FX16 and recon == 12 and nb in (2, 4)
        elif tps == -2:  # staged on (re, im) FP32x2 pairs (12-real only)
            assert recon == 12 and nb in (2, 4)
        else:
            assert nb in (1, 2, 4) and tps in (1, 2, 4, 8, 16) and tps <= max(1, n)


@pytest.mark.parametrize("prec", [stg.STG_FP32, stg.STG_FX16])
def test_apply_A_mrhs_per_system_masses(prec):
    dims, n = (6, 4, 10, 12), 5
    U = gen.gauge_field(dims, "exp", seed=3, eps=0.5)
    masses = gen.log_uniform(n, 0.005, 0.05, seed=9)
    chis = list(gen.source(dims, seed=4, nrhs=n))
    with stg.Gauge(dims, U, sloppy=prec, recon=12) as g:
        buf, fb = _pack_batch(g, chis, prec)
        out = torch.empty_like(buf)
        stg.stg_apply_A_mrhs(g.handle, n, masses, buf, out, prec)
        got = _unpack_batch(g, out, fb, n, prec)
        ins = _unpack_batch(g, buf, fb, n, prec)
    for k in range(n):
        assert rel(got[k], oracle.apply_A(dims, U, masses[k], ins[k])) < TOL[prec]


@pytest.mark.parametrize("prec,shape,nb", [(p, s, nb) for p in (stg.STG_FP32, stg.STG_FX16)
                                           for s, nb in (("9", 2), ("10", 4), ("11", 8),
                                                         ("14", 2), ("15", 4))])
@pytest.mark.parametrize("grid", [None, "2"])
def test_staged_mrhs_matches_register_fed(monkeypatch, prec, shape, nb, grid):
    """The staged multi-system kernel (links of a 64-site tile in shared
    memory, shared by every system) against the register-fed kernel and the
    oracle, for each register block NB; a grid of 2 CTAs makes each CTA walk
    12 of the 23 tiles (ragged last tile) through its 2-stage ring.  Shapes
    14 and 15 are its form on (re, im) FP32x2 pairs, with each tile's links
    rebuilt once into shared memory (row 2 for FP32, the decoded FP32 links
    for FX16)."""
    dims, n = (6, 4, 10, 12), 9
    U = gen.gauge_field(dims, "exp", seed=6, eps=0.5)
    chis = list(gen.source(dims, seed=8, nrhs=n))
    masses = gen.log_uniform(n, 0.005, 0.05, seed=10)
    with stg.Gauge(dims, U, sloppy=prec, recon=12) as g:
        buf, fb = _pack_batch(g, chis, prec)
        ins = _unpack_batch(g, buf, fb, n, prec)
        monkeypatch.setenv("STG_MRHS_SHAPE", "2")  # register-fed, NB = 4
        ref = torch.empty_like(buf)
        stg.stg_dslash_mrhs(g.handle, 1, n, buf, ref, prec)
        ref = _unpack_batch(g, ref, fb, n, prec)
        monkeypatch.setenv("STG_MRHS_SHAPE", shape)
        assert stg.stg_mrhs_tuning(g.handle, prec, n) == (nb, -2 if int(shape) >= 14 else 0)
        if grid is not None:
            monkeypatch.setenv("STG_MRHS_GRID", grid)
        for parity in (0, 1):
            out = torch.empty_like(buf)
            stg.stg_dslash_mrhs(g.handle, parity, n, buf, out, prec)
            got = _unpack_batch(g, out, fb, n, prec)
            for k in range(n):
                assert rel(got[k], oracle.dslash(dims, U, ins[k], parity)) < TOL[prec], (k, parity)
                if parity == 1:
                    assert rel(got[k], ref[k]) < TOL[prec], k
        out = torch.empty_like(buf)
        stg.stg_apply_A_mrhs(g.handle, n, masses, buf, out, prec)
        got = _unpack_batch(g, out, fb, n, prec)
        for k in range(n):
            assert rel(got[k], oracle.apply_A(dims, U, masses[k], ins[k])) < TOL[prec], k
        xs, st = _solve_batch(g, chis, masses, 1e-10, prec)
        for k in range(n):
            r = chis[k] - oracle.apply_A(dims, U, masses[k], xs[k])
            assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(chis[k]), k


@pytest.mark.parametrize("shape,nb", [("12", 2), ("13", 4)])
@pytest.mark.parametrize("grid", [None, "2"])
@pytest.mark.parametrize("n", [9, 16])
def test_paired_staged_mrhs(monkeypatch, shape, nb, grid, n):
    """The FX16 staged multi-system kernel with two sites per thread (site
    pairs in the halves of FP32x2 registers) against the register-fed
    kernel and the oracle: Dslash of both parities, A, and a batched CG; a
    grid of 2 CTAs walks 12 of the 23 tiles each (ragged last tile)."""
    prec = stg.STG_FX16
    dims = (6, 4, 10, 12)
    U = gen.gauge_field(dims, "exp", seed=6, eps=0.5)
    chis = list(gen.source(dims, seed=8, nrhs=n))
    masses = gen.log_uniform(n, 0.005, 0.05, seed=10)
    with stg.Gauge(dims, U, sloppy=prec, recon=12) as g:
        buf, fb = _pack_batch(g, chis, prec)
        ins = _unpack_batch(g, buf, fb, n, prec)
        monkeypatch.setenv("STG_MRHS_SHAPE", "2")  # register-fed, NB = 4
        ref = torch.empty_like(buf)
        stg.stg_dslash_mrhs(g.handle, 1, n, buf, ref, prec)
        ref = _unpack_batch(g, ref, fb, n, prec)
        monkeypatch.setenv("STG_MRHS_SHAPE", shape)
        assert stg.stg_mrhs_tuning(g.handle, prec, n) == (nb, -1)
        if grid is not None:
            monkeypatch.setenv("STG_MRHS_GRID", grid)
        for parity in (0, 1):
            out = torch.empty_like(buf)
            stg.stg_dslash_mrhs(g.handle, parity, n, buf, out, prec)
            got = _unpack_batch(g, out, fb, n, prec)
            for k in range(n):
                assert rel(got[k], oracle.dslash(dims, U, ins[k], parity)) < TOL[prec], (k, parity)
                if parity == 1:
                    assert rel(got[k], ref[k]) < TOL[prec], k
        out = torch.empty_like(buf)
        stg.stg_apply_A_mrhs(g.handle, n, masses, buf, out, prec)
        got = _unpack_batch(g, out, fb, n, prec)
        for k in range(n):
            assert rel(got[k], oracle.apply_A(dims, U, masses[k], ins[k])) < TOL[prec], k
        xs, st = _solve_batch(g, chis, masses, 1e-10, prec)
        for k in range(n):
            r = chis[k] - oracle.apply_A(dims, U, masses[k], xs[k])
            assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(chis[k]), k


def _solve_batch(g, bs, masses, tol, sloppy, policy=stg.STG_CG_RELIABLE):
    n = len(bs)
    src = torch.from_numpy(np.ascontiguousarray(np.stack(bs))).cuda()
    x = torch.zeros_like(src)
    p = g.params(policy=policy, sloppy=sloppy)
    st = stg.stg_cg_solve_mrhs(g.handle, n, src, x, masses, tol, p)
    return x.cpu().numpy(), st


@pytest.mark.parametrize("sloppy", [stg.STG_FP32, stg.STG_FX16])
@pytest.mark.parametrize("policy", [stg.STG_CG_RELIABLE, stg.STG_CG_REFINE])
def test_cg_mrhs_matches_oracle_and_single(sloppy, policy):
    dims, n, tol = (8, 8, 8, 8), 6, 1e-10
    U = gen.gauge_field(dims, "exp", seed=11, eps=0.4)
    masses = gen.log_uniform(n, 0.02, 0.2, seed=12)
    bs = list(gen.source(dims, seed=13, nrhs=n))
    with stg.Gauge(dims, U, sloppy=sloppy, recon=12) as g:
        xs, st = _solve_batch(g, bs, masses, tol, sloppy, policy)
        for k in range(n):
            r = bs[k] - oracle.apply_A(dims, U, masses[k], xs[k])
            assert np.linalg.norm(r) <= tol * np.linalg.norm(bs[k]), k
            assert st[k]["true_res"] <= tol and st[k]["updates"] >= 1
            x1, _ = g.cg_solve(torch.from_numpy(bs[k]).cuda(), masses[k], tol,
                               g.params(policy=policy, sloppy=sloppy))
            kappa = (masses[k] ** 2 + 64) / masses[k] ** 2
            assert rel(xs[k], x1.cpu().numpy()) <= kappa * tol
    # lighter systems need more iterations: each system stops on its own
    iters = [s["iters"] for s in st]
    assert iters[int(np.argmin(masses))] > iters[int(np.argmax(masses))]


def test_cg_mrhs_initial_guess_and_zero_source():
    dims, n = (4, 4, 4, 8), 3
    U = gen.gauge_field(dims, "haar", seed=2)
    masses = [0.1, 0.2, 0.3]
    bs = list(gen.source(dims, seed=3, nrhs=n))
    bs[1] = np.zeros_like(bs[1])
    with stg.Gauge(dims, U, sloppy=stg.STG_FP32) as g:
        xs, st = _solve_batch(g, bs, masses, 1e-10, stg.STG_FP32)
        assert not xs[1].any() and st[1]["iters"] == 0
        src = torch.from_numpy(np.stack(bs)).cuda()
        x = torch.from_numpy(xs).cuda()
        st2 = stg.stg_cg_solve_mrhs(g.handle, n, src, x, masses, 1e-10)
        assert all(s["iters"] == 0 for s in st2)


def test_mrhs_errors():
    dims = (4, 4, 4, 4)
    U = gen.gauge_field(dims, "haar", seed=0)
    with stg.Gauge(dims, U, sloppy=stg.STG_FP32) as g:
        f = g.new_field(stg.STG_FP32)
        o = g.new_field(stg.STG_FP32)
        with pytest.raises(stg.StgError) as e:
            stg.stg_dslash_mrhs(g.handle, 0, 0, f, o, stg.STG_FP32)
        assert e.value.status == stg.STG_ERR_INVALID_ARG
        with pytest.raises(stg.StgError) as e:
            stg.stg_dslash_mrhs(g.handle, 0, 1, f, o, stg.STG_FP64)
        assert e.value.status == stg.STG_ERR_UNSUPPORTED
        b = torch.from_numpy(gen.source(dims, seed=1)).cuda()
        with pytest.raises(stg.StgError) as e:
            stg.stg_cg_solve_mrhs(g.handle, 1, b, torch.zeros_like(b), [0.1], 1e-10,
                                  g.params(maxiter=3))
        assert e.value.status == stg.STG_ERR_NOT_CONVERGED
        assert e.value.stats[0]["iters"] >= 3


def test_c4_batched_24x48_sixteen_masses():
    """24^3 x 48, exp(i 0.5 H) links, 16 sources (seed 1 onward), masses
    log-uniform in [0.005, 0.05] (seed 17), FP32 inner / FP64 updates,
    tol 1e-10: every system's true residual checked with the oracle's A."""
    dims, n, tol = (24, 24, 24, 48), 16, 1e-10
    U = gen.gauge_field(dims, "exp", seed=0, eps=0.5)
    masses = gen.log_uniform(n, 0.005, 0.05, seed=17)
    bs = list(gen.source(dims, seed=1, nrhs=n))
    with stg.Gauge(dims, U, sloppy=stg.STG_FP32, recon=12) as g:
        xs, st = _solve_batch(g, bs, masses, tol, stg.STG_FP32)
    for k in range(n):
        r = bs[k] - oracle.apply_A(dims, U, masses[k], xs[k])
        assert np.linalg.norm(r) <= tol * np.linalg.norm(bs[k]), k


@pytest.mark.parametrize("shape", [None, "9", "11", "15"])
def test_mrhs_at_the_system_limit(monkeypatch, shape):
    """64 systems, the most one call takes: every system's Dslash and A
    against the oracle (tuned shape, the staged kernel with NB = 2 and 8,
    whose per-warp reduction slots run up to system 63, and its (re, im)
    FP32x2 form with NB = 4), then a batched CG of all 64."""
    if shape is not None:
        monkeypatch.setenv("STG_MRHS_SHAPE", shape)
    dims, n, prec = (4, 4, 4, 8), 64, stg.STG_FP32
    U = gen.gauge_field(dims, "exp", seed=31, eps=0.5)
    chis = list(gen.source(dims, seed=32, nrhs=n))
    masses = gen.log_uniform(n, 0.05, 0.5, seed=33)
    with stg.Gauge(dims, U, sloppy=prec, recon=12) as g:
        buf, fb = _pack_batch(g, chis, prec)
        ins = _unpack_batch(g, buf, fb, n, prec)
        out = torch.empty_like(buf)
        stg.stg_dslash_mrhs(g.handle, 0, n, buf, out, prec)
        got = _unpack_batch(g, out, fb, n, prec)
        for k in range(n):
            assert rel(got[k], oracle.dslash(dims, U, ins[k], 0)) < TOL[prec], k
        stg.stg_apply_A_mrhs(g.handle, n, masses, buf, out, prec)
        got = _unpack_batch(g, out, fb, n, prec)
        for k in range(n):
            assert rel(got[k], oracle.apply_A(dims, U, masses[k], ins[k])) < TOL[prec], k
        xs, st = _solve_batch(g, chis, masses, 1e-10, prec)
    for k in range(n):
        r = chis[k] - oracle.apply_A(dims, U, masses[k], xs[k])
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(chis[k]), k
        assert st[k]["true_res"] <= 1e-10
