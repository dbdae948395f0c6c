"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (norm-wise relative error of the whole output field):
  FP64 Dslash / A : 1e-12  (the kernel and the oracle differ only in the
                            order of the 8 x 9 complex multiply-adds)
  FP32            : 1e-6   (24-bit significand, ~10^2 rounding steps)
  FP16 storage    : 2e-3   (11-bit significand on links and fields)
  FX16 storage    : 1e-4   (16-bit fixed point: |error| <= 2^-16 of the site's
                            largest component, links to 2^-16 absolute)
CG: the true residual |b - A x| / |b| computed with the *oracle's* A is <= tol,
and |x - x_oracle| / |x_oracle| <= kappa_hat * tol, kappa_hat = (m^2+64)/m^2.
"""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1111_0125_gb300 as stg
from paper_1111_0125_gb300 import Gauge

pytestmark = pytest.mark.gpu

# BF16 (8 significand bits, unit round-off 2^-8) misses FP16's 2e-3; its
# measured error is asserted separately below
TOL = {stg.STG_FP64: 1e-12, stg.STG_FP32: 1e-6, stg.STG_FP16: 2e-3, stg.STG_FX16: 1e-4,
       stg.STG_BF16: 1e-2}

# several tiles and ragged tails: Vh = 128, 8, 192, 1440, 2520, 20736
DIMS = [(4, 4, 4, 4), (2, 2, 2, 2), (4, 6, 2, 8), (6, 4, 10, 12), (10, 6, 6, 14),
        (12, 12, 12, 24)]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _links(dims, kind="haar", seed=0, eps=0.5):
    return gen.gauge_field(dims, kind, seed=seed, eps=eps)


def _to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    oracle.build()
    yield
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec", [stg.STG_FP64, stg.STG_FP32, stg.STG_FP16, stg.STG_FX16,
                                  stg.STG_BF16])
def test_pack_unpack_roundtrip(prec):
    dims = (6, 4, 10, 12)
    U = _links(dims)
    chi = gen.source(dims, seed=4)
    with Gauge(dims, U, sloppy=prec if prec != stg.STG_FP64 else stg.STG_FP64) as g:
        back = g.unpack(g.pack(_to_dev(chi), prec), prec).cpu().numpy()
    if prec == stg.STG_FP64:
        assert np.array_equal(back, chi)
    else:
        assert rel(back, chi) < {stg.STG_FP32: 1e-7, stg.STG_FP16: 1e-3, stg.STG_FX16: 5e-5,
                                 stg.STG_BF16: 5e-3}[prec]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec,recon", [(stg.STG_FP64, 18), (stg.STG_FP64, 12),
                                        (stg.STG_FP32, 18), (stg.STG_FP32, 12),
                                        (stg.STG_FP16, 18), (stg.STG_FP16, 12),
                                        (stg.STG_FX16, 18), (stg.STG_FX16, 12),
                                        (stg.STG_BF16, 18), (stg.STG_BF16, 12)])
def test_dslash_matches_oracle(dims, prec, recon):
    U = _links(dims, "haar", seed=sum(dims))
    with Gauge(dims, U, sloppy=prec, recon=recon) as g:
        for parity in (0, 1):
            chi = gen.source(dims, seed=parity + 7)
            out = g.unpack(g.dslash(g.pack(_to_dev(chi), prec), parity, prec), prec)
            want = oracle.dslash(dims, U, chi, out_parity=parity)
            assert rel(out.cpu().numpy(), want) < TOL[prec], (dims, prec, recon, parity)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 10, 12), (12, 12, 12, 24)])
@pytest.mark.parametrize("prec,recon", [(stg.STG_FP64, 18), (stg.STG_FP32, 18),
                                        (stg.STG_FP32, 12), (stg.STG_FP16, 12),
                                        (stg.STG_FX16, 12), (stg.STG_BF16, 12)])
def test_apply_A_and_dot_match_oracle(dims, prec, recon):
    U = _links(dims, "exp", seed=3, eps=0.4)
    mass = 0.05
    chi = gen.source(dims, seed=5)
    want = oracle.apply_A(dims, U, mass, chi)
    with Gauge(dims, U, sloppy=prec, recon=recon) as g:
        f = g.pack(_to_dev(chi), prec)
        out = g.unpack(g.apply_A(f, mass, prec), prec).cpu().numpy()
        assert rel(out, want) < TOL[prec]
        out2, dot = g.apply_A_dot(f, mass, prec)
        out2 = g.unpack(out2, prec).cpu().numpy()
        assert np.array_equal(out, out2)
        chi_r = g.unpack(f, prec).cpu().numpy()  # the rounded input the kernel saw
        want_dot = np.vdot(chi_r, out2).real
        assert abs(dot.item() - want_dot) <= TOL[prec] * abs(want_dot) * 10
        # fixed summation order: bitwise reproducible
        _, dot_b = g.apply_A_dot(f, mass, prec)
        assert dot_b.item() == dot.item()


def test_free_field_closed_form_on_gpu():
    """U = 1: A phi = (m^2 + 4 sum sin^2 p) phi on a plane wave (no oracle)."""
    import lattice_util as lu
    dims = (8, 4, 6, 8)
    mass = 0.3
    p = lu.momentum(dims, (1, 1, 2, 0))
    phi = lu.plane_wave(dims, p, [1.0, 0.5j, -0.25])
    with Gauge(dims, gen.unit_gauge(dims), sloppy=stg.STG_FP64) as g:
        out = g.unpack(g.apply_A(g.pack(_to_dev(phi), stg.STG_FP64), mass, stg.STG_FP64),
                       stg.STG_FP64).cpu().numpy()
    assert rel(out, lu.free_eigenvalue(p, mass) * phi) < 1e-13


def _check_solution(dims, U, mass, b, x, tol, x_ref=None):
    r = b - oracle.apply_A(dims, U, mass, x)
    tr = np.linalg.norm(r) / np.linalg.norm(b)
    assert tr <= tol, tr
    if x_ref is not None:
        kappa = (mass ** 2 + 64) / mass ** 2
        assert rel(x, x_ref) <= kappa * tol
    return tr


def test_cg_fp64_c1():
    """4^4, Haar links seed 0, source seed 1, m = 0.1, tol 1e-10, plain FP64 CG."""
    dims, mass, tol = (4, 4, 4, 4), 0.1, 1e-10
    U = gen.gauge_field(dims, "haar", seed=0)
    b = gen.source(dims, seed=1)
    x_ref, info = oracle.cg(dims, U, mass, b, tol=tol)
    with Gauge(dims, U, sloppy=stg.STG_FP64) as g:
        x, st = g.cg_solve(_to_dev(b), mass, tol, g.params(policy=stg.STG_CG_PLAIN))
    _check_solution(dims, U, mass, b, x.cpu().numpy(), tol, x_ref)
    assert st["true_res"] <= tol and st["sloppy_iters"] == 0
    # the same iteration as the oracle's Fig. 1 loop, up to rounding order
    assert abs(st["iters"] - info["iters"]) <= max(3, info["iters"] // 20)


@pytest.mark.parametrize("sloppy,recon", [(stg.STG_FP32, 18), (stg.STG_FP32, 12),
                                          (stg.STG_FP16, 12), (stg.STG_FP16, 18),
                                          (stg.STG_FX16, 12), (stg.STG_FX16, 18)])
@pytest.mark.parametrize("policy", [stg.STG_CG_RELIABLE, stg.STG_CG_REFINE])
def test_cg_mixed_matches_oracle(sloppy, recon, policy):
    dims, mass, tol = (8, 8, 8, 8), 0.05, 1e-10
    U = gen.gauge_field(dims, "exp", seed=11, eps=0.4)
    b = gen.source(dims, seed=12)
    x_ref, _ = oracle.cg(dims, U, mass, b, tol=1e-12)
    with Gauge(dims, U, sloppy=sloppy, recon=recon) as g:
        x, st = g.cg_solve(_to_dev(b), mass, tol, g.params(policy=policy))
    _check_solution(dims, U, mass, b, x.cpu().numpy(), tol, x_ref)
    assert st["sloppy_iters"] == st["iters"] > 0 and st["updates"] >= 1


def test_cg_initial_guess_and_zero_source():
    dims, mass = (4, 4, 4, 8), 0.2
    U = gen.gauge_field(dims, "haar", seed=2)
    b = gen.source(dims, seed=3)
    with Gauge(dims, U, sloppy=stg.STG_FP32) as g:
        x, st = g.cg_solve(_to_dev(b), mass, 1e-10)
        x2, st2 = g.cg_solve(_to_dev(b), mass, 1e-10, x0=x)
        assert st2["iters"] == 0 and torch.equal(x, x2)
        z, st3 = g.cg_solve(torch.zeros_like(x), mass, 1e-10, x0=x)
        assert st3["iters"] == 0 and not z.any()


def test_cg_errors():
    dims = (4, 4, 4, 4)
    U = gen.gauge_field(dims, "haar", seed=0)
    b = gen.source(dims, seed=1)
    with Gauge(dims, U, sloppy=stg.STG_FP32) as g:
        with pytest.raises(stg.StgError) as e:
            g.cg_solve(_to_dev(b), 0.01, 1e-10, g.params(maxiter=5))
        assert e.value.status == stg.STG_ERR_NOT_CONVERGED
        assert e.value.stats["iters"] >= 5 and e.value.stats["true_res"] > 1e-10
        bad = b.copy()
        bad[3, 1] = np.nan
        with pytest.raises(stg.StgError) as e:
            g.cg_solve(_to_dev(bad), 0.1, 1e-10)
        assert e.value.status == stg.STG_ERR_INVALID_ARG
        with pytest.raises(stg.StgError) as e:
            g.cg_solve(_to_dev(b), 0.1, 0.0)
        assert e.value.status == stg.STG_ERR_INVALID_ARG
        f = g.pack(_to_dev(b), stg.STG_FP16)
        with pytest.raises(stg.StgError) as e:   # handle holds FP64 + FP32 only
            g.dslash(f, 1, stg.STG_FP16)
        assert e.value.status == stg.STG_ERR_UNSUPPORTED
        with pytest.raises(stg.StgError) as e:
            stg.stg_dslash(g.handle, 2, f, f, stg.STG_FP32)
        assert e.value.status == stg.STG_ERR_INVALID_ARG


def test_gauge_create_rejects_bad_dims():
    with pytest.raises(stg.StgError) as e:
        stg.stg_gauge_create((4, 4, 3, 4), np.zeros((4, 3, 4, 4, 4, 3, 3), complex))
    assert e.value.status == stg.STG_ERR_DIMS


@pytest.mark.parametrize("grid", ["3", None])
def test_staged_fp16_matches_one_site_kernel(monkeypatch, grid):
    """IEEE FP16 / 12-real links also go through the staged two-site kernel
    (binary16 decode and encode in place of the fixed-point ones).  Against
    the one-site-per-thread FP16 kernel (gauge created with STG_FX16_TILED=0)
    it differs only by rounding order: both within FP16's tolerance of the
    oracle and within 2e-3 of each other; A, d^dag A d and a CG solve on the
    staged path agree with the oracle."""
    dims, mass = (12, 12, 12, 24), 0.05
    U = _links(dims, "exp", seed=4, eps=0.5)
    chi = gen.source(dims, seed=9)
    if grid is not None:
        monkeypatch.setenv("STG_FX16_GRID", grid)
    monkeypatch.setenv("STG_FX16_TILED", "0")
    plain = Gauge(dims, U, sloppy=stg.STG_FP16, recon=12)
    monkeypatch.delenv("STG_FX16_TILED")
    staged = Gauge(dims, U, sloppy=stg.STG_FP16, recon=12)
    try:
        P = stg.STG_FP16
        assert stg.stg_gauge_bytes(dims, P, 12) > stg.stg_gauge_bytes(dims, stg.STG_FP32, 18) // 4
        fp, fs = plain.pack(_to_dev(chi), P), staged.pack(_to_dev(chi), P)
        assert torch.equal(fp, fs)
        for parity in (0, 1):
            a = plain.unpack(plain.dslash(fp, parity, P), P).cpu().numpy()
            b = staged.unpack(staged.dslash(fs, parity, P), P).cpu().numpy()
            ref = oracle.dslash(dims, U, chi, parity)
            assert rel(b, ref) < TOL[P] and rel(a, ref) < TOL[P]
            assert rel(b, a) < 2e-3
        as_, ds = staged.apply_A_dot(fs, mass, P)
        out = staged.unpack(as_, P).cpu().numpy()
        ref = oracle.apply_A(dims, U, mass, chi)
        assert rel(out, ref) < TOL[P]
        ref_dot = float(np.vdot(chi, ref).real)
        assert abs(ds.item() - ref_dot) < 1e-2 * abs(ref_dot)
        b = gen.source(dims, seed=10)
        x, st = staged.cg_solve(_to_dev(b), mass, 1e-10)
        assert st["true_res"] <= 1e-10
        res = np.linalg.norm(b - oracle.apply_A(dims, U, mass, x.cpu().numpy())) / np.linalg.norm(b)
        assert res <= 1.01e-10
    finally:
        plain.close()
        staged.close()


@pytest.mark.parametrize("grid", ["1", "4", "7", None])
def test_staged_fx16_tiles_per_cta(monkeypatch, grid):
    """The staged FX16/12 Dslash (tile-major links streamed through shared
    memory) refills its four stages tile after tile.  A capped grid makes each
    CTA walk several of the 21 tiles of 12^3x24 (the last one ragged).  Its
    arithmetic is the register-fed kernel's, so the outputs are bitwise equal
    to that kernel's (gauge created with STG_FX16_TILED=0), and A agrees
    with the oracle."""
    dims, mass = (12, 12, 12, 24), 0.05
    U = _links(dims, "exp", seed=4, eps=0.5)
    chi = gen.source(dims, seed=9)
    if grid is not None:
        monkeypatch.setenv("STG_FX16_GRID", grid)
    monkeypatch.setenv("STG_FX16_TILED", "0")
    plain = Gauge(dims, U, sloppy=stg.STG_FX16, recon=12)
    monkeypatch.delenv("STG_FX16_TILED")
    staged = Gauge(dims, U, sloppy=stg.STG_FX16, recon=12)
    try:
        P = stg.STG_FX16
        fp, fs = plain.pack(_to_dev(chi), P), staged.pack(_to_dev(chi), P)
        assert torch.equal(fp, fs)
        for parity in (0, 1):
            assert torch.equal(plain.dslash(fp, parity, P), staged.dslash(fs, parity, P))
        ap, dp = plain.apply_A_dot(fp, mass, P)
        as_, ds = staged.apply_A_dot(fs, mass, P)
        assert torch.equal(ap, as_)
        assert abs(dp.item() - ds.item()) <= 1e-6 * abs(dp.item())
        out = staged.unpack(as_, P).cpu().numpy()
        assert rel(out, oracle.apply_A(dims, U, mass, chi)) < TOL[P]
        b = gen.source(dims, seed=10)
        x, st = staged.cg_solve(_to_dev(b), mass, 1e-10)
        _check_solution(dims, U, mass, b, x.cpu().numpy(), 1e-10)
    finally:
        plain.close()
        staged.close()


def test_bf16_error_is_reported_beside_fp16():
    """BF16 storage: the Dslash error against the oracle, measured on
    12^3x24 (printed), lies above FP16's (8 against 11 significand bits)
    and below 1e-2."""
    dims = (12, 12, 12, 24)
    U = _links(dims, "exp", seed=7, eps=0.5)
    chi = gen.source(dims, seed=8)
    want = oracle.dslash(dims, U, chi, out_parity=1)
    err = {}
    for prec in (stg.STG_FP16, stg.STG_BF16):
        with Gauge(dims, U, sloppy=prec, recon=12) as g:
            out = g.unpack(g.dslash(g.pack(_to_dev(chi), prec), 1, prec), prec)
            err[prec] = rel(out.cpu().numpy(), want)
    print(f"Dslash relative error: FP16 {err[stg.STG_FP16]:.2e}, BF16 {err[stg.STG_BF16]:.2e}")
    assert err[stg.STG_FP16] < 2e-3 and err[stg.STG_FP16] < err[stg.STG_BF16] < 1e-2


@pytest.mark.parametrize("mass", [1.0, 0.3, 0.05])
@pytest.mark.parametrize("policy", [stg.STG_CG_RELIABLE, stg.STG_CG_REFINE])
def test_cg_bf16_inner(mass, policy):
    """BF16 inner iterations (8-bit significand, Dslash error ~2e-3) reach a
    1e-10 true residual with reliable updates at delta = 0.1, with the Eq. 6
    start and with Fig. 2's restart, down to m = 0.05 on 8^4 (measured on
    GB300: 133 / 144 iterations with 10 updates at m = 0.05).  The solution
    is checked against the oracle's A."""
    dims, tol = (8, 8, 8, 8), 1e-10
    U = gen.gauge_field(dims, "exp", seed=11, eps=0.4)
    b = gen.source(dims, seed=12)
    with Gauge(dims, U, sloppy=stg.STG_BF16, recon=12) as g:
        bd = _to_dev(b)
        x = torch.zeros_like(bd)
        st = stg.stg_cg_solve(g.handle, bd, x, mass, tol,
                              g.params(policy=policy, delta=0.1, maxiter=20000))
    assert st["true_res"] <= tol
    _check_solution(dims, U, mass, b, x.cpu().numpy(), tol)
    assert 0 < st["updates"] and st["sloppy_iters"] >= 0.9 * st["iters"] > 0


def test_dependent_launch_changes_no_bit():
    """The solver's chunks run with programmatic dependent launch; with
    timing on, chunks rotate through graphs with per-kernel events and with
    serial launches.  All compute the same thing in the same order, so the
    solution is bitwise the same either way (no kernel reads its
    predecessor's output early)."""
    dims, mass, tol = (16, 16, 16, 32), 0.02, 1e-10
    U = _links(dims, "exp", seed=21, eps=0.5)
    b = gen.source(dims, seed=22)
    with Gauge(dims, U, sloppy=stg.STG_FX16, recon=12) as g:
        x0, s0 = g.cg_solve(_to_dev(b), mass, tol, g.params(timing=0))
        x1, s1 = g.cg_solve(_to_dev(b), mass, tol, g.params(timing=1))
    assert s0["iters"] == s1["iters"] and s0["updates"] == s1["updates"]
    assert torch.equal(x0, x1)
    assert s1["t_iter_ms"] > 0 and s1["t_iter_serial_ms"] > 0 and s1["timed_iters"] > 0


@pytest.mark.parametrize("prec,recon", [(stg.STG_FP64, 18), (stg.STG_FP32, 12),
                                        (stg.STG_FX16, 12), (stg.STG_FP16, 18)])
def test_dslash_group_of_lattices(prec, recon):
    """Four lattices of different sizes (2^4 .. 8^4) and parities in one
    launch: each output within the precision's tolerance of the oracle, and
    bitwise equal to its own stg_dslash where that runs the same one-site-
    per-thread arithmetic (FX16 / 12-real runs the packed staged kernel
    there, so the two agree to rounding)."""
    specs = [((4, 4, 4, 4), "haar", 0, 0), ((6, 4, 10, 12), "exp", 1, 1),
             ((8, 8, 8, 8), "exp", 2, 1), ((2, 2, 2, 2), "haar", 3, 0)]
    gauges, ins, outs, chis, Us = [], [], [], [], []
    try:
        for dims, kind, seed, parity in specs:
            U = _links(dims, kind, seed=seed)
            g = Gauge(dims, U, sloppy=prec, recon=recon)
            chi = gen.source(dims, seed=10 + seed)
            gauges.append(g)
            Us.append(U)
            chis.append(chi)
            ins.append(g.pack(_to_dev(chi), prec))
            outs.append(g.new_field(prec))
        stg.stg_dslash_group([g.handle for g in gauges], [sp[3] for sp in specs], ins, outs, prec)
        for k, (dims, _, _, parity) in enumerate(specs):
            single = gauges[k].dslash(ins[k], parity, prec)
            got = gauges[k].unpack(outs[k], prec).cpu().numpy()
            if prec == stg.STG_FX16 and recon == 12:
                one = gauges[k].unpack(single, prec).cpu().numpy()
                assert rel(got, one) < TOL[prec], k
            else:
                assert torch.equal(outs[k], single), k
            want = oracle.dslash(dims, Us[k], gauges[k].unpack(ins[k], prec).cpu().numpy(), parity)
            assert rel(got, want) < TOL[prec], k
        with pytest.raises(stg.StgError) as e:
            stg.stg_dslash_group([], [], [], [], prec)
        assert e.value.status == stg.STG_ERR_INVALID_ARG
    finally:
        for g in gauges:
            g.close()


def test_dslash_group_rejects_mixed_reconstruction():
    dims = (4, 4, 4, 4)
    U = _links(dims)
    with Gauge(dims, U, sloppy=stg.STG_FP32, recon=12) as a, \
            Gauge(dims, U, sloppy=stg.STG_FP32, recon=18) as b:
        f = a.pack(_to_dev(gen.source(dims, seed=1)), stg.STG_FP32)
        o1, o2 = a.new_field(stg.STG_FP32), b.new_field(stg.STG_FP32)
        with pytest.raises(stg.StgError) as e:
            stg.stg_dslash_group([a.handle, b.handle], [0, 0], [f, f], [o1, o2], stg.STG_FP32)
        assert e.value.status == stg.STG_ERR_INVALID_ARG


def test_fp32_mixed_cg_follows_the_emulated_method():
    """C1 with FP32 inner iterations on the GPU against the oracle's
    emulation of the same method (Fig. 2, Eq. 6, Sec. 3.2; single-precision
    inner vectors, double updates) at the same delta: both reach tol, their
    solutions agree within the condition bound, and their iteration counts
    within a factor 1.5 (rounding orders differ, the method does not)."""
    dims, mass, tol, delta = (4, 4, 4, 4), 0.1, 1e-10, 0.05
    U = gen.gauge_field(dims, "haar", seed=0)
    b = gen.source(dims, seed=1)
    xe, ie = oracle.cg_mixed(dims, U, mass, b, tol=tol, delta=delta)
    with Gauge(dims, U, sloppy=stg.STG_FP32, recon=18) as g:
        x, st = g.cg_solve(_to_dev(b), mass, tol, g.params(delta=delta))
    x = x.cpu().numpy()
    _check_solution(dims, U, mass, b, x, tol)
    kappa = (mass ** 2 + 64) / mass ** 2
    assert rel(x, xe) <= kappa * tol
    assert ie["iters"] / 1.5 <= st["iters"] <= 1.5 * ie["iters"], (st["iters"], ie["iters"])
