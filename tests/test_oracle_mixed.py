"""The oracle's emulated mixed-precision CG (Fig. 2, Eq. 6, Sec. 3.2:
single-precision inner vectors, double updates) reaches the same solution as
its FP64 CG, and behaves as the method says: most iterations in the low
precision, updates that fire as the residual falls by delta."""
import numpy as np
import pytest

import gen
import oracle
from lattice_util import free_eigenvalue, momentum, plane_wave, rel


def test_c1_same_solution_as_fp64_cg():
    dims, mass, tol = (4, 4, 4, 4), 0.1, 1e-10
    U = gen.gauge_field(dims, "haar", seed=0)
    b = gen.source(dims, seed=1)
    x64, i64 = oracle.cg(dims, U, mass, b, tol=tol)
    x, info = oracle.cg_mixed(dims, U, mass, b, tol=tol, delta=0.1)
    assert info["status"] == 0 and info["true_res"] <= tol
    kappa = (mass ** 2 + 64) / mass ** 2
    assert rel(x, x64) <= kappa * tol
    # single-precision inner iterations cost some extra iterations only
    assert info["updates"] >= 1 and info["iters"] <= 1.5 * i64["iters"]
    assert info["low_precision_fraction"] >= 0.95


def test_plane_wave_solved_to_closed_form():
    """U = 1, b a plane wave: A b = lambda b, x = b / lambda (single precision
    inner steps plus updates reach it to tol)."""
    dims, mass = (4, 6, 2, 8), 0.3
    p = momentum(dims, (1, 2, 1, 0))
    b = plane_wave(dims, p, [0.3 - 0.1j, 1.0, 0.2j])
    x, info = oracle.cg_mixed(dims, gen.unit_gauge(dims), mass, b, tol=1e-10, delta=0.1)
    assert info["status"] == 0
    assert rel(x, b / free_eigenvalue(p, mass)) < 1e-9


def test_smaller_delta_fewer_updates():
    """The trigger |r^| < delta max|r^|: a smaller delta fires less often."""
    dims, mass = (4, 4, 4, 8), 0.05
    U = gen.gauge_field(dims, "exp", seed=5, eps=0.5)
    b = gen.source(dims, seed=6)
    ups = []
    for delta in (0.01, 0.1, 0.5):
        _, info = oracle.cg_mixed(dims, U, mass, b, tol=1e-10, delta=delta)
        assert info["status"] == 0 and info["true_res"] <= 1e-10
        ups.append(info["updates"])
    assert ups[0] <= ups[1] <= ups[2] and ups[0] < ups[2]


@pytest.mark.parametrize("delta", [0.0, 1.0, -0.5])
def test_bad_delta_rejected(delta):
    dims = (2, 2, 2, 2)
    with pytest.raises(ValueError):
        oracle.cg_mixed(dims, gen.unit_gauge(dims), 0.1, gen.source(dims, seed=1), delta=delta)


def test_refinement_variant_converges_and_restarts_cost_iterations():
    """Fig. 2's plain refinement (d restarted at each update) reaches the same
    solution; keeping d through the update (Eq. 6) needs no more iterations."""
    dims, mass, tol = (4, 4, 4, 8), 0.05, 1e-10
    U = gen.gauge_field(dims, "exp", seed=5, eps=0.5)
    b = gen.source(dims, seed=6)
    xr, ir = oracle.cg_mixed(dims, U, mass, b, tol=tol, delta=0.1, refine=True)
    xe, ie = oracle.cg_mixed(dims, U, mass, b, tol=tol, delta=0.1)
    assert ir["status"] == 0 and ir["true_res"] <= tol and ir["updates"] >= 1
    kappa = (mass ** 2 + 64) / mass ** 2
    assert rel(xr, xe) <= 2 * kappa * tol
    assert ie["iters"] <= ir["iters"]


def _eq6_direction_error(o):
    """Relative distance between the emulation's new search direction at its
    first reliable update and Eq. 6's d = r^ + (|r|^2 / delta_old) d, formed
    here from the new true residual r = b - A x (x as the oracle left it,
    A re-applied) and the oracle's d before the update; also the iterated-
    vs-true gap that makes a plain-CG beta distinguishable."""
    dims, mass = (4, 4, 4, 8), 0.02
    U = gen.gauge_field(dims, "exp", seed=5, eps=0.5)
    b = gen.source(dims, seed=1)
    _, info = o.cg_mixed(dims, U, mass, b, tol=1e-10, delta=1e-3, snapshot=True)
    fu = info["first_update"]
    r = b - o.apply_A(dims, U, mass, fu["x"])
    r_hat = r.astype(np.complex64)                       # group-wise update: r^ = r
    true2 = float(np.vdot(r, r).real)
    want = (r_hat.astype(np.complex128) + (true2 / fu["rho_prev"]) * fu["d_old"])
    want = want.astype(np.complex64)
    err = float(np.linalg.norm(fu["d_new"] - want) / np.linalg.norm(want))
    gap = abs(fu["rho_iter"] - true2) / true2
    same_r = bool(np.array_equal(fu["r_hat"].astype(np.complex64), r_hat))
    return err, gap, same_r


def test_eq6_search_direction_at_the_update():
    """Eq. 6 (reading: r is the new true residual, beta = |r|^2 / delta_old,
    d kept): the oracle's first corrected direction is that formula applied
    to its own outputs.  The iterated |r^|^2 differs from the true |r|^2 by
    about 1e-3 here, so a plain CG beta (|r^|^2 / delta_old) would miss by
    that much."""
    err, gap, same_r = _eq6_direction_error(oracle)
    assert same_r
    assert gap > 1e-4
    assert err < 1e-6 * gap
