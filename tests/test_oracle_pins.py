"""Pins for the FP64 CPU oracle against what the paper and the mathematics fix.

Each check is chosen so that a plausible slip in the oracle fails at least one
of them:

* free-field closed form (U = 1): a dropped direction, a wrong staggered phase
  (the phases must anticommute), a wrong sign on the backward hop or a missing
  antiperiodic boundary all change the plane-wave eigenvalue of
  A = m^2 - D^2 (Eq. 3, Eq. 5 without a factor 1/2: 4 sum sin^2 p);
* anti-Hermiticity of D (Eq. 4/5: <u, D v> = -<D u, v>): a backward hop
  without the dagger, a transposed link, or a boundary sign taken from the
  wrong end of the link breaks it;
* gauge covariance under a random SU(3) transformation: a link used at the
  wrong site or a conjugated instead of daggered link breaks it;
* Hermiticity / positivity of A and its spectrum bounds [m^2, m^2 + 64];
* CG (Fig. 1): exact dense solves on 2^4 (x+mu and x-mu coincide) and 4^4,
  one-iteration convergence on an eigenvector, termination after as many
  iterations as distinct eigenvalues, the closed-form first step, and the
  monotone A-norm error.
"""
import numpy as np
import pytest

import gen
from lattice_util import (dense_A, free_eigenvalue, momentum, plane_wave, rel,
                          site_coords, transform_field, transform_gauge)

pytestmark = pytest.mark.usefixtures("oracle_lib")


def _o():
    import oracle
    return oracle


# --------------------------------------------------------------------------
# free field: closed form on plane waves
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 6, 2, 8), (6, 4, 4, 2)])
@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 0, 1),
                               (1, 2, 1, 0), (3, 1, 1, 2)])
def test_free_field_plane_wave_eigenvalue(dims, n):
    o = _o()
    mass = 0.3
    U = gen.unit_gauge(dims)
    p = momentum(dims, n)
    phi = plane_wave(dims, p, [0.3 - 0.1j, 1.0, 0.2j], parity=0)
    lam = free_eigenvalue(p, mass)
    Aphi = o.apply_A(dims, U, mass, phi)
    assert rel(Aphi, lam * phi) < 1e-13


def test_free_field_single_site_hop_sum():
    """With U = 1, (D_oe phi)(x) at one odd site equals the eight hops written
    out with eta_mu(x) = (-1)^(x_0+..+x_{mu-1}) (x, y, z, t order) and the -1
    carried by the t-link that crosses the time boundary."""
    o = _o()
    dims = (4, 4, 4, 4)
    U = gen.unit_gauge(dims)
    p = momentum(dims, (1, 0, 1, 0))
    phi = plane_wave(dims, p, [1.0, 0.0, 0.0], parity=0)
    out = o.dslash(dims, U, phi, out_parity=1)
    c_odd = site_coords(dims, 1)
    L = np.array(dims)
    for x in ([1, 0, 0, 0], [0, 1, 2, 0], [3, 3, 2, 3]):
        x = np.array(x)
        k = int(np.nonzero((c_odd == x).all(axis=1))[0][0])
        want = 0
        for mu in range(4):
            e = np.zeros(4, int)
            e[mu] = 1
            eta = (-1) ** int(np.sum(x[:mu]))
            xf, xb = (x + e) % L, (x - e) % L
            sf = -1 if (mu == 3 and x[3] == L[3] - 1) else 1   # link at x
            sb = -1 if (mu == 3 and xb[3] == L[3] - 1) else 1  # link at x - mu
            want += eta * (sf * np.exp(1j * p @ xf) - sb * np.exp(1j * p @ xb))
        assert abs(out[k, 0] - want) < 1e-13
        assert abs(out[k, 1]) < 1e-14 and abs(out[k, 2]) < 1e-14


# --------------------------------------------------------------------------
# anti-Hermiticity, Hermiticity, positivity
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(4, 2, 6, 4), (2, 2, 2, 2), (4, 4, 4, 6)])
def test_dslash_anti_hermitian(dims):
    o = _o()
    U = gen.gauge_field(dims, "haar", seed=3)
    vh = np.prod(dims) // 2
    g = gen.rng(11)
    ue = gen.complex_gaussian(g, (vh, 3))
    vo = gen.complex_gaussian(g, (vh, 3))
    lhs = np.vdot(ue, o.dslash(dims, U, vo, out_parity=0))   # <u_e, D_eo v_o>
    rhs = -np.vdot(o.dslash(dims, U, ue, out_parity=1), vo)  # -<D_oe u_e, v_o>
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_A_hermitian_positive_and_bounded():
    o = _o()
    dims = (4, 4, 2, 6)
    mass = 0.2
    U = gen.gauge_field(dims, "exp", seed=5, eps=0.6)
    vh = np.prod(dims) // 2
    g = gen.rng(12)
    for _ in range(4):
        u = gen.complex_gaussian(g, (vh, 3))
        v = gen.complex_gaussian(g, (vh, 3))
        Au, Av = o.apply_A(dims, U, mass, u), o.apply_A(dims, U, mass, v)
        assert abs(np.vdot(u, Av) - np.vdot(Au, v)) < 1e-12 * abs(np.vdot(u, Av))
        rq = np.vdot(u, Au) / np.vdot(u, u)
        assert abs(rq.imag) < 1e-12 * abs(rq)
        assert mass ** 2 <= rq.real <= mass ** 2 + 64.0


# --------------------------------------------------------------------------
# gauge covariance
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 2, 6)])
def test_gauge_covariance(dims):
    o = _o()
    mass = 0.15
    U = gen.gauge_field(dims, "haar", seed=21)
    G = gen.gauge_transform(dims, seed=22)
    Ug = transform_gauge(dims, U, G)
    chi = gen.source(dims, seed=23)
    chig = transform_field(dims, G, chi, parity=0)
    # D_oe is covariant: D[U^g] (g chi) = g D[U] chi  (odd output)
    lhs = o.dslash(dims, Ug, chig, out_parity=1)
    rhs = transform_field(dims, G, o.dslash(dims, U, chi, out_parity=1), parity=1)
    assert rel(lhs, rhs) < 1e-13
    lhs = o.apply_A(dims, Ug, mass, chig)
    rhs = transform_field(dims, G, o.apply_A(dims, U, mass, chi), parity=0)
    assert rel(lhs, rhs) < 1e-13


def test_gauge_covariance_fails_for_wrong_transform():
    """The covariance check has teeth: an inconsistent transform is caught."""
    o = _o()
    dims = (4, 4, 4, 4)
    U = gen.gauge_field(dims, "haar", seed=21)
    G = gen.gauge_transform(dims, seed=22)
    Ug = transform_gauge(dims, U, np.conj(G))  # conj(g) applied to links only
    chi = gen.source(dims, seed=23)
    lhs = o.apply_A(dims, Ug, 0.15, transform_field(dims, G, chi, 0))
    rhs = transform_field(dims, G, o.apply_A(dims, U, 0.15, chi), 0)
    assert rel(lhs, rhs) > 1e-2


# --------------------------------------------------------------------------
# dense matrices: 2^4 and 4^4
# --------------------------------------------------------------------------
def test_dense_2x4_matrix_and_solve():
    o = _o()
    dims = (2, 2, 2, 2)
    mass = 0.1
    U = gen.gauge_field(dims, "haar", seed=0)
    M = dense_A(o, dims, U, mass)
    assert M.shape == (24, 24)
    assert np.abs(M - M.conj().T).max() < 1e-13
    w = np.linalg.eigvalsh(M)
    assert w.min() >= mass ** 2 - 1e-12 and w.max() <= mass ** 2 + 64 + 1e-12
    b = gen.source(dims, seed=1)
    x_dense = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
    x, info = o.cg(dims, U, mass, b, tol=1e-10, maxiter=500)
    assert info["status"] == 0 and info["true_res"] <= 1e-10
    kappa = w.max() / w.min()
    assert rel(x, x_dense) <= kappa * 1e-10


def test_dense_4x4_c1_solve():
    """4^4, Haar links (seed 0), m = 0.1, source seed 1, tol 1e-10, FP64 CG."""
    o = _o()
    dims = (4, 4, 4, 4)
    mass = 0.1
    U = gen.gauge_field(dims, "haar", seed=0)
    b = gen.source(dims, seed=1)
    M = dense_A(o, dims, U, mass)
    w = np.linalg.eigvalsh(M)
    x_dense = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
    x, info = o.cg(dims, U, mass, b, tol=1e-10)
    assert info["status"] == 0
    assert info["true_res"] <= 1e-10
    # independent residual with the dense matrix
    r = b.reshape(-1) - M @ x.reshape(-1)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    assert rel(x, x_dense) <= (w.max() / w.min()) * 1e-10


# --------------------------------------------------------------------------
# CG behaviour fixed by the mathematics
# --------------------------------------------------------------------------
def test_cg_eigenvector_converges_in_one_iteration():
    o = _o()
    dims = (4, 4, 4, 8)
    mass = 0.05
    U = gen.unit_gauge(dims)
    p = momentum(dims, (1, 1, 0, 2))
    b = plane_wave(dims, p, [0.5, 0.25j, -1.0])
    x, info = o.cg(dims, U, mass, b, tol=1e-12)
    assert info["iters"] == 1
    assert rel(x, b / free_eigenvalue(p, mass)) < 1e-13


def test_cg_terminates_after_distinct_eigenvalues():
    """b in the span of 3 eigenvectors with distinct eigenvalues: CG ends in
    exactly 3 iterations at the closed-form solution sum c_k/lambda_k phi_k."""
    o = _o()
    dims = (4, 4, 4, 4)
    mass = 0.2
    U = gen.unit_gauge(dims)
    modes = [(0, 0, 0, 0), (1, 0, 0, 0), (1, 1, 1, 1)]
    coefs = [1.0, 0.5 - 0.5j, 2.0j]
    b = 0
    xstar = 0
    lams = []
    for n, c in zip(modes, coefs):
        p = momentum(dims, n)
        phi = plane_wave(dims, p, [1.0, -1.0j, 0.5])
        lam = free_eigenvalue(p, mass)
        lams.append(lam)
        b = b + c * phi
        xstar = xstar + c / lam * phi
    assert len(set(np.round(lams, 12))) == 3
    x, info = o.cg(dims, U, mass, b, tol=1e-13)
    assert info["iters"] == 3
    assert rel(x, xstar) < 1e-12


def test_cg_first_step_closed_form_and_monotone_error():
    """x_1 = (b^dag b / b^dag A b) b (Fig. 1 with x0 = 0), and the A-norm of
    the error decreases every iteration (4^4, Haar, m = 0.1)."""
    o = _o()
    dims = (4, 4, 4, 4)
    mass = 0.1
    U = gen.gauge_field(dims, "haar", seed=0)
    b = gen.source(dims, seed=1)
    M = dense_A(o, dims, U, mass)
    xstar = np.linalg.solve(M, b.reshape(-1))
    bv = b.reshape(-1)
    x1, _ = o.cg(dims, U, mass, b, tol=0.0, maxiter=1, max_restarts=0)
    want = (np.vdot(bv, bv) / np.vdot(bv, M @ bv)).real * bv
    assert rel(x1.reshape(-1), want) < 1e-13
    prev = np.inf
    for k in range(1, 40):
        xk, info = o.cg(dims, U, mass, b, tol=0.0, maxiter=k, max_restarts=0)
        assert info["iters"] == k
        e = xk.reshape(-1) - xstar
        anorm = np.sqrt(np.vdot(e, M @ e).real)
        assert anorm < prev
        prev = anorm


def test_cg_restart_from_true_residual():
    """With maxiter hit first, the status is not-converged and x is the k-th
    iterate; the default call restarts on the true residual and converges."""
    o = _o()
    dims = (4, 4, 4, 4)
    U = gen.gauge_field(dims, "exp", seed=2, eps=0.5)
    b = gen.source(dims, seed=3)
    x, info = o.cg(dims, U, 0.1, b, tol=1e-10, maxiter=5, max_restarts=0)
    assert info["status"] == o.NOT_CONVERGED and info["iters"] == 5
    x, info = o.cg(dims, U, 0.1, b, tol=1e-10)
    assert info["status"] == 0 and info["true_res"] <= 1e-10


def test_x0_is_respected():
    o = _o()
    dims = (4, 4, 4, 4)
    U = gen.gauge_field(dims, "haar", seed=0)
    b = gen.source(dims, seed=1)
    xs, _ = o.cg(dims, U, 0.1, b, tol=1e-12)
    x, info = o.cg(dims, U, 0.1, b, tol=1e-10, x0=xs)
    assert info["iters"] == 0 and rel(x, xs) == 0.0


# --------------------------------------------------------------------------
# argument checking
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(3, 4, 4, 4), (4, 4, 0, 4), (4, 4, 4, 5)])
def test_odd_or_zero_dims_rejected(dims):
    o = _o()
    lx, ly, lz, lt = dims
    U = np.zeros((lt, lz, ly, lx, 4, 3, 3), complex)
    chi = np.zeros((lx * ly * lz * lt // 2, 3), complex)
    with pytest.raises(ValueError, match="oracle error -1"):
        o.dslash(dims, U, chi, 0)


def test_dslash_sites_matches_full():
    o = _o()
    dims = (4, 6, 4, 4)
    U = gen.gauge_field(dims, "haar", seed=9)
    chi = gen.source(dims, seed=10)
    full = o.dslash(dims, U, chi, out_parity=0)
    sites = [0, 7, 95, 191, 13]
    part = o.dslash_sites(dims, U, chi, 0, sites)
    assert np.array_equal(part, full[sites])
