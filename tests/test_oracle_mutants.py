"""The oracle's pins catch plausible mistakes.

Each case below plants one mistake in a copy of oracle/stg_oracle.c -- a
dropped direction, a wrong sign, a missing dagger, a transposed link, a wrong
staggered phase or boundary, a wrong neighbour or checkerboard index, a wrong
CG coefficient, a plain-CG beta at the mixed solver's update -- compiles the copy, and requires at least one pin check to
fail; the unchanged oracle must pass all of them.  A reversed phase order is
a valid convention with the same spectrum, so only the explicit single-site
hop sum catches that one.  The mistakes live only in temporary copies on the
CPU.
"""
import importlib.util
import os
import shutil

import numpy as np
import pytest

import gen
from lattice_util import (dense_A, free_eigenvalue, momentum, plane_wave, rel,
                          site_coords, transform_field, transform_gauge)
from test_oracle_mixed import _eq6_direction_error

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "stg_oracle.c")

MUTANTS = {
    "drop_t_direction": ("for (int mu = 0; mu < 4; ++mu) {\n        int cf[4], cb[4];",
                         "for (int mu = 0; mu < 3; ++mu) {\n        int cf[4], cb[4];"),
    "backward_hop_sign": ("acc[a] -= sb * conj(ub[b * 3 + a]) * xb[b];",
                          "acc[a] += sb * conj(ub[b * 3 + a]) * xb[b];"),
    "no_dagger": ("acc[a] -= sb * conj(ub[b * 3 + a]) * xb[b];",
                  "acc[a] -= sb * ub[a * 3 + b] * xb[b];"),
    "conjugate_not_transposed": ("acc[a] -= sb * conj(ub[b * 3 + a]) * xb[b];",
                                 "acc[a] -= sb * conj(ub[a * 3 + b]) * xb[b];"),
    "transposed_forward_link": ("acc[a] += sf * uf[a * 3 + b] * xf[b];",
                                "acc[a] += sf * uf[b * 3 + a] * xf[b];"),
    "eta_reversed_order": ("for (int nu = 0; nu < mu; ++nu) s += c[nu];",
                           "for (int nu = mu + 1; nu < 4; ++nu) s += c[nu];"),
    "boundary_sign_from_wrong_end": ("double sb = (double)(eta(mu, cb) * bsign(L, mu, cb));",
                                     "double sb = (double)(eta(mu, cb) * bsign(L, mu, c));"),
    "periodic_time": ("return (mu == 3 && c[3] == L[3] - 1) ? -1 : 1;", "return 1;"),
    "mass_term_sign": ("out[k] = m2 * in[k] - out[k];", "out[k] = m2 * in[k] + out[k];"),
    "forward_reads_backward_site": ("const cplx *xf = in + (lex(L, cf) >> 1) * 3;",
                                    "const cplx *xf = in + (lex(L, cb) >> 1) * 3;"),
    "wrong_checkerboard_site": ("if (((x + y + z + t) & 1) != p) x += 1;",
                                "if (((x + y + z + t) & 1) == p) x += 1;"),
    "cg_beta_inverted": ("double beta = delta_new / delta_old;",
                         "double beta = delta_old / delta_new;"),
    "cg_alpha_without_A": ("double alpha = delta_new / dq;",
                           "double alpha = delta_new / re_dot(d, d, n);"),
    "mixed_beta_from_iterated_residual": ("mult = refine ? 0.0 : true2 / rho_prev;",
                                          "mult = refine ? 0.0 : rho / rho_prev;"),
}


def _load(tmpdir, name, src_text):
    """A private copy of the oracle package compiled from `src_text`."""
    d = os.path.join(tmpdir, name)
    os.makedirs(d, exist_ok=True)
    with open(os.path.join(d, "stg_oracle.c"), "w") as f:
        f.write(src_text)
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), os.path.join(d, "__init__.py"))
    spec = importlib.util.spec_from_file_location(f"oracle_{name}", os.path.join(d, "__init__.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    return mod


def _pin_failures(o):
    fails = []

    def check(name, fn):
        try:
            if not fn():
                fails.append(name)
        except Exception:
            fails.append(name)

    def free_field():
        dims, mass = (4, 6, 2, 8), 0.3
        p = momentum(dims, (1, 2, 1, 0))
        phi = plane_wave(dims, p, [0.3 - 0.1j, 1.0, 0.2j])
        return rel(o.apply_A(dims, gen.unit_gauge(dims), mass, phi),
                   free_eigenvalue(p, mass) * phi) < 1e-13

    def anti_hermitian():
        dims = (4, 2, 6, 4)
        U = gen.gauge_field(dims, "haar", seed=3)
        g = gen.rng(11)
        vh = np.prod(dims) // 2
        u, v = gen.complex_gaussian(g, (vh, 3)), gen.complex_gaussian(g, (vh, 3))
        lhs = np.vdot(u, o.dslash(dims, U, v, 0))
        rhs = -np.vdot(o.dslash(dims, U, u, 1), v)
        return abs(lhs - rhs) < 1e-12 * abs(lhs)

    def covariance():
        dims, mass = (2, 4, 2, 6), 0.15
        U = gen.gauge_field(dims, "haar", seed=21)
        G = gen.gauge_transform(dims, seed=22)
        chi = gen.source(dims, seed=23)
        lhs = o.apply_A(dims, transform_gauge(dims, U, G), mass, transform_field(dims, G, chi, 0))
        rhs = transform_field(dims, G, o.apply_A(dims, U, mass, chi), 0)
        return rel(lhs, rhs) < 1e-13

    def dense_solve():
        dims, mass = (2, 2, 2, 2), 0.1
        U = gen.gauge_field(dims, "haar", seed=0)
        b = gen.source(dims, seed=1)
        M = dense_A(o, dims, U, mass)
        if np.abs(M - M.conj().T).max() > 1e-13:
            return False
        xd = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
        x, info = o.cg(dims, U, mass, b, tol=1e-10, maxiter=500)
        w = np.linalg.eigvalsh(M)
        return info["status"] == 0 and rel(x, xd) <= w.max() / w.min() * 1e-10

    def one_iteration():
        dims, mass = (4, 4, 4, 8), 0.05
        p = momentum(dims, (1, 1, 0, 2))
        b = plane_wave(dims, p, [0.5, 0.25j, -1.0])
        x, info = o.cg(dims, gen.unit_gauge(dims), mass, b, tol=1e-12)
        return info["iters"] == 1 and rel(x, b / free_eigenvalue(p, mass)) < 1e-13

    def hop_sum():
        # the explicit eta convention (x, y, z, t order) at single sites: the
        # spectral pins cannot tell it from other valid phase conventions
        dims = (4, 4, 4, 4)
        p = momentum(dims, (1, 0, 1, 0))
        phi = plane_wave(dims, p, [1.0, 0.0, 0.0])
        out = o.dslash(dims, gen.unit_gauge(dims), phi, 1)
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
                sf = -1 if (mu == 3 and x[3] == L[3] - 1) else 1
                sb = -1 if (mu == 3 and xb[3] == L[3] - 1) else 1
                want += eta * (sf * np.exp(1j * p @ xf) - sb * np.exp(1j * p @ xb))
            if abs(out[k, 0] - want) > 1e-13:
                return False
        return True

    def eq6_direction():
        err, gap, same_r = _eq6_direction_error(o)
        return same_r and gap > 1e-4 and err < 1e-6 * gap

    for name, fn in [("free_field", free_field), ("hop_sum", hop_sum),
                     ("eq6_direction", eq6_direction),
                     ("anti_hermitian", anti_hermitian),
                     ("covariance", covariance), ("dense_solve", dense_solve),
                     ("one_iteration", one_iteration)]:
        check(name, fn)
    return fails


@pytest.fixture(scope="module")
def source_text():
    with open(SRC) as f:
        return f.read()


def test_unchanged_oracle_passes_every_pin(tmp_path, source_text):
    assert _pin_failures(_load(str(tmp_path), "base", source_text)) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, source_text, name):
    old, new = MUTANTS[name]
    assert source_text.count(old) == 1, f"mutation site of {name} not unique"
    mutant = _load(str(tmp_path), name, source_text.replace(old, new))
    assert _pin_failures(mutant), f"no pin catches {name}"
