"""Small helpers for tests: coordinates, plane waves, gauge transforms.

These restate lattice bookkeeping (coordinates of checkerboard sites) and the
free-field closed form; they are independent of both the oracle and the CUDA
library, and carry none of the method's kernels.
"""
import numpy as np


def site_coords(dims, parity):
    """(Vh, 4) integer coordinates (x, y, z, t) of the sites of ``parity``,
    in checkerboard order i = lex >> 1."""
    lx, ly, lz, lt = dims
    lexi = np.arange(lx * ly * lz * lt)
    x = lexi % lx
    y = (lexi // lx) % ly
    z = (lexi // (lx * ly)) % lz
    t = lexi // (lx * ly * lz)
    par = (x + y + z + t) % 2
    sel = par == parity
    c = np.stack([x[sel], y[sel], z[sel], t[sel]], axis=1)
    idx = lexi[sel] >> 1
    order = np.argsort(idx)
    assert np.array_equal(idx[order], np.arange(idx.size))
    return c[order]


def momentum(dims, n):
    """Allowed momentum: periodic in x, y, z (2 pi n / L), antiperiodic in t
    (pi (2 n + 1) / L)."""
    lx, ly, lz, lt = dims
    return np.array([2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly,
                     2 * np.pi * n[2] / lz, np.pi * (2 * n[3] + 1) / lt])


def plane_wave(dims, p, colour, parity=0):
    c = site_coords(dims, parity)
    phase = np.exp(1j * (c @ p))
    return phase[:, None] * np.asarray(colour, dtype=np.complex128)[None, :]


def free_eigenvalue(p, mass):
    """A = m^2 - D^2 on a free-field plane wave, D without a factor 1/2:
    -D^2 phi = 4 sum_mu sin^2(p_mu) phi."""
    return mass ** 2 + 4.0 * np.sum(np.sin(p) ** 2)


def transform_gauge(dims, U, g):
    """U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dag (periodic index arithmetic; the
    transformation does not touch boundary signs, which the consumer adds)."""
    Ug = np.empty_like(U)
    axes = {0: 3, 1: 2, 2: 1, 3: 0}  # mu -> array axis in [t][z][y][x]
    for mu in range(4):
        g_fwd = np.roll(g, -1, axis=axes[mu])
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(g_fwd, -1, -2))
    return Ug


def transform_field(dims, g, chi, parity):
    c = site_coords(dims, parity)
    gs = g[c[:, 3], c[:, 2], c[:, 1], c[:, 0]]
    return np.einsum("sab,sb->sa", gs, chi)


def dense_A(oracle, dims, U, mass):
    vh = np.prod(dims) // 2
    n = vh * 3
    M = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        e[:] = 0
        e[k] = 1
        M[:, k] = oracle.apply_A(dims, U, mass, e.reshape(vh, 3)).reshape(-1)
    return M


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)
