"""Seeded synthetic inputs for the staggered-fermion CG path.

This module only *draws* inputs: SU(3) gauge links, colour-vector sources and
gauge transformations, in the canonical FP64 host layouts that both the CPU
oracle and the CUDA library accept.  It contains none of the method's
arithmetic (no staggered phases, no boundary signs, no Dirac operator, no CG):
those live separately in ``oracle/`` and in the CUDA sources.

Canonical layouts (complex128, C order):

* gauge field ``[Lt][Lz][Ly][Lx][4][3][3]`` -- U_mu(x) for mu = x, y, z, t,
  *without* staggered phases or boundary signs (the paper folds eta_mu(x)
  into the links as a preconditioning step, Sec. 2 after Eq. 5; here that
  step belongs to the consumer);
* fermion field on one checkerboard ``[Vh][3]`` with site index
  i = (x + Lx*(y + Ly*(z + Lz*t))) >> 1 over the sites of that parity.

Random streams: ``numpy.random.Generator(PCG64(seed))``.  Links are drawn in
lexicographic site order (x fastest), then mu.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "complex_gaussian",
    "haar_su3",
    "exp_ih_su3",
    "gauge_field",
    "unit_gauge",
    "source",
    "gauge_transform",
    "lattice_volume",
    "log_uniform",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def lattice_volume(dims) -> int:
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def complex_gaussian(g: np.random.Generator, shape) -> np.ndarray:
    """Complex normal with E|z|^2 = 1 (real and imaginary parts N(0, 1/2))."""
    re = g.standard_normal(shape)
    im = g.standard_normal(shape)
    return (re + 1j * im) * np.sqrt(0.5)


def _cbrt_principal(z: np.ndarray) -> np.ndarray:
    return np.abs(z) ** (1.0 / 3.0) * np.exp(1j * np.angle(z) / 3.0)


def haar_su3(g: np.random.Generator, n: int, chunk: int = 1 << 20) -> np.ndarray:
    """n Haar-distributed SU(3) matrices.

    QR of a complex Gaussian 3x3 matrix gives a Haar unitary once the phases
    of R's diagonal are moved into Q; dividing by the principal cube root of
    the determinant then lands in SU(3).
    """
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        z = complex_gaussian(g, (m, 3, 3))
        q, r = np.linalg.qr(z)
        d = np.diagonal(r, axis1=-2, axis2=-1)
        q = q * (d / np.abs(d))[:, None, :]
        det = np.linalg.det(q)
        out[s:s + m] = q / _cbrt_principal(det)[:, None, None]
    return out


def _project_su3_rows(u: np.ndarray) -> np.ndarray:
    """Gram-Schmidt on rows 0 and 1, row 2 = conj(row0 x row1)."""
    r0 = u[:, 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[:, 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=1)


def exp_ih_su3(g: np.random.Generator, n: int, eps: float,
               chunk: int = 1 << 20) -> np.ndarray:
    """n links U = exp(i*eps*H), H random traceless Hermitian, then SU(3).

    H = (G + G^dag)/2 - tr(.)/3 with G i.i.d. complex Gaussian (E|g|^2 = 1);
    the exponential goes through a Hermitian eigendecomposition in FP64 and
    the result is re-projected onto SU(3) row by row.
    """
    out = np.empty((n, 3, 3), dtype=np.complex128)
    eye = np.eye(3)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        gm = complex_gaussian(g, (m, 3, 3))
        h = 0.5 * (gm + np.conj(np.swapaxes(gm, -1, -2)))
        tr = np.trace(h, axis1=-2, axis2=-1).real
        h = h - (tr / 3.0)[:, None, None] * eye
        w, v = np.linalg.eigh(h)
        u = (v * np.exp(1j * eps * w)[:, None, :]) @ np.conj(np.swapaxes(v, -1, -2))
        out[s:s + m] = _project_su3_rows(u)
    return out


def gauge_field(dims, kind: str = "haar", seed: int = 0, eps: float = 0.5) -> np.ndarray:
    """Gauge field in the canonical layout [Lt][Lz][Ly][Lx][4][3][3].

    kind: "haar" (Haar SU(3) links), "exp" (exp(i*eps*H) links) or "unit".
    """
    lx, ly, lz, lt = (int(d) for d in dims)
    n = lattice_volume(dims) * 4
    if kind == "unit":
        u = np.broadcast_to(np.eye(3, dtype=np.complex128), (n, 3, 3)).copy()
    elif kind == "haar":
        u = haar_su3(rng(seed), n)
    elif kind == "exp":
        u = exp_ih_su3(rng(seed), n, eps)
    else:
        raise ValueError(f"unknown gauge kind {kind!r}")
    return u.reshape(lt, lz, ly, lx, 4, 3, 3)


def unit_gauge(dims) -> np.ndarray:
    return gauge_field(dims, kind="unit")


def source(dims, seed: int = 1, nrhs: int | None = None) -> np.ndarray:
    """Complex Gaussian colour vectors on one checkerboard, [Vh][3] (or
    [nrhs][Vh][3] when nrhs is given, drawn one right-hand side after another)."""
    vh = lattice_volume(dims) // 2
    g = rng(seed)
    if nrhs is None:
        return complex_gaussian(g, (vh, 3))
    return complex_gaussian(g, (int(nrhs), vh, 3))


def gauge_transform(dims, seed: int = 7) -> np.ndarray:
    """Haar SU(3) matrix per site, [Lt][Lz][Ly][Lx][3][3]."""
    lx, ly, lz, lt = (int(d) for d in dims)
    return haar_su3(rng(seed), lattice_volume(dims)).reshape(lt, lz, ly, lx, 3, 3)


def log_uniform(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """n values log-uniform in [lo, hi] (e.g. quark masses of a batch)."""
    g = rng(seed)
    return np.exp(g.uniform(np.log(lo), np.log(hi), size=int(n)))
