"""FP64 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline / reference leg may import this package.  The product library never
loads it, and it never loads the product library: the two share no code.

The arithmetic lives in ``stg_oracle.c`` (plain C, FP64, loops over lattice
coordinates); this module compiles it with gcc and wraps it with ctypes.
Every function takes and returns canonical complex128 numpy arrays:
links ``[Lt][Lz][Ly][Lx][4][3][3]`` without phases, fields ``[Vh][3]`` on one
checkerboard.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_DIMS, ERR_ARG, ERR_OOM, NOT_CONVERGED, BREAKDOWN = 0, -1, -2, -3, 1, 2

# Compiler flags: plain -O2, no fast-math (IEEE FP64 semantics), no
# machine-specific ISA flags so x86 and Arm hosts compute the same thing.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile stg_oracle.c into liboracle.so next to it (gcc)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        p = ctypes.c_void_p
        lib.orc_dslash.argtypes = [p, p, p, p, ctypes.c_int]
        lib.orc_dslash_sites.argtypes = [p, p, p, ctypes.c_int, p, ctypes.c_long, p]
        lib.orc_apply_A.argtypes = [p, p, ctypes.c_double, p, p]
        lib.orc_cg.argtypes = [p, p, ctypes.c_double, p, p, ctypes.c_double,
                               ctypes.c_long, ctypes.c_int, p, p]
        lib.orc_cg_mixed.argtypes = [p, p, ctypes.c_double, p, p, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_long, ctypes.c_int, p, p]
        lib.orc_cg_mixed_snap.argtypes = [p, p, ctypes.c_double, p, p, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_long, ctypes.c_int, p, p,
                                          p, p]
        for f in ("orc_dslash", "orc_dslash_sites", "orc_apply_A", "orc_cg", "orc_cg_mixed"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _dims(dims) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(4))


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _vh(dims) -> int:
    d = [int(v) for v in dims]
    return d[0] * d[1] * d[2] * d[3] // 2


def _check_shapes(dims, U, chi):
    d = [int(v) for v in dims]
    if U.shape != (d[3], d[2], d[1], d[0], 4, 3, 3):
        raise ValueError(f"links have shape {U.shape}, expected "
                         f"{(d[3], d[2], d[1], d[0], 4, 3, 3)}")
    if chi is not None and chi.shape != (_vh(dims), 3):
        raise ValueError(f"field has shape {chi.shape}, expected {(_vh(dims), 3)}")


def _raise(code: int, what: str):
    if code < 0:
        raise ValueError(f"{what}: oracle error {code}")


def dslash(dims, U, chi, out_parity: int) -> np.ndarray:
    """D_{p <- 1-p} chi (Eq. 5) on the sites of parity ``out_parity``."""
    lib = _load()
    dd, U, chi = _dims(dims), _c128(U), _c128(chi)
    _check_shapes(dims, U, chi)
    out = np.empty_like(chi)
    _raise(lib.orc_dslash(_ptr(dd), _ptr(U), _ptr(chi), _ptr(out), int(out_parity)), "dslash")
    return out


def dslash_sites(dims, U, chi, out_parity: int, sites) -> np.ndarray:
    """D_{p <- 1-p} chi evaluated only at the checkerboard indices ``sites``."""
    lib = _load()
    dd, U, chi = _dims(dims), _c128(U), _c128(chi)
    _check_shapes(dims, U, chi)
    s = np.ascontiguousarray(np.asarray(sites, dtype=np.int64).reshape(-1))
    out = np.empty((s.size, 3), dtype=np.complex128)
    _raise(lib.orc_dslash_sites(_ptr(dd), _ptr(U), _ptr(chi), int(out_parity),
                                _ptr(s), s.size, _ptr(out)), "dslash_sites")
    return out


def apply_A(dims, U, mass: float, chi) -> np.ndarray:
    """(m^2 - D_eo D_oe) chi on even sites (Eq. 3)."""
    lib = _load()
    dd, U, chi = _dims(dims), _c128(U), _c128(chi)
    _check_shapes(dims, U, chi)
    out = np.empty_like(chi)
    _raise(lib.orc_apply_A(_ptr(dd), _ptr(U), float(mass), _ptr(chi), _ptr(out)), "apply_A")
    return out


def cg(dims, U, mass: float, b, tol: float = 1e-10, maxiter: int | None = None,
       x0=None, max_restarts: int = 10):
    """Fig. 1 CG with a true-residual restart.

    Returns (x, info) with info = dict(status, iters, restarts, true_res).
    maxiter defaults to 10 N_dim (N_dim = 3 Vh is Fig. 1's loop bound, which
    finite-precision CG can exceed once the search directions lose their
    A-orthogonality).
    """
    lib = _load()
    dd, U, b = _dims(dims), _c128(U), _c128(b)
    _check_shapes(dims, U, b)
    x = np.zeros_like(b) if x0 is None else _c128(x0).copy()
    if maxiter is None:
        maxiter = 10 * 3 * _vh(dims)
    info = np.zeros(2, dtype=np.int64)
    res = np.zeros(1, dtype=np.float64)
    st = lib.orc_cg(_ptr(dd), _ptr(U), float(mass), _ptr(b), _ptr(x), float(tol),
                    int(maxiter), int(max_restarts), _ptr(info), _ptr(res))
    _raise(st, "cg")
    return x, dict(status=int(st), iters=int(info[0]), restarts=int(info[1]),
                   true_res=float(res[0]))


def cg_mixed(dims, U, mass: float, b, tol: float = 1e-10, delta: float = 0.1,
             maxiter: int | None = None, x0=None, refine: bool = False,
             snapshot: bool = False):
    """Mixed-precision CG (Fig. 2, Eq. 6, Sec. 3.2) emulated with single-
    precision inner vectors and double updates; refine=True gives Fig. 2's
    plain iterative refinement (inner solves restart from d = r).

    Returns (x, info) with info = dict(status, iters, updates, true_res,
    low_precision_fraction = iters / (iters + updates)).  With snapshot=True,
    info["first_update"] holds the state around the first reliable update
    that does not end the solve (None if there is none): rho_prev and
    rho_iter (the iterated |r^|^2 before and after the triggering step),
    true2 (|r|^2 of the new true residual), and the vectors x (after the
    update), d_old, r_hat (after it) and d_new.
    """
    lib = _load()
    dd, U, b = _dims(dims), _c128(U), _c128(b)
    _check_shapes(dims, U, b)
    x = np.zeros_like(b) if x0 is None else _c128(x0).copy()
    if maxiter is None:
        maxiter = 10 * 3 * _vh(dims)
    info = np.zeros(2, dtype=np.int64)
    res = np.zeros(1, dtype=np.float64)
    snap_s = np.zeros(4, dtype=np.float64)
    snap_v = np.zeros((4,) + b.shape, dtype=np.complex128) if snapshot else None
    st = lib.orc_cg_mixed_snap(_ptr(dd), _ptr(U), float(mass), _ptr(b), _ptr(x), float(tol),
                               float(delta), int(maxiter), int(bool(refine)), _ptr(info),
                               _ptr(res), _ptr(snap_s) if snapshot else None,
                               _ptr(snap_v) if snapshot else None)
    _raise(st, "cg_mixed")
    it, up = int(info[0]), int(info[1])
    out = dict(status=int(st), iters=it, updates=up, true_res=float(res[0]),
               low_precision_fraction=it / max(1, it + up))
    if snapshot:
        out["first_update"] = None if snap_s[3] == 0.0 else dict(
            rho_prev=float(snap_s[0]), rho_iter=float(snap_s[1]), true2=float(snap_s[2]),
            x=snap_v[0].copy(), d_old=snap_v[1].copy(), r_hat=snap_v[2].copy(),
            d_new=snap_v[3].copy())
    return x, out
