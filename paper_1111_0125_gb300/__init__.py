"""GB300 staggered-fermion Dirac operator and CG solver (Python binding).

A thin ctypes layer over the C ABI of ``include/stg.h``: every function
below has the name of the C entry point it calls and only marshals
arguments (device pointers, sizes, the CUDA stream).  All arithmetic runs in
the CUDA library ``libstg.so``; there is no Python or CPU fallback, and
importing this package fails loudly when the library has not been built
(``python -m paper_1111_0125_gb300.build`` or ``__graft_entry__.build()``).

PyTorch is used only as plumbing: tensors for device memory and the current
CUDA stream.  Pointer arguments accept an ``int`` address or a tensor.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstg.so")

STG_FP64, STG_FP32, STG_FP16, STG_FX16, STG_BF16 = 0, 1, 2, 3, 4
STG_CG_RELIABLE, STG_CG_REFINE, STG_CG_PLAIN = 0, 1, 2
(STG_OK, STG_ERR_INVALID_ARG, STG_ERR_DIMS, STG_ERR_OOM, STG_ERR_CUDA,
 STG_ERR_NOT_CONVERGED, STG_ERR_BREAKDOWN, STG_ERR_TIMEOUT,
 STG_ERR_UNSUPPORTED) = range(9)

PREC_NAMES = {STG_FP64: "f64", STG_FP32: "f32", STG_FP16: "f16", STG_FX16: "fx16", STG_BF16: "bf16"}
FIELD_SITE_BYTES = {STG_FP64: 48, STG_FP32: 24, STG_FP16: 16, STG_FX16: 16, STG_BF16: 16}


class StgError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str, stats=None):
        self.status = status
        self.stats = stats
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {detail}")


_STATUS = {STG_OK: "ok", STG_ERR_INVALID_ARG: "invalid argument",
           STG_ERR_DIMS: "invalid lattice dimensions", STG_ERR_OOM: "out of memory",
           STG_ERR_CUDA: "CUDA error", STG_ERR_NOT_CONVERGED: "not converged",
           STG_ERR_BREAKDOWN: "CG breakdown", STG_ERR_TIMEOUT: "device wait timed out",
           STG_ERR_UNSUPPORTED: "unsupported precision or reconstruction"}


class stg_cg_params(ctypes.Structure):
    _fields_ = [("policy", ctypes.c_int), ("sloppy", ctypes.c_int),
                ("delta", ctypes.c_double), ("maxiter", ctypes.c_long),
                ("check_every", ctypes.c_int), ("timing", ctypes.c_int)]


class stg_cg_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_long), ("sloppy_iters", ctypes.c_long),
                ("updates", ctypes.c_long), ("true_res", ctypes.c_double),
                ("iter_res", ctypes.c_double), ("seconds", ctypes.c_double),
                ("launches", ctypes.c_long), ("timed_iters", ctypes.c_long),
                ("t_dslash_ms", ctypes.c_double), ("t_dslash_a_ms", ctypes.c_double),
                ("t_update_ms", ctypes.c_double), ("t_xpay_ms", ctypes.c_double),
                ("t_iter_ms", ctypes.c_double), ("t_iter_serial_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: the CUDA library has not been built "
            "(run `python -m paper_1111_0125_gb300.build`); there is no fallback")
    lib = ctypes.CDLL(LIB_PATH)
    p, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "stg_version": (i, []),
        "stg_status_string": (ctypes.c_char_p, [i]),
        "stg_last_error": (ctypes.c_char_p, []),
        "stg_gauge_create": (i, [p, p, i, i, p, p]),
        "stg_gauge_destroy": (i, [p]),
        "stg_gauge_bytes": (sz, [p, i, i]),
        "stg_gauge_dims": (i, [p, p, p]),
        "stg_field_bytes": (i, [p, i, p]),
        "stg_pack_field": (i, [p, i, p, p, p]),
        "stg_unpack_field": (i, [p, i, p, p, p]),
        "stg_dslash": (i, [p, i, p, p, i, p]),
        "stg_apply_A": (i, [p, d, p, p, i, p]),
        "stg_apply_A_dot": (i, [p, d, p, p, p, i, p]),
        "stg_apply_A_dot_noalloc": (i, [p, d, p, p, p, i, p]),
        "stg_cg_params_default": (i, [p, p]),
        "stg_cg_solve": (i, [p, p, p, d, d, p, p, p]),
        "stg_dslash_mrhs": (i, [p, i, i, p, p, i, p]),
        "stg_dslash_group": (i, [i, p, p, p, p, i, p]),
        "stg_apply_A_mrhs": (i, [p, i, p, p, p, i, p]),
        "stg_cg_solve_mrhs": (i, [p, i, p, p, p, d, p, p, p]),
        "stg_mrhs_tuning": (i, [p, i, i, p, p]),
        "stg_batch_create": (i, [p, i, p, p, p]),
        "stg_batch_destroy": (i, [p]),
        "stg_batch_add": (i, [p, p, p, d, d, p]),
        "stg_batch_step": (i, [p, i, p, p, p, p, p]),
        "stg_batch_bytes": (sz, [p, i, i]),
        "stg_lgroup_create": (i, [i, ctypes.c_long, i, i, p, p, p]),
        "stg_lgroup_destroy": (i, [p]),
        "stg_lgroup_add": (i, [p, p, p, p, d, d, p]),
        "stg_lgroup_step": (i, [p, i, p, p, p, p, p]),
        "stg_lgroup_bytes": (sz, [i, ctypes.c_long, i]),
        "stg_slabs_create": (i, [p, p, i, i, i, p, p]),
        "stg_slabs_destroy": (i, [p]),
        "stg_slabs_set_exchange": (i, [p, i, i]),
        "stg_slabs_load": (i, [p, i, p, p]),
        "stg_slabs_store": (i, [p, i, p, p]),
        "stg_slabs_dslash": (i, [p, i, i, i, p]),
        "stg_slabs_apply_A_dot": (i, [p, d, i, i, p, p]),
        "stg_slabs_cg_solve": (i, [p, p, p, d, d, ctypes.c_long, p, p]),
        "stg_slabs_profile": (i, [p, i, p, p]),
        "stg_slabs_bytes": (sz, [p, i, i, i]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s) -> int:
    if s is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _check(st: int, where: str, stats=None):
    if st != STG_OK:
        raise StgError(st, where, stg_last_error(), stats)


def stg_version() -> int:
    return lib.stg_version()


def stg_status_string(status: int) -> str:
    return lib.stg_status_string(status).decode()


def stg_last_error() -> str:
    return lib.stg_last_error().decode()


def stg_gauge_create(dims, links_host: np.ndarray, sloppy: int = STG_FP32, recon: int = 18,
                     stream=None) -> int:
    """Upload canonical complex128 links [Lt][Lz][Ly][Lx][4][3][3] (host)."""
    dd = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(4))
    links = np.ascontiguousarray(links_host, dtype=np.complex128)
    lx, ly, lz, lt = (int(v) for v in dd)
    if links.size != lx * ly * lz * lt * 4 * 9:
        raise StgError(STG_ERR_INVALID_ARG, "stg_gauge_create",
                       f"links have {links.size} entries, expected {lx * ly * lz * lt * 36}")
    h = ctypes.c_void_p()
    st = lib.stg_gauge_create(dd.ctypes.data, links.ctypes.data, int(sloppy), int(recon),
                              _stream(stream), ctypes.byref(h))
    _check(st, "stg_gauge_create")
    return h.value


def stg_gauge_destroy(handle: int) -> None:
    lib.stg_gauge_destroy(handle)


def stg_gauge_dims(handle: int):
    dd = (ctypes.c_int * 4)()
    vh = ctypes.c_long()
    _check(lib.stg_gauge_dims(handle, dd, ctypes.byref(vh)), "stg_gauge_dims")
    return tuple(dd), vh.value


def stg_field_bytes(handle: int, prec: int) -> int:
    n = ctypes.c_size_t()
    _check(lib.stg_field_bytes(handle, int(prec), ctypes.byref(n)), "stg_field_bytes")
    return n.value


def stg_pack_field(handle: int, prec: int, canon_dev, field_dev, stream=None) -> None:
    _check(lib.stg_pack_field(handle, int(prec), _ptr(canon_dev), _ptr(field_dev), _stream(stream)),
           "stg_pack_field")


def stg_unpack_field(handle: int, prec: int, field_dev, canon_dev, stream=None) -> None:
    _check(lib.stg_unpack_field(handle, int(prec), _ptr(field_dev), _ptr(canon_dev), _stream(stream)),
           "stg_unpack_field")


def stg_dslash(handle: int, out_parity: int, in_dev, out_dev, prec: int, stream=None) -> None:
    _check(lib.stg_dslash(handle, int(out_parity), _ptr(in_dev), _ptr(out_dev), int(prec),
                          _stream(stream)), "stg_dslash")


def stg_apply_A(handle: int, mass: float, in_dev, out_dev, prec: int, stream=None) -> None:
    _check(lib.stg_apply_A(handle, float(mass), _ptr(in_dev), _ptr(out_dev), int(prec),
                           _stream(stream)), "stg_apply_A")


def stg_apply_A_dot(handle: int, mass: float, in_dev, out_dev, dot_dev, prec: int,
                    stream=None) -> None:
    _check(lib.stg_apply_A_dot(handle, float(mass), _ptr(in_dev), _ptr(out_dev), _ptr(dot_dev),
                               int(prec), _stream(stream)), "stg_apply_A_dot")


def stg_apply_A_dot_noalloc(handle: int, mass: float, in_dev, out_dev, dot_dev, prec: int,
                            stream=None) -> None:
    """stg_apply_A_dot for callers that cannot allocate device memory: the
    scratch is a fixed 32 MiB array reserved by the library on each device."""
    _check(lib.stg_apply_A_dot_noalloc(handle, float(mass), _ptr(in_dev), _ptr(out_dev),
                                       _ptr(dot_dev), int(prec), _stream(stream)),
           "stg_apply_A_dot_noalloc")


def stg_cg_params_default(handle: int) -> stg_cg_params:
    p = stg_cg_params()
    _check(lib.stg_cg_params_default(handle, ctypes.byref(p)), "stg_cg_params_default")
    return p


def stg_cg_solve(handle: int, src_dev, x_dev, mass: float, tol: float, params=None,
                 stream=None) -> dict:
    """Solve A x = b; x_dev holds x0 on entry.  Returns the stats as a dict;
    raises StgError (with .stats) on any non-OK status."""
    stats = stg_cg_stats()
    pp = ctypes.byref(params) if params is not None else None
    st = lib.stg_cg_solve(handle, _ptr(src_dev), _ptr(x_dev), float(mass), float(tol), pp,
                          ctypes.byref(stats), _stream(stream))
    _check(st, "stg_cg_solve", stats.as_dict())
    return stats.as_dict()


def stg_dslash_group(handles, out_parities, ins, outs, prec: int, stream=None) -> None:
    """out[k] = D in[k] on handles[k] for up to 16 lattices in one launch."""
    n = len(handles)
    if not (len(out_parities) == len(ins) == len(outs) == n):
        raise ValueError("stg_dslash_group: handles, parities, ins and outs differ in length")
    hs = (ctypes.c_void_p * n)(*[int(h) for h in handles])
    ps = (ctypes.c_int * n)(*[int(q) for q in out_parities])
    xi = (ctypes.c_void_p * n)(*[_ptr(x) for x in ins])
    xo = (ctypes.c_void_p * n)(*[_ptr(x) for x in outs])
    _check(lib.stg_dslash_group(n, hs, ps, xi, xo, int(prec), _stream(stream)), "stg_dslash_group")


def stg_dslash_mrhs(handle: int, out_parity: int, nrhs: int, in_dev, out_dev, prec: int,
                    stream=None) -> None:
    """out_k = D in_k for nrhs consecutive fields of one precision."""
    _check(lib.stg_dslash_mrhs(handle, int(out_parity), int(nrhs), _ptr(in_dev), _ptr(out_dev),
                               int(prec), _stream(stream)), "stg_dslash_mrhs")


def stg_apply_A_mrhs(handle: int, nrhs: int, masses, in_dev, out_dev, prec: int,
                     stream=None) -> None:
    m = np.ascontiguousarray(np.asarray(masses, dtype=np.float64).reshape(-1))
    if m.size != nrhs:
        raise StgError(STG_ERR_INVALID_ARG, "stg_apply_A_mrhs", "need one mass per system")
    _check(lib.stg_apply_A_mrhs(handle, int(nrhs), m.ctypes.data, _ptr(in_dev), _ptr(out_dev),
                                int(prec), _stream(stream)), "stg_apply_A_mrhs")


def stg_cg_solve_mrhs(handle: int, nrhs: int, src_dev, x_dev, masses, tol: float, params=None,
                      stream=None) -> list:
    """Batched solve of nrhs systems; returns one stats dict per system and
    raises StgError (with .stats = that list) on any non-OK status."""
    m = np.ascontiguousarray(np.asarray(masses, dtype=np.float64).reshape(-1))
    if m.size != nrhs:
        raise StgError(STG_ERR_INVALID_ARG, "stg_cg_solve_mrhs", "need one mass per system")
    stats = (stg_cg_stats * nrhs)()
    pp = ctypes.byref(params) if params is not None else None
    st = lib.stg_cg_solve_mrhs(handle, int(nrhs), _ptr(src_dev), _ptr(x_dev), m.ctypes.data,
                               float(tol), pp, stats, _stream(stream))
    out = [s.as_dict() for s in stats]
    _check(st, "stg_cg_solve_mrhs", out)
    return out


def stg_batch_create(handle: int, max_systems: int, params=None, stream=None) -> int:
    """Batch session of up to max_systems systems on one gauge handle."""
    b = ctypes.c_void_p()
    pp = ctypes.byref(params) if params is not None else None
    _check(lib.stg_batch_create(handle, int(max_systems), pp, _stream(stream), ctypes.byref(b)),
           "stg_batch_create")
    return b.value


def stg_batch_destroy(batch: int) -> None:
    lib.stg_batch_destroy(batch)


def stg_batch_add(batch: int, src_dev, x_dev, mass: float, tol: float) -> int:
    slot = ctypes.c_int()
    _check(lib.stg_batch_add(batch, _ptr(src_dev), _ptr(x_dev), float(mass), float(tol),
                             ctypes.byref(slot)), "stg_batch_add")
    return slot.value


def stg_batch_step(batch: int, max_done: int = 64):
    """One chunk for every system of the session; returns ([(slot, status,
    stats), ...] for finished systems, systems still present)."""
    slots = (ctypes.c_int * max(1, max_done))()
    status = (ctypes.c_int * max(1, max_done))()
    stats = (stg_cg_stats * max(1, max_done))()
    n_done, n_act = ctypes.c_int(), ctypes.c_int()
    _check(lib.stg_batch_step(batch, int(max_done), slots, status, stats, ctypes.byref(n_done),
                              ctypes.byref(n_act)), "stg_batch_step")
    return ([(slots[k], status[k], stats[k].as_dict()) for k in range(n_done.value)], n_act.value)


def stg_lgroup_create(max_systems: int, max_vh: int, sloppy: int, recon: int = 12, params=None,
                      stream=None) -> int:
    """Lattice-group session: systems on different lattices in lock-step."""
    b = ctypes.c_void_p()
    pp = ctypes.byref(params) if params is not None else None
    _check(lib.stg_lgroup_create(int(max_systems), int(max_vh), int(sloppy), int(recon), pp,
                                 _stream(stream), ctypes.byref(b)), "stg_lgroup_create")
    return b.value


def stg_lgroup_destroy(group: int) -> None:
    lib.stg_lgroup_destroy(group)


def stg_lgroup_add(group: int, handle: int, src_dev, x_dev, mass: float, tol: float) -> int:
    slot = ctypes.c_int()
    _check(lib.stg_lgroup_add(group, handle, _ptr(src_dev), _ptr(x_dev), float(mass), float(tol),
                              ctypes.byref(slot)), "stg_lgroup_add")
    return slot.value


def stg_lgroup_step(group: int, max_done: int = 16):
    """One chunk for every system of the group; returns ([(slot, status,
    stats), ...] for finished systems, systems still present)."""
    slots = (ctypes.c_int * max(1, max_done))()
    status = (ctypes.c_int * max(1, max_done))()
    stats = (stg_cg_stats * max(1, max_done))()
    n_done, n_act = ctypes.c_int(), ctypes.c_int()
    _check(lib.stg_lgroup_step(group, int(max_done), slots, status, stats, ctypes.byref(n_done),
                               ctypes.byref(n_act)), "stg_lgroup_step")
    return ([(slots[k], status[k], stats[k].as_dict()) for k in range(n_done.value)], n_act.value)


def stg_lgroup_bytes(max_systems: int, max_vh: int, sloppy: int) -> int:
    return int(lib.stg_lgroup_bytes(int(max_systems), int(max_vh), int(sloppy)))


STG_SLAB_COPY, STG_SLAB_DIRECT, STG_SLAB_SLOTS = 0, 1, 6


def stg_slabs_create(dims, links_host: np.ndarray, nslabs: int, prec: int = STG_FP64,
                     recon: int = 18, stream=None) -> int:
    """t-slab decomposition of the lattice into nslabs slabs on the current
    device; canonical complex128 links as for stg_gauge_create (host)."""
    dd = (ctypes.c_int * 4)(*[int(v) for v in dims])
    links = np.ascontiguousarray(links_host, dtype=np.complex128)
    lx, ly, lz, lt = (int(v) for v in dims)
    if links.size != lx * ly * lz * lt * 4 * 9:
        raise ValueError("links_host must hold Lt*Lz*Ly*Lx*4*3*3 complex entries")
    h = ctypes.c_void_p()
    _check(lib.stg_slabs_create(dd, links.ctypes.data, int(nslabs), int(prec), int(recon),
                                _stream(stream), ctypes.byref(h)), "stg_slabs_create")
    return h.value


def stg_slabs_destroy(h: int) -> None:
    lib.stg_slabs_destroy(h)


def stg_slabs_set_exchange(h: int, mode: int, overlap: int) -> None:
    _check(lib.stg_slabs_set_exchange(h, int(mode), int(overlap)), "stg_slabs_set_exchange")


def stg_slabs_load(h: int, slot: int, canon_dev, stream=None) -> None:
    _check(lib.stg_slabs_load(h, int(slot), _ptr(canon_dev), _stream(stream)), "stg_slabs_load")


def stg_slabs_store(h: int, slot: int, canon_dev, stream=None) -> None:
    _check(lib.stg_slabs_store(h, int(slot), _ptr(canon_dev), _stream(stream)), "stg_slabs_store")


def stg_slabs_dslash(h: int, out_parity: int, in_slot: int, out_slot: int, stream=None) -> None:
    _check(lib.stg_slabs_dslash(h, int(out_parity), int(in_slot), int(out_slot), _stream(stream)),
           "stg_slabs_dslash")


def stg_slabs_apply_A_dot(h: int, mass: float, in_slot: int, out_slot: int, dot_dev,
                          stream=None) -> None:
    _check(lib.stg_slabs_apply_A_dot(h, float(mass), int(in_slot), int(out_slot), _ptr(dot_dev),
                                     _stream(stream)), "stg_slabs_apply_A_dot")


def stg_slabs_cg_solve(h: int, src_dev, x_dev, mass: float, tol: float, maxiter: int = 0,
                       stream=None) -> dict:
    st = stg_cg_stats()
    rc = lib.stg_slabs_cg_solve(h, _ptr(src_dev), _ptr(x_dev), float(mass), float(tol),
                                int(maxiter), ctypes.byref(st), _stream(stream))
    _check(rc, "stg_slabs_cg_solve", st.as_dict())
    return st.as_dict()


def stg_slabs_profile(h: int, reps: int = 20, stream=None) -> dict:
    ms = (ctypes.c_double * 4)()
    _check(lib.stg_slabs_profile(h, int(reps), ms, _stream(stream)), "stg_slabs_profile")
    return {"collect_ms": ms[0], "exchange_ms": ms[1], "compute_ms": ms[2], "total_ms": ms[3]}


def stg_slabs_bytes(dims, nslabs: int, prec: int, recon: int) -> int:
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    return int(lib.stg_slabs_bytes(d, int(nslabs), int(prec), int(recon)))


def stg_gauge_bytes(dims, sloppy: int, recon: int) -> int:
    """Device bytes a handle with these arguments keeps resident (0: invalid)."""
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    return int(lib.stg_gauge_bytes(d, int(sloppy), int(recon)))


def stg_batch_bytes(handle: int, max_systems: int, sloppy: int) -> int:
    return int(lib.stg_batch_bytes(handle, int(max_systems), int(sloppy)))


def stg_mrhs_tuning(handle: int, prec: int, nrhs: int):
    nb, bs = ctypes.c_int(), ctypes.c_int()
    _check(lib.stg_mrhs_tuning(handle, int(prec), int(nrhs), ctypes.byref(nb), ctypes.byref(bs)),
           "stg_mrhs_tuning")
    return nb.value, bs.value


from .fields import Gauge  # noqa: E402  (convenience layer over the names above)
