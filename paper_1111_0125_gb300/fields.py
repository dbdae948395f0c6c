"""Convenience layer: a gauge handle plus torch-allocated device fields.

Only argument marshalling: every method calls one C entry point of
``include/stg.h`` through the same-named binding in ``__init__``.
"""
from __future__ import annotations

import torch

from . import (FIELD_SITE_BYTES, STG_FP32, stg_apply_A, stg_apply_A_dot, stg_cg_params_default,
               stg_cg_solve, stg_dslash, stg_field_bytes, stg_gauge_create, stg_gauge_destroy,
               stg_gauge_dims, stg_pack_field, stg_unpack_field)


class Gauge:
    """Owns one ``stg_gauge`` handle on the current CUDA device."""

    def __init__(self, dims, links_host, sloppy: int = STG_FP32, recon: int = 18, stream=None):
        self.handle = stg_gauge_create(dims, links_host, sloppy, recon, stream)
        self.dims, self.vh = stg_gauge_dims(self.handle)
        self.sloppy = sloppy
        self.recon = recon
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "handle", None):
            stg_gauge_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- fields -----------------------------------------------------------
    def new_field(self, prec: int) -> torch.Tensor:
        n = stg_field_bytes(self.handle, prec)
        assert n == self.vh * FIELD_SITE_BYTES[prec]
        return torch.empty(n, dtype=torch.uint8, device=self.device)

    def pack(self, canon: torch.Tensor, prec: int, stream=None) -> torch.Tensor:
        canon = canon.to(self.device, torch.complex128).contiguous()
        assert canon.shape == (self.vh, 3)
        out = self.new_field(prec)
        stg_pack_field(self.handle, prec, canon, out, stream)
        return out

    def unpack(self, field: torch.Tensor, prec: int, stream=None) -> torch.Tensor:
        out = torch.empty((self.vh, 3), dtype=torch.complex128, device=self.device)
        stg_unpack_field(self.handle, prec, field, out, stream)
        return out

    # -- operators --------------------------------------------------------
    def dslash(self, field: torch.Tensor, out_parity: int, prec: int, out=None, stream=None):
        out = self.new_field(prec) if out is None else out
        stg_dslash(self.handle, out_parity, field, out, prec, stream)
        return out

    def apply_A(self, field: torch.Tensor, mass: float, prec: int, out=None, stream=None):
        out = self.new_field(prec) if out is None else out
        stg_apply_A(self.handle, mass, field, out, prec, stream)
        return out

    def apply_A_dot(self, field: torch.Tensor, mass: float, prec: int, stream=None):
        out = self.new_field(prec)
        dot = torch.empty(1, dtype=torch.float64, device=self.device)
        stg_apply_A_dot(self.handle, mass, field, out, dot, prec, stream)
        return out, dot

    # -- solver -----------------------------------------------------------
    def params(self, **kw):
        p = stg_cg_params_default(self.handle)
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    def cg_solve(self, b: torch.Tensor, mass: float, tol: float, params=None, x0=None,
                 stream=None):
        b = b.to(self.device, torch.complex128).contiguous()
        x = torch.zeros_like(b) if x0 is None else x0.to(self.device, torch.complex128).clone()
        stats = stg_cg_solve(self.handle, b, x, mass, tol, params, stream)
        return x, stats
