"""Byte and flop model of the staggered Dslash (host-side bookkeeping).

Two models per output site of one half-pass:

* the paper's (Sec. 2, after Eq. 5): every one of the 8 SU(3) x colour-vector
  products loads its link and its neighbour vector, plus one output vector:
  8 L + 8 S + S bytes.  In FP64 with 18-real links: 8*144 + 8*48 + 48 = 1584 B.
  Flops: 8 products x 9 complex multiply-adds x 8 real flops = 576.
* the compulsory one used for the HBM roofline: each link once, the input
  field once (the other seven neighbour reads are cache hits), the output
  once: 8 L + 2 S (+ one S per extra streamed field of a fused epilogue).
"""
from __future__ import annotations

LINK_BYTES = {("f64", 18): 144, ("f64", 12): 96, ("f32", 18): 72, ("f32", 12): 48,
              ("f16", 18): 36, ("f16", 12): 24, ("fx16", 18): 36, ("fx16", 12): 24,
              ("bf16", 18): 36, ("bf16", 12): 24}
FIELD_BYTES = {"f64": 48, "f32": 24, "f16": 16, "fx16": 16, "bf16": 16}

FLOPS_PER_SITE = 8 * 9 * 8          # 576
A_FLOPS_PER_SITE = 2 * FLOPS_PER_SITE + 12


def paper_bytes_per_site(prec: str = "f64", recon: int = 18) -> int:
    L, S = LINK_BYTES[(prec, recon)], FIELD_BYTES[prec]
    return 8 * L + 8 * S + S


def compulsory_bytes_per_site(prec: str, recon: int, extra_fields: int = 0) -> int:
    L, S = LINK_BYTES[(prec, recon)], FIELD_BYTES[prec]
    return 8 * L + (2 + extra_fields) * S


def even_sites(dims) -> int:
    lx, ly, lz, lt = dims
    return lx * ly * lz * lt // 2


def dslash_totals(dims, prec: str = "f64", recon: int = 18):
    """(flops, paper-model bytes) of one Dslash over the even sites."""
    n = even_sites(dims)
    return n * FLOPS_PER_SITE, n * paper_bytes_per_site(prec, recon)


def cg_iteration_bytes_per_site(prec: str, recon: int, vec_prec: str | None = None) -> int:
    """Compulsory bytes of one CG iteration (two half-passes, the fused A
    epilogue, the x/r update and the xpay) per even site."""
    L, S = LINK_BYTES[(prec, recon)], FIELD_BYTES[prec]
    R = FIELD_BYTES[vec_prec or prec]
    return 16 * L + 5 * S + (2 * S + 4 * R) + (S + R + S)
