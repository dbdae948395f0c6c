"""The C ABI library loads and exports every entry point declared in
include/*.h; host-side argument checks that need no GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(stg_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def stg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1111_0125_gb300 as m
    return m


def test_header_declares_the_entry_points():
    names = _declared()
    for want in ("stg_dslash", "stg_apply_A", "stg_cg_solve", "stg_gauge_create",
                 "stg_gauge_destroy", "stg_pack_field", "stg_unpack_field"):
        assert want in names


def test_every_declared_symbol_is_exported(stg):
    lib = ctypes.CDLL(stg.LIB_PATH)
    for name in sorted(_declared()):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
        assert hasattr(stg, name), f"{name} has no same-named Python binding"


def test_library_is_built_for_sm_103a(stg):
    import __graft_entry__
    assert "arch=compute_103a,code=sm_103a" in __graft_entry__._build_module().ARCH


def test_status_strings_and_version(stg):
    assert stg.stg_version() >= 1
    assert stg.stg_status_string(stg.STG_OK) == "ok"
    assert "converged" in stg.stg_status_string(stg.STG_ERR_NOT_CONVERGED)
    assert stg.stg_status_string(999) == "unknown status"


def test_host_side_argument_checks(stg):
    # rejected before any CUDA call
    for dims in [(4, 4, 3, 4), (0, 4, 4, 4), (4, -2, 4, 4)]:
        lx, ly, lz, lt = (abs(d) for d in dims)
        links = np.zeros((max(lt, 1), max(lz, 1), max(ly, 1), max(lx, 1), 4, 3, 3), complex)
        h = ctypes.c_void_p()
        d = np.asarray(dims, np.int32)
        st = stg.lib.stg_gauge_create(d.ctypes.data, links.ctypes.data, 1, 18, 0, ctypes.byref(h))
        assert st == stg.STG_ERR_DIMS
        assert "even" in stg.stg_last_error()
    d = np.asarray((4, 4, 4, 4), np.int32)
    h = ctypes.c_void_p()
    assert stg.lib.stg_gauge_create(d.ctypes.data, None, 1, 18, 0, ctypes.byref(h)) == \
        stg.STG_ERR_INVALID_ARG
    links = np.zeros((4, 4, 4, 4, 4, 3, 3), complex)
    assert stg.lib.stg_gauge_create(d.ctypes.data, links.ctypes.data, 1, 16, 0,
                                    ctypes.byref(h)) == stg.STG_ERR_INVALID_ARG
    assert stg.lib.stg_dslash(None, 0, 1, 2, 1, 0) == stg.STG_ERR_INVALID_ARG
    assert stg.lib.stg_cg_solve(None, 1, 2, 0.1, 1e-10, None, None, 0) == \
        stg.STG_ERR_INVALID_ARG
    p = stg.stg_cg_params()
    assert stg.lib.stg_cg_params_default(None, ctypes.byref(p)) == stg.STG_OK
    assert p.policy == stg.STG_CG_RELIABLE and p.delta == 0.1
    assert stg.lib.stg_gauge_destroy(None) == stg.STG_OK


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1111_0125_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "stg_oracle" not in text and "liboracle" not in text, f


def test_gauge_bytes_counts_every_link_copy(stg, monkeypatch):
    """Resident bytes of a handle (host arithmetic, no GPU): FP64/18 links,
    the sloppy links, and the tile-major copies of 12-real sloppy links (64-
    site tiles for the multi-system kernel; 1024-site tiles of four 48 KB
    stages for the single-system FX16 kernel)."""
    def a256(n):
        return (n + 255) // 256 * 256

    dims = (24, 24, 24, 48)
    vh = 24 * 24 * 24 * 48 // 2
    hi = 8 * a256(vh * 144)
    assert stg.stg_gauge_bytes(dims, stg.STG_FP64, 18) == hi
    assert stg.stg_gauge_bytes(dims, stg.STG_FP64, 12) == 8 * a256(vh * 96)
    mt32 = 2 * (-(-vh // 64)) * 64 * 8 * 48
    assert stg.stg_gauge_bytes(dims, stg.STG_FP32, 12) == hi + 8 * a256(vh * 48) + mt32
    assert stg.stg_gauge_bytes(dims, stg.STG_FP32, 18) == hi + 8 * a256(vh * 72)
    fx = 2 * (-(-vh // 1024)) * 4 * 1024 * 48
    mtx = 2 * (-(-vh // 64)) * 64 * 8 * 24
    assert stg.stg_gauge_bytes(dims, stg.STG_FX16, 12) == hi + 8 * a256(vh * 24) + fx + mtx
    monkeypatch.setenv("STG_FX16_TILED", "0")
    monkeypatch.setenv("STG_MRHS_TILED", "0")
    assert stg.stg_gauge_bytes(dims, stg.STG_FX16, 12) == hi + 8 * a256(vh * 24)
    assert stg.stg_gauge_bytes((4, 4, 3, 4), stg.STG_FP32, 12) == 0
    assert stg.stg_gauge_bytes(dims, stg.STG_FP32, 10) == 0


def test_group_launch_argument_checks(stg):
    """stg_dslash_group rejects an empty or oversized group and NULL
    handles before any CUDA call."""
    for n in (0, 17):
        with pytest.raises(stg.StgError) as e:
            stg.stg_dslash_group([0] * n, [0] * n, [0] * n, [0] * n, stg.STG_FP32, stream=0)
        assert e.value.status == stg.STG_ERR_INVALID_ARG
    with pytest.raises(stg.StgError) as e:
        stg.stg_dslash_group([0], [0], [16], [32], stg.STG_FP32, stream=0)
    assert e.value.status == stg.STG_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        stg.stg_dslash_group([0, 0], [0], [0], [0], stg.STG_FP32, stream=0)


def test_lattice_group_host_checks(stg):
    # rejected before any CUDA call
    assert stg.stg_lgroup_bytes(0, 128, stg.STG_FP32) == 0
    assert stg.stg_lgroup_bytes(17, 128, stg.STG_FP32) == 0
    for n, vh, recon in [(0, 128, 12), (17, 128, 12), (4, 0, 12), (4, 128, 10)]:
        with pytest.raises(stg.StgError) as e:
            stg.stg_lgroup_create(n, vh, stg.STG_FP32, recon, stream=0)
        assert e.value.status == stg.STG_ERR_INVALID_ARG
    with pytest.raises(stg.StgError) as e:
        stg.stg_lgroup_create(4, 128, 9, 12, stream=0)
    assert e.value.status == stg.STG_ERR_INVALID_ARG


def test_slab_decomposition_host_checks(stg):
    # rejected before any CUDA call
    U = np.zeros(4 * 4 * 4 * 8 * 36, dtype=np.complex128)
    for nslabs in (0, 3, 8, 65):  # 3 does not divide 8; 8 slabs would be one slice thick
        with pytest.raises(stg.StgError) as e:
            stg.stg_slabs_create((4, 4, 4, 8), U, nslabs, stg.STG_FP64, 18, stream=0)
        assert e.value.status == stg.STG_ERR_DIMS
    for prec, recon in [(9, 18), (stg.STG_FP64, 10)]:
        with pytest.raises(stg.StgError) as e:
            stg.stg_slabs_create((4, 4, 4, 8), U, 2, prec, recon, stream=0)
        assert e.value.status == stg.STG_ERR_INVALID_ARG
    assert stg.stg_slabs_bytes((4, 4, 4, 8), 3, stg.STG_FP64, 18) == 0
    assert stg.stg_slabs_bytes((4, 4, 4, 8), 8, stg.STG_FP64, 18) == 0
    # links, ghost links, six field slots, four faces per slab: the byte count
    # grows with the slab count only through the per-slab face and ghost terms
    one = stg.stg_slabs_bytes((8, 8, 8, 16), 1, stg.STG_FP64, 18)
    four = stg.stg_slabs_bytes((8, 8, 8, 16), 4, stg.STG_FP64, 18)
    vh = 8 * 8 * 8 * 16 // 2
    assert one >= vh * (8 * 144 + 6 * 48)
    assert four > one
    assert four - one < 4 * 2 * (256 * 144 + 4 * 256 * 48) + 8 * 4096
