"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/tdb.h declares.  No GPU calls."""

import ctypes as C
import os
import re

import pytest

from paper_2201_06958_gb300 import build_lib, tdb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tdb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(tdb_[a-z_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return tdb.load()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    assert set(tdb.EXPORTS) <= set(names)


def test_version_and_status_strings(lib):
    assert b"sm_103a" in lib.tdb_version()
    assert lib.tdb_status_string(0) == b"TDB_OK"
    assert lib.tdb_status_string(9) == b"TDB_WARN_RANK_CAP"


def test_workspace_bytes_and_validation(lib):
    cfg, keep = tdb.make_config([512, 256, 12], [0, 0, 0], [16, 16, 12], eps_th=1e-4)
    n = lib.tdb_workspace_bytes(C.byref(cfg))
    assert 10 * 2 ** 20 < n < 2 ** 30
    bad, _ = tdb.make_config([5], [1])
    assert lib.tdb_workspace_bytes(C.byref(bad)) == 0            # ndim 1
    bad, _ = tdb.make_config([5, 4, 3, 2], [1] * 4)
    bad.ndim = 5
    assert lib.tdb_workspace_bytes(C.byref(bad)) == 0            # ndim 5
    bad, _ = tdb.make_config([8, 8], [40, 2])
    assert lib.tdb_workspace_bytes(C.byref(bad)) == 0            # rank > 32
    heun, _ = tdb.make_config([512, 256, 12], [0, 0, 0], [16, 16, 12], eps_th=1e-4, integrator="heun")
    assert lib.tdb_workspace_bytes(C.byref(heun)) == n           # Heun reuses the step's buffers
    heun.integrator = 2
    assert lib.tdb_workspace_bytes(C.byref(heun)) == n           # the midpoint scheme reuses them too
    heun.integrator = 3
    assert lib.tdb_workspace_bytes(C.byref(heun)) == 0           # no such integrator
    # init with a null workspace fails cleanly with TDB_ERR_WORKSPACE, before any device work
    ctx = C.c_void_p()
    st = lib.tdb_init(C.byref(ctx), C.byref(cfg), None, 0, C.c_void_p(16), None)
    assert st == 10
    assert b"workspace" in lib.tdb_last_error(None)
    st = lib.tdb_push_snapshot(None, None, None)
    assert st == 1


def test_long_mode_shape_rules(lib):
    """A mode of more than 1024 points is accepted as the first or the last mode when the
    other modes hold at most 1024 points together (its HOSVD comes from the short side);
    otherwise tdb_workspace_bytes refuses the shape (0).  The long mode's Gram is never
    sized: the paper-size TDB-2 shape (19,076 x 23) needs far less than a 19,076^2 matrix."""
    for dims in ([4, 2000, 4], [2000, 40, 40], [2000, 2000], [1025, 1025]):
        cfg, _ = tdb.make_config(dims, [2] * len(dims), precision="fp64")
        assert lib.tdb_workspace_bytes(C.byref(cfg)) == 0, dims
    for dims in ([2000, 8, 4], [8, 4, 2000], [19076, 23], [1024, 1024]):
        cfg, _ = tdb.make_config(dims, [2] * len(dims), precision="fp64")
        assert lib.tdb_workspace_bytes(C.byref(cfg)) > 0, dims
    cfg, _ = tdb.make_config([19076, 23], [0, 0], [23, 23], precision="fp64")
    assert lib.tdb_workspace_bytes(C.byref(cfg)) < 19076 * 19076 * 8 // 10


def test_struct_layout_matches_header():
    # offsets computed by the C compiler for include/tdb.h (x86-64 and aarch64 agree)
    assert C.sizeof(tdb.tdb_config) == 144
    assert tdb.tdb_config.eps_th.offset == 104
    assert tdb.tdb_config.reorth.offset == 136
    assert C.sizeof(tdb.tdb_step_info) == 160
    assert tdb.tdb_step_info.cr.offset == 120
