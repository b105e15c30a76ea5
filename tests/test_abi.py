"""The C ABI library loads, exports every declared symbol, and validates arguments on the host (no GPU)."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "o3g.h")


@pytest.fixture(scope="module")
def L():
    from paper_1801_09847_gb300 import build, o3g
    build.build()
    return o3g.lib()


def declared_symbols():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"O3G_API\s+[\w\s\*]+?\b(o3g_\w+)\s*\(", txt)))


def test_header_declares_the_paper_calls():
    names = declared_symbols()
    for required in ["o3g_build_grid", "o3g_estimate_normals", "o3g_icp_point_to_plane", "o3g_free_grid",
                     "o3g_last_error", "o3g_correspondences", "o3g_normal_equations", "o3g_knn_hybrid",
                     "o3g_icp_point_to_plane_grid", "o3g_register_point_to_plane_host"]:
        assert required in names


def test_library_exports_every_declared_symbol(L):
    from paper_1801_09847_gb300 import o3g
    lib = ctypes.CDLL(o3g.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(declared_symbols()) <= set(o3g._SIGNATURES)


def test_abi_version(L):
    assert L.o3g_abi_version() == 1


def test_build_grid_rejects_bad_arguments(L):
    from paper_1801_09847_gb300 import o3g
    h = ctypes.c_void_p()
    assert L.o3g_build_grid(None, 10, 3, 0.1, None, ctypes.byref(h)) == o3g.ERR_ARG
    assert L.o3g_build_grid(ctypes.c_void_p(16), -1, 3, 0.1, None, ctypes.byref(h)) == o3g.ERR_ARG
    assert L.o3g_build_grid(ctypes.c_void_p(16), 10, 2, 0.1, None, ctypes.byref(h)) == o3g.ERR_ARG
    assert L.o3g_build_grid(ctypes.c_void_p(16), 10, 3, 0.0, None, ctypes.byref(h)) == o3g.ERR_ARG
    assert L.o3g_build_grid(ctypes.c_void_p(16), 10, 3, float("nan"), None, ctypes.byref(h)) == o3g.ERR_ARG
    assert L.o3g_build_grid(ctypes.c_void_p(16), 10, 3, 0.1, None, None) == o3g.ERR_ARG
    assert "invalid" in o3g.last_error() or "null" in o3g.last_error()


def test_normals_must_match_points(L):
    """Sec. 3.1: normals are valid only with as many records as the points."""
    from paper_1801_09847_gb300 import o3g
    T = np.eye(4).ravel()
    out = np.zeros(16)
    f, r = ctypes.c_double(), ctypes.c_double()
    dp = ctypes.c_void_p(256)  # never dereferenced: the count check comes first
    st = L.o3g_icp_point_to_plane(dp, 10, 3, dp, 20, 3, dp, 19, 3, T.ctypes.data_as(o3g._f64p), 0.05, 10,
                                  out.ctypes.data_as(o3g._f64p), ctypes.byref(f), ctypes.byref(r))
    assert st == o3g.ERR_ARG
    assert "match" in o3g.last_error()
    assert L.o3g_grid_set_normals(None, dp, 5, 3, None) == o3g.ERR_ARG


def test_null_handles_are_rejected(L):
    from paper_1801_09847_gb300 import o3g
    T = np.eye(4).ravel()
    assert L.o3g_free_grid(None) == o3g.OK
    assert L.o3g_grid_info(None, None, None) == o3g.ERR_ARG
    assert L.o3g_correspondences(None, None, 0, 3, T.ctypes.data_as(o3g._f64p), 0.1, None, None, None) == o3g.ERR_ARG
    assert L.o3g_knn_hybrid(None, None, 0, 3, 0.1, 30, None, None, None, None, None) == o3g.ERR_ARG
    assert L.o3g_estimate_normals(None, 0.1, 30, None, None, 3, None) == o3g.ERR_ARG


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1801_09847_gb300 import o3g
    monkeypatch.setattr(o3g, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(o3g, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        o3g.lib()


def test_server_request_bytes_is_host_only_and_monotone(L):
    """The server's admission estimate needs no device: positive, growing with either cloud, -1 for bad sizes."""
    from paper_1801_09847_gb300 import o3g
    L.o3g_server_request_bytes.restype = ctypes.c_int64
    L.o3g_server_request_bytes.argtypes = [ctypes.c_int64, ctypes.c_int64]
    base = L.o3g_server_request_bytes(1000, 2000)
    assert base > 0
    assert L.o3g_server_request_bytes(5000, 2000) > base and L.o3g_server_request_bytes(1000, 9000) > base
    assert L.o3g_server_request_bytes(0, 0) > 0
    assert L.o3g_server_request_bytes(-1, 10) == -1 and L.o3g_server_request_bytes(10, -1) == -1
    assert o3g.Server.request_bytes(1000, 2000) == base
