"""The C-ABI library loads and exports every entry point declared in include/cvetl.h (no GPU:
no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cvetl.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cvetl_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def so():
    import __graft_entry__

    return __graft_entry__._lib_build().build()


def test_header_declares_the_five_etl_calls():
    names = declared()
    for f in ("cvetl_create", "cvetl_extract", "cvetl_transform", "cvetl_load", "cvetl_results"):
        assert f in names


def test_library_exports_every_declared_symbol(so):
    lib = ctypes.CDLL(so)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (cvetl_[a-z_0-9]+)", out))
    assert set(declared()) <= exported


def test_binding_lists_the_exports(so):
    import paper_2305_07454_b300 as P

    assert set(P.EXPORTS) == set(declared())
    assert P.lib.cvetl_version() == 1


def test_create_rejects_bad_config_without_touching_the_gpu(so):
    import paper_2305_07454_b300 as P

    cfg = P.default_config(n_rows=0)
    h = ctypes.c_void_p()
    assert P.lib.cvetl_create(ctypes.byref(cfg), ctypes.byref(h)) == P.EINVAL
    assert b"positive" in P.lib.cvetl_last_error(None)
    cfg = P.default_config(n_rows=100000, n_cols=100000)
    assert P.lib.cvetl_create(ctypes.byref(cfg), ctypes.byref(h)) == P.EINVAL
    cfg = P.default_config(precision=7)
    assert P.lib.cvetl_create(ctypes.byref(cfg), ctypes.byref(h)) == P.EINVAL
    assert P.lib.cvetl_transform(None) == P.EINVAL
    assert P.lib.cvetl_destroy(None) == P.OK


def test_server_rejects_bad_slot_counts_without_touching_the_gpu(so):
    import ctypes

    import paper_2305_07454_b300 as P

    for n in (0, -1, P.SERVE_MAX_SLOTS + 1):
        cfg = P.ServerConfig(n_slots=n, device=0, mem_budget_bytes=0)
        h = ctypes.c_void_p()
        assert P.lib.cvetl_server_create(ctypes.byref(cfg), ctypes.byref(h)) == P.EINVAL
        assert b"n_slots" in P.lib.cvetl_server_last_error(None)
        assert not h.value
