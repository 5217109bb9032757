"""The C-ABI library loads and exports every symbol include/gsk.h declares
(no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gsk.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "for", "sizeof")))


@pytest.fixture(scope="module")
def gsk_lib():
    from paper_0812_2769_gb300 import build

    build.build()
    import paper_0812_2769_gb300 as g

    return g


def test_header_declares_the_paper_entry_points():
    names = _declared_functions()
    for want in ["gs_scale", "gmres_solve", "bicgstab_solve", "gsk_spmv", "gsk_ctx_create", "gsk_ctx_destroy",
                 "gsk_workspace_bytes", "gsk_last_error", "gsk_opts_default", "gsk_version"]:
        assert want in names


def test_library_exports_every_declared_symbol(gsk_lib):
    lib = ctypes.CDLL(gsk_lib.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(gsk_lib):
    assert set(_declared_functions()) <= set(gsk_lib.SIGNATURES)


def test_host_only_entry_points(gsk_lib):
    assert "sm_103a" in gsk_lib.version()
    o = gsk_lib.opts()
    assert o.maxit == 10000 and o.refresh == 3 and o.metric == gsk_lib.METRIC_GS2
    b = gsk_lib.workspace_bytes(2_097_152, 14_581_760, "gmres", 30)
    assert b > 31 * 2_097_152 * 8
    with pytest.raises(gsk_lib.GskError):
        gsk_lib.workspace_bytes(10, 10, "gmres", 0)


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    import paper_0812_2769_gb300 as g

    monkeypatch.setattr(g, "_lib", None)
    monkeypatch.setattr(g, "LIB_PATH", str(tmp_path / "libgsk.so"))
    with pytest.raises(ImportError, match="no CPU fallback"):
        g.lib()
