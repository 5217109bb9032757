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


def test_plain_c_program_builds_and_links_against_the_library(gsk_lib, tmp_path):
    """The boundary is a C ABI: a C99 program includes include/gsk.h, links
    libgsk.so and calls its host-only entry points (no GPU involved)."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(
        '#include <stdio.h>\n#include <string.h>\n#include "gsk.h"\n'
        "int main(void) {\n"
        "  gsk_opts o;\n  size_t bytes = 0;\n"
        "  gsk_opts_default(&o);\n"
        "  if (o.maxit != 10000 || o.refresh != 3) return 1;\n"
        "  if (gsk_workspace_bytes(1000, 5000, 1, 0, 0, &bytes) != GSK_OK || bytes == 0) return 2;\n"
        "  if (gsk_workspace_bytes(10, 10, 0, 0, 0, &bytes) != GSK_ERR_ARG) return 3;\n"
        "  if (strstr(gsk_version(), \"sm_103a\") == NULL) return 4;\n"
        "  printf(\"%s\\n\", gsk_version());\n  return 0;\n}\n")
    exe = tmp_path / "abi"
    libdir = os.path.dirname(gsk_lib.LIB_PATH)
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-lgsk", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stderr)
    assert "sm_103a" in out.stdout
