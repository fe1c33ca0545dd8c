"""The C ABI library without a GPU: it builds, loads, exports every entry point
that include/vag.h declares, the ctypes structs match the C layout, and calls
fail with a status code (never a crash) when no device is present."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

import __graft_entry__ as ge

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vag.h")


@pytest.fixture(scope="module")
def vag():
    ge.build()
    import paper_1602_03641_gb300.vag as v
    return v


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vag_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["vag_assemble", "vag_solve", "vag_transport", "vag_ctx_create", "vag_spmv"]:
        assert must in names


def test_library_exports_every_declared_symbol(vag):
    L = vag.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", vag.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (vag_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(L, n)
    assert set(vag.declared_symbols()) <= exported


STRUCTS = ["vag_mesh", "vag_props", "vag_dirichlet", "vag_system_info", "vag_solve_opts", "vag_solve_info",
           "vag_transport_opts", "vag_transport_info", "vag_server_opts", "vag_request", "vag_result",
           "vag_server_stats"]


def test_ctypes_layout_matches_c(vag):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "vag.h"', "int main(void){"]
    for s in STRUCTS:
        cls = getattr(vag, s)
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = dict(l.split() for l in out.strip().splitlines())
    for s in STRUCTS:
        cls = getattr(vag, s)
        assert int(got[s]) == C.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, (s, f)


def test_null_arguments_are_rejected(vag):
    L = vag.lib()
    assert L.vag_ctx_create(0, 0, None) == vag.VAG_EINVAL
    assert L.vag_solve(None, None, None, None) == vag.VAG_EINVAL
    assert L.vag_transport(None, None, None, None) == vag.VAG_EINVAL
    assert L.vag_assemble(None, None, None, None, 0, None) == vag.VAG_EINVAL
    assert L.vag_last_error(None) == b"null context"


def test_without_gpu_context_creation_reports_an_error(vag):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    st = vag.lib().vag_ctx_create(0, 0, C.byref(h))
    assert st in (vag.VAG_ECUDA, vag.VAG_EINVAL)
    assert not h.value


def test_binding_constants_match_the_header(vag):
    """Every VAG_* enumerator of include/vag.h has the same value in the
    binding (status codes, precisions, preconditioners, Krylov methods,
    memory spaces, kernels)."""
    src = ['#include <stdio.h>', '#include "vag.h"', "int main(void){"]
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    names = sorted(set(n for body in re.findall(r"enum\s*\{([^}]*)\}", txt)
                       for n in re.findall(r"\b(VAG_[A-Z0-9_]+)\b", body)))
    assert "VAG_KRYLOV_GMRES" in names and "VAG_PC_CHEBYSHEV" in names
    for n in names:
        src.append(f'printf("{n} %lld\\n", (long long){n});')
    src.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "e.c")
        exe = os.path.join(d, "e")
        open(c, "w").write("\n".join(src))
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    import paper_1602_03641_gb300 as pkg
    for line in out.splitlines():
        n, v = line.split()
        assert hasattr(vag, n) or hasattr(pkg, n), n
        got = getattr(vag, n, getattr(pkg, n, None))
        assert got == int(v), (n, got, v)


def test_binding_fails_loudly_without_the_library(vag, monkeypatch):
    """No fallback: without libvag.so the binding raises instead of computing
    anything another way."""
    monkeypatch.setattr(vag, "_LIB", None)
    monkeypatch.setattr(vag, "LIB_PATH", os.path.join(tempfile.mkdtemp(), "libvag.so"))
    with pytest.raises(RuntimeError, match="missing"):
        vag.lib()


def test_product_never_imports_the_oracle():
    """The package and its kernels share nothing with the oracle: no import of
    it anywhere in the package's sources."""
    pkg = os.path.join(ROOT, "paper_1602_03641_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", txt, flags=re.M), f
                assert "vag_oracle" not in txt, f
