"""Host-side checks of the C ABI library (no GPU): it builds for sm_103a, loads,
and exports every entry point include/tbsci.h declares; the binding refuses to
run without it; struct layouts match the header."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tbsci.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:tbsci_status|void|const char\s*\*)\s*(tbsci_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2503_10335_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["tbsci_build_strings", "tbsci_build_excitation_tables", "tbsci_sigma", "tbsci_davidson"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2503_10335_gb300 import _binding
    assert sorted(_binding.EXPORTS) == _declared()


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2503_10335_gb300 import _binding
    with pytest.raises(RuntimeError):
        _binding.load(str(tmp_path / "missing.so"))


def test_entry_layouts():
    from paper_2503_10335_gb300 import _binding as B
    assert ctypes.sizeof(B.SingleLink) == 8
    assert ctypes.sizeof(B.DoubleLink) == 12
    assert ctypes.sizeof(B.SigmaCounts) == 80


def test_product_path_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2503_10335_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert "tbsci_oracle" not in src and "liboracle" not in src, f


def test_binding_struct_layout_matches_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets that
    the C compiler gives the struct of the same name in include/tbsci.h (field
    names must match the header's member names, or the probe does not compile)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2503_10335_gb300 import _binding as B
    pairs = [("tbsci_single_link", B.SingleLink), ("tbsci_double_link", B.DoubleLink),
             ("tbsci_sigma_counts", B.SigmaCounts), ("tbsci_davidson_opts", B.DavidsonOpts),
             ("tbsci_davidson_info", B.DavidsonInfo), ("tbsci_server_opts", B.ServerOpts),
             ("tbsci_request", B.Request), ("tbsci_result", B.Result), ("tbsci_trace_entry", B.TraceEntry),
             ("tbsci_options", B.Options)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tbsci.h"', "int main(void) {"]
    for cname, cls in pairs:
        lines.append('printf("%%zu\\n", sizeof(%s));' % cname)
        for f in cls._fields_:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (cname, f[0]))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    want = []
    for _, cls in pairs:
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, f[0]).offset for f in cls._fields_]
    assert got == want
