"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/gicpcg.h declares (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gicpcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gic_\w+)\s*\(", src)))


def test_header_declares_entry_points():
    names = _declared()
    assert "gic_pcg" in names and "gic_ic0" in names and len(names) >= 15


def test_library_exports_every_declared_symbol():
    from paper_2412_07127_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_2412_07127_gb300 import gicpcg
    missing = [n for n in _declared() if n not in gicpcg._SIGS]
    assert not missing, missing


def test_status_strings_without_gpu():
    from paper_2412_07127_gb300 import gicpcg
    lib = gicpcg.lib()
    for s in range(-9, 1):
        assert lib.gic_status_string(s)
    n, nnz = gicpcg.fem_hex_sizes(40)
    assert (n, nnz) == (201720, 15548742)


def test_binding_argument_counts_match_header():
    """Every ctypes signature in the binding has as many arguments as the
    header's prototype (a missing or extra argument would shift every later
    one in the call)."""
    from paper_2412_07127_gb300 import gicpcg
    src = open(os.path.join(ROOT, "include", "gicpcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    protos = re.findall(r"\b(gic_\w+)\s*\(([^;{()]*)\)\s*;", src)
    assert len(protos) >= 15
    bad = []
    for name, args in protos:
        a = args.strip()
        count = 0 if a in ("", "void") else a.count(",") + 1
        if name in gicpcg._SIGS and len(gicpcg._SIGS[name][1]) != count:
            bad.append((name, count, len(gicpcg._SIGS[name][1])))
    assert not bad, bad
