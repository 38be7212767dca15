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


def _kind_of_c(param):
    """'p' pointer, 'f8'/'f4' floating, 'i8'/'i4' integer, from a C parameter."""
    p = " ".join(param.replace("const", " ").split())
    if "*" in p:
        return "p"
    t = p.rsplit(" ", 1)[0] if " " in p else p
    if t == "double":
        return "f8"
    if t == "float":
        return "f4"
    if t in ("int64_t", "size_t", "uint64_t", "long long"):
        return "i8"
    if t in ("int", "int32_t", "unsigned", "uint32_t"):
        return "i4"
    return "?" + t


def _kind_of_ctypes(t):
    if t is ctypes.c_void_p or t is ctypes.c_char_p or hasattr(t, "_type_") and isinstance(t._type_, type):
        return "p"
    if t in (ctypes.c_double, ctypes.c_float):
        return "f%d" % ctypes.sizeof(t)
    return "i%d" % ctypes.sizeof(t)


def test_binding_argument_kinds_match_header():
    """Each argument's kind and width (pointer, 8- or 4-byte integer, double
    or float) in the binding is the header's, so no value is truncated or
    passed in the wrong register class."""
    from paper_2412_07127_gb300 import gicpcg
    src = open(os.path.join(ROOT, "include", "gicpcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    bad = []
    for name, args in re.findall(r"\b(gic_\w+)\s*\(([^;{()]*)\)\s*;", src):
        a = args.strip()
        if a in ("", "void") or name not in gicpcg._SIGS:
            continue
        want = [_kind_of_c(x) for x in a.split(",")]
        have = [_kind_of_ctypes(t) for t in gicpcg._SIGS[name][1]]
        if want != have:
            bad.append((name, want, have))
    assert not bad, bad
