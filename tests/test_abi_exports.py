"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/dtn.h (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dtn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dtn_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1210_1491_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    import paper_1210_1491_gb300 as pkg
    assert set(pkg.EXPORTS) == set(names)


def test_status_strings_without_gpu():
    import paper_1210_1491_gb300 as pkg
    L = pkg.load()
    assert L.dtn_status_string(0) == b"ok"
    assert L.dtn_status_string(6).startswith(b"unsupported")
    # argument errors are reported synchronously, before any device work
    assert L.dtn_create_geometry(None, None) == 1


def test_invalid_geometry_rejected_on_host():
    import ctypes as C
    import paper_1210_1491_gb300 as pkg
    from paper_1210_1491_gb300.binding import GeometryDesc
    L = pkg.load()
    d = GeometryDesc()
    d.kind = 1
    d.lo[:] = [0, 0, 0]
    d.hi[:] = [1, 0, 1]   # empty box
    h = C.c_void_p()
    assert L.dtn_create_geometry(C.byref(d), C.byref(h)) == 1
    d.kind = 7
    assert L.dtn_create_geometry(C.byref(d), C.byref(h)) == 1
