"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/phfem.h (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "phfem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"PHFEM_API\s+[\w\s\*]+?\b(phfem_\w+)\s*\(", src)))


def test_library_exports_every_declared_entry_point():
    from paper_2401_15557_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 17, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # status strings need no device
    lib.phfem_status_str.restype = ctypes.c_char_p
    assert lib.phfem_status_str(-2) == b"invalid mesh"


def test_binding_declares_every_entry_point():
    from paper_2401_15557_gb300 import phfem as P
    L = P.lib()
    for n in declared_symbols():
        assert getattr(L, n).restype is not None or n.endswith("destroy"), n
        assert hasattr(P, n), f"binding lacks {n}"
