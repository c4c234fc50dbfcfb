"""CPU-side checks of the boundary: the library builds, loads, and exports
every function include/polarscl.h declares (no GPU call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "polarscl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pscl_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["pscl_create_code", "pscl_destroy_code", "pscl_decode", "pscl_encode", "pscl_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1710_08314_gb300 import polarscl
    lib = polarscl.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert polarscl.pscl_version().startswith("polarscl")


def test_oracle_is_not_linked_into_the_library():
    from paper_1710_08314_gb300 import build
    so = build.build()
    data = open(so, "rb").read()
    assert b"orc_decode" not in data and b"orc_crc" not in data


def test_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1710_08314_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "polar_oracle" not in txt, f
