"""The ctypes structures of the Python bindings have the layout of the C
structures they stand for: a small C program compiled against the headers
prints every field's offset and each structure's size, and the ctypes
classes must agree field by field (names, order, offsets, sizes).  A field
added to a header but not to its binding (or the other way round) shifts the
arguments the library reads."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _library_structs():
    from paper_1710_08314_gb300 import polarscl as ps
    return "polarscl.h", os.path.join(ROOT, "include"), [
        ("pscl_pruning", ps.pscl_pruning), ("pscl_work_item", ps.pscl_work_item),
        ("pscl_context", ps.pscl_context), ("pscl_server_cfg", ps.pscl_server_cfg),
        ("pscl_request", ps.pscl_request), ("pscl_completion", ps.pscl_completion)]


def _oracle_structs():
    import oracle
    return "polar_oracle.h", os.path.join(ROOT, "oracle"), [
        ("orc_code", oracle._Code), ("orc_pruning", oracle._Pruning), ("orc_stats", oracle.Stats)]


@pytest.mark.parametrize("which", [_library_structs, _oracle_structs])
def test_ctypes_layouts_match_the_headers(which, tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    header, incdir, structs = which()
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{header}"', "int main(void) {"]
    for cname, cls in structs:
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    r = subprocess.run([gcc, "-I", incdir, str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            a, b, v = line.split()
            got[(a, b)] = int(v)
    for cname, cls in structs:
        assert got[(cname, "size")] == C.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
