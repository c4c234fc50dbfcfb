"""In-tree build of libpolarscl.so for sm_103a (nvcc, no cmake).

Each .cu translation unit compiles in parallel; the objects link into
paper_1710_08314_gb300/_build/libpolarscl.so.  variant="checked" builds a
copy whose kernels bounds-check every buffer access and record violations in
a debug word instead of touching memory (libpolarscl_checked.so).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
ROOT = os.path.dirname(HERE)
UNITS = ["api.cu", "scl_f32.cu", "scl_i16.cu", "scl_i8.cu", "scl_f32_nodes.cu", "scl_i16_nodes.cu",
         "scl_i8_nodes.cu", "scl_attrs.cu", "encode.cu", "server.cu", "server_nodes.cu",
         "sc_kernel.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def lib_path(variant: str = "release") -> str:
    return os.path.join(OUT, "libpolarscl.so" if variant == "release" else f"libpolarscl_{variant}.so")


def _sources():
    return [os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(ROOT, "include", "polarscl.h")]


def up_to_date(variant: str = "release") -> bool:
    so = lib_path(variant)
    if not os.path.exists(so):
        return False
    t = os.path.getmtime(so)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(variant: str = "release", force: bool = False, verbose: bool = False) -> str:
    so = lib_path(variant)
    if not force and up_to_date(variant):
        return so
    os.makedirs(OUT, exist_ok=True)
    objdir = os.path.join(OUT, f"obj_{variant}")
    os.makedirs(objdir, exist_ok=True)
    flags = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-cudart", "shared", "-Xcompiler", "-fPIC",
             "-I", os.path.join(ROOT, "include")] + ARCH
    if variant == "checked":
        flags.append("-DPSCL_CHECKED")
    elif variant == "opprof":
        flags.append("-DPSCL_OPPROF")
    if verbose:
        flags += ["-Xptxas", "-v"]

    def one(u):
        obj = os.path.join(objdir, u.replace(".cu", ".o"))
        cmd = [nvcc()] + flags + ["-c", os.path.join(SRC, u), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {u}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(one, UNITS))
    if verbose:
        for _, err in results:
            if err:
                print(err)
    tmp = so + f".{os.getpid()}.tmp"
    cudalib = os.path.join(os.path.dirname(os.path.dirname(nvcc())), "lib64")
    cmd = ([nvcc(), "-shared", "-cudart", "shared", "-o", tmp] + [o for o, _ in results] + ARCH
           + ["-Xlinker", "-rpath=" + cudalib])
    subprocess.check_call(cmd)
    os.replace(tmp, so)
    return so


if __name__ == "__main__":
    import sys
    v = sys.argv[1] if len(sys.argv) > 1 else "release"
    print(build(v, force=True, verbose=True))
