"""Build libosog.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked into a shared
library next to this file.  Run as ``python -m paper_2606_21381_gb300.build``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import tempfile
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libosog.so")
SOURCES = ("osog_api.cu", "osog_bin.cu", "osog_render.cu", "osog_backward.cu",
           "osog_noalloc.cu", "osog_cnn.cu", "osog_noise.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE,
         "--expt-relaxed-constexpr"]

_lock = threading.Lock()


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if os.path.exists(cand):
        return cand
    found = shutil.which("nvcc")
    if not found:
        raise RuntimeError("nvcc not found")
    return os.path.realpath(found)


def _inputs() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)
             if f.endswith((".cu", ".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "osog.h"))
    files.append(os.path.join(INCLUDE, "osog_cnn.h"))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libosog.so unless it is newer than every source."""
    with _lock:
        if not force and up_to_date():
            return LIB
        nvcc = _nvcc()
        with tempfile.TemporaryDirectory(prefix="osog_build_") as tmp:
            procs = []
            for src in SOURCES:
                obj = os.path.join(tmp, src.replace(".cu", ".o"))
                cmd = [nvcc, *FLAGS, *ARCH, "-c", os.path.join(CSRC, src), "-o", obj]
                if verbose:
                    cmd.insert(1, "-Xptxas=-v")
                procs.append((src, obj, subprocess.Popen(
                    cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
            objs = []
            for src, obj, p in procs:
                out, _ = p.communicate()
                if verbose or p.returncode:
                    sys.stderr.write(out)
                if p.returncode:
                    raise RuntimeError(f"nvcc failed on {src}")
                objs.append(obj)
            tmp_lib = os.path.join(tmp, "libosog.so")
            cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
            subprocess.check_call([nvcc, *ARCH, "-shared", "-cudart", "shared",
                                   "-Xlinker", "-rpath," + cuda_lib, *objs, "-o", tmp_lib])
            _install(tmp_lib)
    return LIB


def _install(tmp_lib: str) -> None:
    staged = LIB + f".tmp{os.getpid()}"
    with open(tmp_lib, "rb") as src, open(staged, "wb") as dst:
        dst.write(src.read())
    os.replace(staged, LIB)


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
