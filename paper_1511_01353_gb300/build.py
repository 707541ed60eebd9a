"""Build libfmt.so in-tree with nvcc for sm_103a (GB300).

Each .cu under csrc/ is compiled in parallel, then linked into a shared
library next to this file.  Rebuilds only when a source or header is newer
than the library.  build_checked() makes libfmt_checked.so, the same sources
with -DFMT_CHECKED: every kernel tests the indices it reads from device
memory against the sizes of the buffers they address (include/fmt.h).
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfmt.so")
LIB_CHECKED = os.path.join(HERE, "libfmt_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    return compile_library(LIB, BUILD, verbose=verbose)


def build_checked(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale(LIB_CHECKED):
        return LIB_CHECKED
    return compile_library(LIB_CHECKED, os.path.join(BUILD, "checked"), defines=("FMT_CHECKED",), verbose=verbose)


def compile_library(lib: str, objdir: str, host_flags=(), defines=(), verbose: bool = False) -> str:
    """Compile every csrc/*.cu in parallel into objdir and link them into lib.
    host_flags go to the host compiler of each object and of the link (the
    sanitizer test builds an ASan/UBSan variant this way); defines are
    preprocessor macros of every object (FMT_CHECKED)."""
    xhost = [a for f in host_flags for a in ("-Xcompiler", f)] + ["-D" + d for d in defines]
    os.makedirs(objdir, exist_ok=True)
    procs = []
    objs = []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [NVCC, *ARCH, *FLAGS, *xhost, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
        elif verbose and out:
            sys.stdout.write(out.decode(errors="replace"))
    if failed:
        msg = "\n".join("%s\n%s" % (" ".join(c), o) for c, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", *xhost]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    if "--checked" in sys.argv:
        print(build_checked(force="--force" in sys.argv, verbose=True))
    else:
        print(build(force="--force" in sys.argv, verbose=True))
