"""In-tree build of libpespace_gb300.so for sm_103a (GB300).

Each CUDA translation unit under csrc/ is compiled by its own nvcc process (in parallel), then
linked into paper_2602_12011_gb300/lib/libpespace_gb300.so. No cmake, one -gencode.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libpespace_gb300.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _newest_input() -> float:
    files = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


# The test build: host-side fault injection (PE_FAULT_INJECTION) and the hot kernels' index checks
# (PE_CHECKED), exported through include/pespace_gb300_test.h. Never the product library.
TEST_LIB = os.path.join(LIBDIR, "libpespace_gb300_test.so")
TEST_FLAGS = ["-DPE_FAULT_INJECTION", "-DPE_CHECKED"]


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, variant: str = "product") -> str:
    """Compile every .cu under csrc/ for sm_103a and link the shared library. Returns its path.
    variant "test" builds libpespace_gb300_test.so (fault injection and index checks) instead."""
    lib_path = TEST_LIB if variant == "test" else LIB
    objdir = os.path.join(LIBDIR, "test") if variant == "test" else LIBDIR
    extra = TEST_FLAGS if variant == "test" else []
    if not force and not ptxas_info and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= _newest_input():
        return lib_path
    os.makedirs(objdir, exist_ok=True)
    nvcc = _nvcc()
    objs = []
    cmds = []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        if ptxas_info:
            cmd += ["-Xptxas", "-v"]
        cmds.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=max(1, min(len(cmds), os.cpu_count() or 1))) as ex:
        results = list(ex.map(run, cmds))
    for cmd, r in results:
        if verbose or ptxas_info:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    tmp = lib_path + ".tmp%d" % os.getpid()
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s%s" % (" ".join(link), r.stdout, r.stderr))
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    build(force=True, verbose=True, ptxas_info="-v" in sys.argv)
    print(LIB)
