"""Build libstemeels.so in-tree for sm_103a (nvcc + the host C++ compiler, no cmake).

Each translation unit is compiled in parallel; the shared object lands in
paper_1908_07628_gb300/_build/.  Rebuilds only when a source or header is newer
than the library.  With check=True (or STEM_CHECK=1 in the environment) the
bounds-checked debug variant is built instead, with -DSTEM_CHECK, into
paper_1908_07628_gb300/_build_check/: its kernels verify the indices they derive from
host lists and report a violation through the device status word instead of touching
the memory (the call then fails with EELS_ERR_CUDA).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def checked_from_env() -> bool:
    return os.environ.get("STEM_CHECK", "") == "1"


def build_dir(check: bool) -> str:
    return os.path.join(PKG, "_build_check" if check else "_build")


def lib_path(check: bool) -> str:
    return os.path.join(build_dir(check), "libstemeels_check.so" if check else "libstemeels.so")


BUILD = build_dir(False)
LIB = lib_path(False)


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or "/usr/local/cuda"
    if not os.path.isdir(home):
        nvcc = shutil.which("nvcc")
        if nvcc:
            home = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return home


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


def _compile(src: str, nvcc: str, cuda: str, check: bool = False) -> str:
    obj = os.path.join(build_dir(check), os.path.basename(src) + ".o")
    defs = ["-DSTEM_CHECK"] if check else []
    if src.endswith(".cu"):
        cmd = [nvcc, "-c", src, "-o", obj, "-O3", "-std=c++17", "-lineinfo", *ARCH, *defs,
               "-Xcompiler", "-fPIC,-ffp-contract=off", "-Xptxas", "-v", "-I", INCLUDE, "-I", CSRC]
    else:
        cxx = os.environ.get("CXX", "g++")
        cmd = [cxx, "-c", src, "-o", obj, "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", *defs,
               "-I", INCLUDE, "-I", CSRC, "-I", os.path.join(cuda, "include")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    with open(obj + ".log", "w") as fh:
        fh.write(r.stdout + r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, check=None) -> str:
    """Compile every CUDA/C++ source of the library for sm_103a and link it (the
    bounds-checked variant if check, or if STEM_CHECK=1 when check is None)."""
    if check is None:
        check = checked_from_env()
    lib_file = lib_path(check)
    os.makedirs(build_dir(check), exist_ok=True)
    if not force and os.path.exists(lib_file):
        t = os.path.getmtime(lib_file)
        if all(os.path.getmtime(p) <= t for p in _deps()):
            return lib_file
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc") or "nvcc"
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, nvcc, cuda, check), srcs))
    tmp = lib_file + ".tmp"
    cmd = [nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_file)
    if verbose:
        for o in objs:
            print(open(o + ".log").read())
    return lib_file


if __name__ == "__main__":
    print(build(force=True, verbose=True))
