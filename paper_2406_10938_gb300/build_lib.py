"""Compile libdetlsh.so (CUDA for sm_103a) in-tree with nvcc.

Each translation unit under csrc/ is compiled in parallel, then linked into
``_lib/libdetlsh.so``. A rebuild happens only when a source or header is newer
than the library (or when forced).
"""

import concurrent.futures
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libdetlsh.so")
# the checked build (device index checks, DETLSH_CHECKED), built on request
LIBDIR_CHECKED = os.path.join(HERE, "_lib_checked")
LIB_CHECKED = os.path.join(LIBDIR_CHECKED, "libdetlsh.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(p) > t for p in deps)


def _compile(src, obj, verbose, defines=()):
    nvcc = _nvcc()
    if src.endswith(".cu"):
        cmd = [nvcc, *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2",
               *[f"-D{d}" for d in defines], "-I", INCLUDE, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
    else:
        # host-only code: no contraction of a*b+c into a fused multiply-add,
        # so that host arithmetic rounds the same way on every CPU
        cmd = [nvcc, "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O2,-ffp-contract=off",
               *[f"-D{d}" for d in defines], "-I", INCLUDE, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build the library if needed and return its path; checked=True builds the
    variant with device index checks (DETLSH_CHECKED) beside it."""
    libdir, lib = (LIBDIR_CHECKED, LIB_CHECKED) if checked else (LIBDIR, LIB)
    defines = ("DETLSH_CHECKED",) if checked else ()
    if not force and not _stale(lib):
        return lib
    objdir = os.path.join(libdir, "obj")
    os.makedirs(objdir, exist_ok=True)
    srcs = _sources()
    objs = [os.path.join(objdir, os.path.basename(s) + ".o") for s in srcs]
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        logs = list(ex.map(lambda so: _compile(so[0], so[1], verbose, defines), zip(srcs, objs)))
    if verbose:
        for s, log in zip(srcs, logs):
            if log.strip():
                print(f"--- {os.path.basename(s)}\n{log}")
    tmp = lib + ".tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
