"""Builds libnfs.so in-tree (paper_1402_6297_gb300/_lib/) with nvcc for sm_103a.

Translation units compile in parallel; the library is relinked only when a
source or header is newer than it.  No CMake, no torch extension machinery.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIBNAME = "libnfs.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["nfs_api.cu", "matvec_f32.cu", "matvec_f64.cu", "matvec_df.cu", "noalloc.cu", "host_eig.cpp", "host_zeig.cpp", "krylov.cpp", "nfsep.cu"]


def nvcc_path():
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def lib_path():
    return os.path.join(LIBDIR, LIBNAME)


def _newest_input():
    files = glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(ROOT, "include", "*.h")) + [__file__]
    return max(os.path.getmtime(f) for f in files)


def up_to_date():
    lp = lib_path()
    return os.path.exists(lp) and os.path.getmtime(lp) >= _newest_input()


def build(force=False, verbose=False, libdir=None, defines=()):
    """Compile and link libnfs.so into libdir (default: the package's _lib).
    defines: extra NAME=VALUE preprocessor settings (kernel tuning knobs)."""
    out_dir = libdir or LIBDIR
    out_lib = os.path.join(out_dir, LIBNAME)
    if not force and not defines and libdir is None and up_to_date():
        return out_lib
    os.makedirs(out_dir, exist_ok=True)
    nvcc = nvcc_path()
    common = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")] + ARCH
    common += [f"-D{d}" for d in defines]
    objs = []

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = out_lib + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out_lib)
    return out_lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
