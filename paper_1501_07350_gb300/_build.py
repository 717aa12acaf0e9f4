"""Builds libopenfft_gb.so in-tree from csrc/ with nvcc for sm_103a.

Each translation unit is compiled in its own nvcc process (in parallel) and
the objects are linked into one shared library next to this file, under
``_build/``.  Nothing is installed outside the repository.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libopenfft_gb.so"
LIB_PATH = os.path.join(OUT_DIR, LIB_NAME)
# the bounds-checked build (-DOPENFFT_CHECKED): same ABI, its own folder and name
CHECKED_DIR = os.path.join(HERE, "_build_checked")
CHECKED_LIB_PATH = os.path.join(CHECKED_DIR, "libopenfft_gb_checked.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["capi.cu", "fft_stage.cu", "redistribute.cu", "fft_tile_f64.cu", "fft_tile_df.cu", "fft_tile_f32.cu", "noalloc.cu", "batch.cu", "mlp.cu", "tcgemm.cu", "dftgemm.cu", "r2c.cu", "dist.cu", "fft_tma_256.cu", "fft_tma_512.cu", "nd.cu", "fft_tma_f32.cu", "fft_warp_mixed.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I" + CSRC, "-I" + INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "openfft_gb.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date(lib: str = LIB_PATH) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra_flags=(), checked: bool = False) -> str:
    """Compile every CUDA source for sm_103a and link the shared library
    (checked=True: the bounds-checked library, compiled with -DOPENFFT_CHECKED)."""
    out_dir, lib_path = (CHECKED_DIR, CHECKED_LIB_PATH) if checked else (OUT_DIR, LIB_PATH)
    if checked:
        extra_flags = ["-DOPENFFT_CHECKED", *extra_flags]
    if not force and up_to_date(lib_path):
        return lib_path
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    objs = []
    cmds = []
    for src in SOURCES:
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmds.append([nvcc, *ARCH, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
        return r.stderr

    with ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        logs = list(ex.map(run, cmds))
    if verbose:
        for lg in logs:
            if lg:
                print(lg, file=sys.stderr)
    tmp = lib_path + ".%d.tmp" % os.getpid()
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv,
                extra_flags=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else []))
