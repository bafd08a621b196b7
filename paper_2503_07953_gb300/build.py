"""Build the CUDA library (libmfcgb.so) in-tree for sm_103a with nvcc.

Each translation unit compiles in its own nvcc process (in parallel); the
objects are linked into ``paper_2503_07953_gb300/_build/libmfcgb.so``.
"""
from __future__ import annotations

import hashlib
import os
import re
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmfcgb.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]
SOURCES = ["mfc_api.cu"] + [f"mfc_nf{n}_{m}.cu" for n in (1, 2, 3, 4) for m in ("exact", "fast", "df")]
# The exact-arithmetic kernels follow the defining formulas operation by
# operation: no FMA contraction there.
PER_SOURCE_FLAGS = {src: ["--fmad=false"] for src in SOURCES if src.endswith("_exact.cu")}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _fingerprint() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            p = os.path.join(d, name)
            if os.path.isfile(p):
                h.update(name.encode())
                with open(p, "rb") as fh:
                    h.update(fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS).encode())
    h.update(repr(sorted(PER_SOURCE_FLAGS.items())).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


# The files the forward directional sweep kernels are compiled from.
SWEEP_SOURCES = ["mfc_df64.cuh", "mfc_device.cuh", "mfc_fwd.cuh", "mfc_split.cuh", "mfc_launch.h",
                 "mfc_launch_impl.cuh"] + \
    [f"mfc_nf{n}_{m}.cu" for n in (1, 2, 3, 4) for m in ("exact", "fast", "df")]


def _code_only(text: str) -> str:
    """C++ source without comments, whitespace runs collapsed (the sweep
    sources hold no string literal with a comment marker)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def source_fingerprint() -> str:
    """Hash of the forward sweep kernels' code (comments and layout
    ignored) and flags, no machine: identifies the code an ncu capture of
    those kernels was taken on."""
    h = hashlib.sha256()
    for name in SWEEP_SOURCES:
        h.update(name.encode())
        with open(os.path.join(CSRC, name), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    flags = [f for f in ARCH + NVCC_FLAGS if f not in (INCLUDE, CSRC)]  # no machine paths
    h.update(" ".join(flags).encode())
    h.update(repr(sorted(PER_SOURCE_FLAGS.items())).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile and link; skipped when sources, flags and machine are unchanged."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp")
    fp = _fingerprint() + " ".join(extra_flags)
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read() == fp:
                return LIB
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *NVCC_FLAGS, *PER_SOURCE_FLAGS.get(src, []), *extra_flags, "-c",
               os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(fp)
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=True, verbose=v or bool(extra), extra_flags=extra))
