"""Builds the CUDA libraries in-tree for sm_103a with nvcc.

libspgemm.so computes in double, libspgemm_f32.so (the same sources with SPGEMM_FLOAT
defined: the same C ABI with float values) in single precision.  Each .cu translation
unit of both is compiled in parallel, then linked into one shared object each under
paper_1504_05022_gb300/_build/.  No CMake, no torch extension machinery: the libraries
are a plain C ABI (include/spgemm.h)."""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libspgemm.so")
LIB_F32 = os.path.join(BUILD, "libspgemm_f32.so")
LIB_CHECK = os.path.join(BUILD, "check", "libspgemm_check.so")
# variant -> (library, object directory, extra nvcc flags); "check" is the bounds-checked
# double-precision build (SPGEMM_CHECK), made only on request
VARIANTS = {"f64": (LIB, BUILD, []), "f32": (LIB_F32, os.path.join(BUILD, "f32"), ["-DSPGEMM_FLOAT"]),
            "check": (LIB_CHECK, os.path.join(BUILD, "check"), ["-DSPGEMM_CHECK"])}

SOURCES = ["stage12.cu", "heap.cu", "esc.cu", "merge.cu", "merge_bm.cu", "dense.cu", "merge_micro.cu", "arrange.cu", "predictor.cu", "replay.cu", "batched.cu",
           "spgemm_api.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libspgemm.so")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                   "-I", INCLUDE, "-I", CSRC] + list(extra)


def _digest() -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(INCLUDE, "spgemm.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(_flags() + SOURCES).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra_flags=(), variants=("f64", "f32")) -> str:
    """Compile and link the libraries of `variants` (both precisions by default) where a
    source changed; returns the first variant's library path."""
    nvcc = _nvcc()
    todo = []
    for name in variants:
        lib, odir, vflags = VARIANTS[name]
        os.makedirs(odir, exist_ok=True)
        stamp = os.path.join(odir, "stamp.txt" if name != "f32" else "stamp_f32.txt")
        dig = _digest() + repr(tuple(extra_flags) + tuple(vflags))
        if not force and os.path.exists(lib) and os.path.exists(stamp):
            with open(stamp) as f:
                if f.read() == dig:
                    continue
        todo.append((lib, odir, _flags(list(extra_flags) + vflags), stamp, dig))
    if not todo:
        return VARIANTS[variants[0]][0]

    def compile_one(job):
        src, odir, flags = job
        obj = os.path.join(odir, src.replace(".cu", ".o"))
        cmd = [nvcc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    jobs = [(src, odir, flags) for (_, odir, flags, _, _) in todo for src in SOURCES]
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, jobs))
    for k, (lib, odir, flags, stamp, dig) in enumerate(todo):
        mine = objs[k * len(SOURCES):(k + 1) * len(SOURCES)]
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + mine + ["-Xlinker", "--no-undefined"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
        with open(stamp, "w") as f:
            f.write(dig)
    return VARIANTS[variants[0]][0]


def build_check(force: bool = False) -> str:
    """The bounds-checked double-precision library (SPGEMM_CHECK); returns its path."""
    return build(force=force, variants=("check",))


if __name__ == "__main__":
    print(build(force=True, verbose=True))
