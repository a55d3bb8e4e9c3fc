"""Build liblb.so (the C-ABI CUDA library) in-tree with nvcc for sm_103a.

Each ``csrc/*.cu`` file is compiled to an object in parallel and the objects
are linked into ``paper_1405_6162_gb300/_build/liblb.so`` (CUDA runtime linked
statically, so the library needs only the driver).  ``-Xptxas -v`` output
(registers, spills, shared memory per kernel) is kept in
``_build/ptxas.log``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblb")


def library_path() -> str:
    return LIB


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(INCLUDE, "lb.h")]


def _manifest() -> str:
    """The set of dependency files (a removed or added file forces a rebuild)."""
    return "\n".join(os.path.basename(d) for d in sorted(_deps())) + "\n"


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    try:
        with open(os.path.join(OUT_DIR, "manifest.txt")) as fh:
            if fh.read() != _manifest():
                return False
    except OSError:
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), out_dir=None) -> str:
    """Compile and link liblb.so; returns its path.

    ``extra_flags`` / ``out_dir`` build a variant elsewhere (e.g. with a -D
    tuning macro) without touching the default library."""
    OUT = out_dir or OUT_DIR
    lib_path = os.path.join(OUT, "liblb.so")
    if not force and out_dir is None and not extra_flags and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    srcs = _sources()

    def compile_one(src):
        obj = os.path.join(OUT, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        results = list(ex.map(compile_one, srcs))
    with open(os.path.join(OUT, "ptxas.log"), "w") as fh:
        for obj, log in results:
            fh.write(f"== {os.path.basename(obj)}\n{log}\n")
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    with open(os.path.join(OUT, "manifest.txt"), "w") as fh:
        fh.write(_manifest())
    if verbose:
        print(open(os.path.join(OUT, "ptxas.log")).read())
    return lib_path


if __name__ == "__main__":
    print(build(force=True, verbose=True))
