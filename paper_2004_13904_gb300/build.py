"""Build libtf.so in-tree with nvcc for sm_103a (no cmake, no torch extension machinery).

Usage: ``python -m paper_2004_13904_gb300.build`` or ``build()`` from Python.  The
translation units are compiled in parallel and linked into
``paper_2004_13904_gb300/_build/libtf.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libtf.so")
SOURCES = ["tf_api.cu", "tf_kernels.cu", "tf_ct_f32.cu", "tf_ct_f64.cu", "tf_irls.cu", "tf_batch.cu",
           "tf_batch_f32.cu", "tf_batch_f64.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(verbose: bool):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
                "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-I", os.path.join(HERE, "..", "include")]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _newer(target: str, deps) -> bool:
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(d) <= t for d in deps)


def build(verbose: bool = False, force: bool = False, checked: bool = False,
          defines=(), tag: str = "") -> str:
    """Compile libtf.so (or, with checked=True, the bounds-checked libtf_checked.so).
    `defines` (e.g. ["TF_CT_V_TWO_PASS=1"]) with a `tag` build a variant libtf_<tag>.so,
    loadable with TF_LIB_PATH, for tuning experiments."""
    os.makedirs(OUT, exist_ok=True)
    if checked:
        tag = "checked"
    lib = os.path.join(OUT, f"libtf_{tag}.so") if tag else LIB
    tag = f"_{tag}" if tag else ""
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "tf.h"))
    if not force and _newer(lib, deps):
        return lib
    cc = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT, os.path.splitext(src)[0] + tag + ".o")
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(verbose)
        if checked:
            cmd.append("-DTF_BOUNDS_CHECK")
        cmd += [f"-D{d}" for d in defines]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(cc))), "lib64")
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC", "-lcublas", "-lcusolver",
                                                      "-Xlinker", f"-rpath={cuda_lib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv, checked="--checked" in sys.argv))
