"""The C ABI from plain C: tests/c_abi/products.c includes only include/tf.h and the CUDA
runtime.  On the CPU it must compile as C99 with warnings as errors and link against
libtf.so.  On a GPU its G x and G^T y must match the Python binding's on the same inputs
(a different caller of the same library: results agree to rounding of the inputs)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "c_abi", "products.c")


def _cuda_home():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _build_caller(tmp_path):
    from paper_2004_13904_gb300 import build
    lib = build.build()
    cuda = _cuda_home()
    exe = str(tmp_path / "products")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cuda, "include"), SRC, "-o", exe,
           "-L", os.path.dirname(lib), "-ltf", "-L", os.path.join(cuda, "lib64"), "-lcudart", "-lm",
           f"-Wl,-rpath,{os.path.dirname(lib)}", f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def test_c_caller_compiles_and_links(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    exe = _build_caller(tmp_path)
    assert os.path.exists(exe)


@pytest.mark.gpu
@pytest.mark.parametrize("dtn", ["f64", "f32"])
def test_c_caller_matches_python_binding(tmp_path, dtn):
    import torch
    from paper_2004_13904_gb300 import Operator
    exe = _build_caller(tmp_path)
    sx, sy, nz, pad = 12, 10, 3, 1
    r = subprocess.run([exe, str(sx), str(sy), str(nz), str(pad), dtn], capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    vals = r.stdout.split()
    m, n = int(vals[0]), int(vals[1])
    out = np.array([float(v) for v in vals[2:]])
    assert out.size == m + n
    g = synth.Grid(sx, sy, nz, pad, pad, pad, pad)
    assert (m, n) == (g.m, g.n)
    dt = torch.float32 if dtn == "f32" else torch.float64
    op = Operator(g, "gravity", dtype=dt)
    x = torch.tensor(np.sin(0.37 * np.arange(n)) + 0.25, dtype=dt, device="cuda")
    y = torch.tensor(np.cos(0.11 * np.arange(m)), dtype=dt, device="cuda")
    d = op.matvec(x).double().cpu().numpy()
    xt = op.rmatvec(y).double().cpu().numpy()
    tol = 1e-12 if dtn == "f64" else 1e-6
    assert np.linalg.norm(out[:m] - d) <= tol * np.linalg.norm(d)
    assert np.linalg.norm(out[m:] - xt) <= tol * np.linalg.norm(xt)
