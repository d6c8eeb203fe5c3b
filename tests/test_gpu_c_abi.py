"""The library used from C: tests/c/c_abi_example.c includes include/snap.h only, links the
shared library, builds a hydrostatic column, steps it and checks conservation. Compiles on
the host (no GPU needed to build); runs on the GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1901_02955_gb300")


def compile_example(tmp_path):
    from paper_1901_02955_gb300 import build
    lib = build.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    exe = tmp_path / "c_abi_example"
    subprocess.check_call([cc, "-std=c99", "-O2", "-I", os.path.join(ROOT, "include"), "-I",
                           cuda_inc, os.path.join(ROOT, "tests", "c", "c_abi_example.c"), "-o",
                           str(exe), lib, "-Wl,-rpath," + os.path.dirname(lib), "-lm"])
    return exe


def test_c_example_compiles_against_the_header(tmp_path):
    assert compile_example(tmp_path).exists()


@pytest.mark.gpu
def test_c_example_runs(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = compile_example(tmp_path)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok")
