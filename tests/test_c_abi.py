"""The C ABI used from plain C: tests/c_abi_example.c compiles against
include/cbct.h alone and links against libcbct.so (CPU); on a GPU it runs
and checks the adjoint identity of the projector pair."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _build(tmp):
    from paper_1001_0599_gb300 import build
    lib = build.build()
    cc = shutil.which("gcc")
    if cc is None or not os.path.isdir(os.path.join(CUDA, "include")):
        pytest.skip("gcc or the CUDA headers are not available")
    exe = os.path.join(tmp, "c_abi_example")
    libdir = os.path.dirname(lib)
    cuda_lib = next((d for d in (os.path.join(CUDA, "lib64"), os.path.join(CUDA, "lib"),
                                 os.path.join(CUDA, "targets", "sbsa-linux", "lib"),
                                 os.path.join(CUDA, "targets", "x86_64-linux", "lib"))
                     if os.path.exists(os.path.join(d, "libcudart.so"))), None)
    if cuda_lib is None:
        pytest.skip("libcudart.so not found")
    cmd = [cc, "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(CUDA, "include"), os.path.join(ROOT, "tests", "c_abi_example.c"), "-o", exe,
           "-L", libdir, "-lcbct", "-L", cuda_lib, "-lcudart", "-lm",
           f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{cuda_lib}"]
    libcbct = os.path.join(libdir, "libcbct.so")
    if not os.path.exists(libcbct):
        pytest.skip("libcbct.so not built")
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe


def test_c_example_compiles_and_links(tmp_path):
    exe = _build(str(tmp_path))
    assert os.path.exists(exe)


@pytest.mark.gpu
def test_c_example_runs(tmp_path):
    exe = _build(str(tmp_path))
    res = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "relative difference" in res.stdout
