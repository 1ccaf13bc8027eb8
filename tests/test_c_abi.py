"""The C ABI used from plain C, without Python or torch on the call path: tests/c_abi_example.c
includes include/xe.h, allocates its own device buffers, correlates and normalises a constant frame
and checks the closed forms (V = T x_i conj(x_j), V / T). On the CPU the program must compile as C11
and link against libxe and the CUDA runtime; on a GPU it must run and match."""
import os
import subprocess

import pytest

import paper_1503_06189_b300 as xe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _build(tmp_path):
    exe = str(tmp_path / "c_abi_example")
    lib_dir = os.path.dirname(xe.LIB_PATH)
    cuda_lib = os.path.join(CUDA, "lib64")
    cmd = ["gcc", "-std=c11", "-O2", "-Wall", "-Wextra", "-Werror",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           os.path.join(ROOT, "tests", "c_abi_example.c"), "-o", exe,
           "-L", lib_dir, "-lxe", f"-Wl,-rpath,{lib_dir}", "-L", cuda_lib, "-lcudart", f"-Wl,-rpath,{cuda_lib}", "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_example_compiles_and_links(tmp_path):
    assert os.access(_build(tmp_path), os.X_OK)


@pytest.mark.gpu
def test_c_example_runs(tmp_path):
    r = subprocess.run([_build(tmp_path)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok:")
