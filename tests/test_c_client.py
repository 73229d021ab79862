"""The C ABI from a plain C program (tests/c_client.c): it compiles against
include/lsg.h as C99, links liblsg.so and the CUDA runtime, and makes its
calls with no Python or torch in the process."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def build_client(tmp_path):
    from paper_2005_02704_gb300 import _build
    lib = _build.build()
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    cuda = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    libdirs = [d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib")) if os.path.isdir(d)]
    cc = shutil.which("gcc") or shutil.which("cc")
    exe = str(tmp_path / "c_client")
    pkg = os.path.dirname(lib)
    cmd = [cc, "-std=c99", "-O2", "-Wall", "-Wextra", "-Werror", os.path.join(ROOT, "tests", "c_client.c"),
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"), "-L", pkg, "-llsg"]
    for d in libdirs:
        cmd += ["-L", d, f"-Wl,-rpath,{d}"]
    cmd += [f"-Wl,-rpath,{pkg}", "-lcudart", "-lm", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_client_host_calls(tmp_path):
    exe = build_client(tmp_path)
    r = subprocess.run([exe, "host"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stderr


@pytest.mark.gpu
def test_c_client_segments_a_wall(gpu_lib, tmp_path):
    exe = build_client(tmp_path)
    r = subprocess.run([exe, "gpu"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stderr
