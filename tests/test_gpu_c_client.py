"""The C ABI from a plain C program (gcc, no Python or PyTorch in the
loop): compile tests/c_client/oct_client.c against include/oct_hydro.h and
the library, run it on the GPU."""
import os
import subprocess

import pytest

from paper_2210_06439_gb300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_client(tmp_path):
    lib = build.build()
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = tmp_path / "oct_client"
    src = os.path.join(ROOT, "tests", "c_client", "oct_client.c")
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-O2", "-std=c99", src, "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
           "-L", libdir, "-loct_hydro", "-L", os.path.join(cuda, "lib64"), "-lcudart", "-lm",
           f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "c client ok" in r.stdout
