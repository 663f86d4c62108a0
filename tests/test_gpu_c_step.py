"""The C ABI from plain C: tests/c_step.c allocates device arrays with the
CUDA runtime, bins the species, builds the tables and runs three FP64 steps
(every process, then Trident alone and Bethe-Heitler alone) through
include/pcc.h, then checks the status, the step counters and every live
particle against the oracle stepping the same host particles in the same
program."""
import glob
import os
import shutil
import subprocess

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_dirs(nvcc):
    home = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    inc = os.path.join(home, "include")
    libs = [os.path.join(home, "lib64")] + sorted(glob.glob(os.path.join(home, "targets", "*", "lib")))
    lib = next((d for d in libs if os.path.exists(os.path.join(d, "libcudart.so"))), None)
    return inc, lib


def test_c_program_steps_like_the_oracle(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    from paper_1907_02814_gb300 import build
    build.build()
    inc, lib = _cuda_dirs(build.NVCC)
    assert lib is not None, "libcudart.so not found beside nvcc"
    libdir = os.path.dirname(build.LIB)
    exe = str(tmp_path / "c_step")
    cmd = ["gcc", "-std=c11", "-O2", "-Wall", "-Wextra", "-Werror", "-ffp-contract=off", "-fno-fast-math",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "oracle"), "-I", inc,
           os.path.join(ROOT, "tests", "c_step.c"), os.path.join(ROOT, "oracle", "pcc_oracle.c"),
           "-L", libdir, "-l:libpcc.so", "-L", lib, "-lcudart", "-lm",
           f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{lib}", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "C step matches the oracle" in r.stdout
