"""The oracle, and the host code of the C ABI, under AddressSanitizer and
UndefinedBehaviorSanitizer.

A native C driver (sanitize_oracle.c, beside this file) links the oracle's
source and calls every entry point on small inputs that reach its edges:
empty, single-particle and ion-free cells, ragged counts, energies above
the table, a step long enough that every pair collides, a photon store
that overflows, both screening modes and both nonrelativistic bounds.  It
also checks, with -Wall -Wextra -Werror, that the oracle compiles without
warnings.  Running the C programs natively keeps the sanitizer runtimes out of
the Python process."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ORACLE = os.path.join(ROOT, "oracle")
SRC = [os.path.join(HERE, "sanitize_oracle.c"), os.path.join(ORACLE, "pcc_oracle.c")]

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")


@pytest.mark.parametrize("openmp", [False, True])
def test_oracle_compiles_without_warnings(tmp_path, openmp):
    r = subprocess.run(["gcc", "-std=c11", "-O2", "-Wall", "-Wextra", "-Werror", "-ffp-contract=off",
                        "-fsyntax-only", "-I", ORACLE] + (["-fopenmp"] if openmp else []) + SRC,
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_oracle_under_asan_and_ubsan(tmp_path):
    exe = str(tmp_path / "sanitize_oracle")
    cc = subprocess.run(["gcc", "-std=c11", "-O1", "-g", "-fsanitize=address,undefined", "-fno-omit-frame-pointer",
                         "-fno-sanitize-recover=all", "-ffp-contract=off", "-I", ORACLE] + SRC + ["-lm", "-o", exe],
                        capture_output=True, text=True)
    if cc.returncode != 0 and ("asan" in cc.stderr or "ubsan" in cc.stderr):
        pytest.skip("sanitizer runtimes not installed: " + cc.stderr.strip().splitlines()[-1])
    assert cc.returncode == 0, cc.stderr
    env = dict(os.environ, ASAN_OPTIONS="abort_on_error=0:detect_leaks=1:strict_string_checks=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "all checks passed" in r.stdout
    assert "runtime error" not in r.stderr and "Sanitizer" not in r.stderr, r.stderr


@pytest.mark.slow
def test_c_abi_argument_checks_under_asan_and_ubsan(tmp_path):
    """The C ABI's host code, built with the sanitizers (device code as PTX
    only, never run), driven by sanitize_abi.c: every entry point rejects
    null contexts, null arrays and bad sizes with the documented code and a
    message naming the call, before any CUDA work and without a GPU."""
    import concurrent.futures as cf
    import glob

    from paper_1907_02814_gb300 import build as B
    if not os.path.exists(B.NVCC):
        pytest.skip("needs nvcc")
    san = "-fsanitize=address,-fsanitize=undefined,-fno-omit-frame-pointer,-fPIC"
    arch = ["-gencode", "arch=compute_103a,code=compute_103a"]

    def compile_one(src):
        obj = str(tmp_path / (os.path.basename(src) + ".o"))
        r = subprocess.run([B.NVCC, *arch, "-O1", "-std=c++17", "-Xcompiler", san, "-I", B.INCLUDE, "-c", src,
                            "-o", obj], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        return obj

    srcs = sorted(glob.glob(os.path.join(B.CSRC, "*.cu")))
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    main_o = str(tmp_path / "sanitize_abi.o")
    r = subprocess.run(["gcc", "-std=c11", "-g", "-c", "-fsanitize=address,undefined", "-fno-omit-frame-pointer",
                        "-I", B.INCLUDE, os.path.join(HERE, "sanitize_abi.c"), "-o", main_o],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    exe = str(tmp_path / "sanitize_abi")
    r = subprocess.run([B.NVCC, *arch, "-Xcompiler", san, "-o", exe, main_o, *objs], capture_output=True, text=True)
    if r.returncode != 0 and ("asan" in r.stderr or "ubsan" in r.stderr):
        pytest.skip("sanitizer runtimes not installed")
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="protect_shadow_gap=0:detect_leaks=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "all checks passed" in r.stdout
    assert "runtime error" not in r.stderr and "Sanitizer" not in r.stderr, r.stderr
