"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every function declared in include/pcc.h (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(pcc_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1907_02814_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("pcc_create", "pcc_tables_build", "pcc_bin", "pcc_collide", "pcc_append_secondaries",
                 "pcc_read_status", "pcc_expected_emission_fwd", "pcc_expected_emission_bwd"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_1907_02814_gb300 import pcc
    assert set(declared_functions()) == set(pcc.EXPORTS)
    pcc.load()
    assert pcc.load().pcc_version().decode().startswith("pcc")


def test_null_arguments_rejected_without_a_device(lib):
    from paper_1907_02814_gb300 import pcc
    L = pcc.load()
    assert L.pcc_create(None, 0) == pcc.PCC_E_INVALID
    assert L.pcc_tables_build(None, None, 0, None, None) == pcc.PCC_E_INVALID
    assert L.pcc_collide(None, None, None, None, None, None, 1.0, 0, 0, 7, 0, None, None) == pcc.PCC_E_INVALID
    assert b"invalid" in L.pcc_last_error()
    thr = (ctypes.c_int * 4)(20, 18, 14, 0)
    assert L.pcc_set_scan_classes(None, 0, thr) == pcc.PCC_E_INVALID
    assert L.pcc_get_scan_classes(None, 0, thr) == pcc.PCC_E_INVALID


def test_status_strings_without_a_device(lib):
    from paper_1907_02814_gb300 import pcc
    L = pcc.load()
    names = {pcc.PCC_OK: "PCC_OK", pcc.PCC_E_INVALID: "PCC_E_INVALID", 2: "PCC_E_CUDA", 3: "PCC_E_CAPACITY",
             4: "PCC_E_NO_TABLES"}
    for code, name in names.items():
        assert L.pcc_status_string(code).decode().startswith(name + ": ")
    assert L.pcc_status_string(5) == b"unknown return code"
    assert L.pcc_status_string(-1) == b"unknown return code"
    bits = {pcc.ST_TABLE_RANGE: "PCC_ST_TABLE_RANGE", pcc.ST_PROB_LARGE: "PCC_ST_PROB_LARGE",
            pcc.ST_CAPACITY: "PCC_ST_CAPACITY", pcc.ST_NONFINITE: "PCC_ST_NONFINITE",
            pcc.ST_ID_RANGE: "PCC_ST_ID_RANGE", pcc.ST_TIMEOUT: "PCC_ST_TIMEOUT",
            pcc.ST_BOUND_RANGE: "PCC_ST_BOUND_RANGE"}
    for bit, name in bits.items():
        assert L.pcc_status_bit_string(bit).decode() == name
    assert L.pcc_status_bit_string(0) == b"unknown status bit"
    assert L.pcc_status_bit_string(3) == b"unknown status bit"
    assert L.pcc_status_bit_string(0x80) == b"unknown status bit"
    assert pcc.status_bits(pcc.ST_TIMEOUT | pcc.ST_TABLE_RANGE) == ["PCC_ST_TABLE_RANGE", "PCC_ST_TIMEOUT"]
    with pytest.raises(pcc.PccError, match="PCC_E_INVALID"):
        pcc._check(L.pcc_create(None, 0), "pcc_create")


def test_c_program_links_against_the_library(lib, tmp_path):
    """A plain C program (the argument-check driver beside this file)
    compiles against include/pcc.h with gcc, links libpcc.so and runs
    without a GPU: the boundary is usable from C, not only through ctypes."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    from paper_1907_02814_gb300 import build
    libdir = os.path.dirname(build.LIB)
    exe = str(tmp_path / "abi_c")
    r = subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "sanitize_abi.c"), "-o", exe, "-L", libdir, "-l:libpcc.so",
                        f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120,
                       env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stdout + r.stderr
    assert "all checks passed" in r.stdout


@pytest.mark.parametrize("lang,std", [("c", "c99"), ("c", "c11"), ("c++", "c++11"), ("c++", "c++17")])
def test_header_is_clean_c_and_cxx(tmp_path, lang, std):
    """include/pcc.h compiles on its own, pedantic and warning-free, as C99
    and later and as C++11 and later (extern "C" guarded)."""
    import shutil
    import subprocess
    cc = "gcc" if lang == "c" else "g++"
    if shutil.which(cc) is None:
        pytest.skip(f"needs {cc}")
    src = tmp_path / ("h.c" if lang == "c" else "h.cpp")
    src.write_text('#include "pcc.h"\n#include "pcc.h"\nint main(void) { return PCC_OK; }\n')
    r = subprocess.run([cc, f"-std={std}", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I",
                        os.path.join(ROOT, "include"), "-c", str(src), "-o", str(tmp_path / "h.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
