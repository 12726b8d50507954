"""The C-ABI library loads and exports every function include/sparse_spectral.h
declares (no GPU needed: nothing is called that touches a device)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sparse_spectral.h")
LIB = os.path.join(ROOT, "paper_2302_00752_gb300", "libsparse_spectral.so")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s+([a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2302_00752_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_path():
    names = declared_functions()
    for n in ("sft_recover", "stamp_build", "galerkin_apply", "solve", "batch_solve", "lattice_random",
              "lattice_cbc", "lattice_check", "lattice_sample"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), f"{n} missing from the library"


def test_host_only_calls(lib):
    lib.ss_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.ss_version()
    M = ctypes.c_int64()
    lib.lattice_size.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_int64,
                                 ctypes.POINTER(ctypes.c_int64)]
    assert lib.lattice_size(2048, 35, 0.05, 0, ctypes.byref(M)) == 0
    from oracle import lattice as olat
    assert M.value == olat.random_lattice_size(2048, 35, 0.05)
    assert lib.lattice_size(10, 3, 0.0, 0, ctypes.byref(M)) == 1     # sigma must be positive


def test_no_cpu_compute_path_in_binding():
    # the binding is marshalling only: it must not import the oracle
    src = open(os.path.join(ROOT, "paper_2302_00752_gb300", "binding.py")).read()
    src += open(os.path.join(ROOT, "paper_2302_00752_gb300", "pipeline.py")).read()
    assert "oracle" not in re.sub(r'""".*?"""', "", src, flags=re.S)


def test_symbols_have_c_linkage():
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    for n in declared_functions():
        assert n in exported
