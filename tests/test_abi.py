"""The C-ABI library loads without a GPU and exports every function that
include/kry.h declares; the Python binding's signatures cover the header."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kry.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kry_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2012_13133_gb300.build import build_library
    return build_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["kry_embed_eigs", "kry_matvec", "kry_logdet", "kry_solve", "kry_profile_loglik", "kry_krige"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (kry_[a-z_0-9]+)", out))
    assert set(declared_functions()) <= exported


def test_binding_signatures_cover_header(libpath):
    from paper_2012_13133_gb300 import kry
    assert set(kry.SIGNATURES) == set(declared_functions())
