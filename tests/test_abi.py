"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
symbol that include/flgf.h declares (no compute calls here)."""
import ctypes
import os
import re

from paper_1911_10228_gb300 import build as B
from paper_1911_10228_gb300 import flgf as F

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "flgf.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(flgf_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("flgf_create", "flgf_blockset_create", "flgf_load_source", "flgf_solve",
                     "flgf_get_potential", "flgf_laplacian", "flgf_lgf_eval"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_prototypes_match_header():
    assert sorted(F.PROTOTYPES) == declared_symbols()


def test_library_is_built_for_sm_103a_only():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
