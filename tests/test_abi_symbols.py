"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    names = []
    for h in sorted((ROOT / "include").glob("*.h")):
        text = h.read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(gwas_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gwas_init", "gwas_factor", "gwas_solve_block", "gwas_sync",
                     "gwas_finalize", "gwas_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1304_2272_gb300 import build, gwas
    lib_path = build.build()
    lib = ctypes.CDLL(str(lib_path))
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    # the Python binding wraps exactly the declared C entry points
    assert set(gwas.SIGNATURES) == set(declared_functions())


def test_binding_names_match_the_abi():
    from paper_1304_2272_gb300 import gwas
    for name in declared_functions():
        assert callable(getattr(gwas, name))


def test_init_fails_loudly_without_a_gpu():
    from conftest import has_gpu
    if has_gpu():
        pytest.skip("a GPU is present")
    from paper_1304_2272_gb300 import gwas
    with pytest.raises(gwas.GwasError):
        gwas.gwas_init(100, 4, 1)
