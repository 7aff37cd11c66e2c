"""The C library loads and exports every symbol that include/tdks.h declares (CPU only:
no compute call is made without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "tdks.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tdks_[A-Za-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("tdks_create_grid", "tdks_set_atoms_projectors", "tdks_set_field", "tdks_apply_H",
              "tdks_propagate_n", "tdks_reductions", "tdks_destroy", "tdks_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_07921_gb300 import _lib
    lib = _lib.load()
    names = _declared()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(_lib.SIGNATURES) == names


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1912_07921_gb300 import _lib
    with pytest.raises(RuntimeError, match="not built"):
        old = _lib._lib
        _lib._lib = None
        try:
            _lib.load(str(tmp_path / "missing.so"))
        finally:
            _lib._lib = old
