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


def test_checkpoint_load_rejects_bad_files_without_touching_the_device(tmp_path):
    """tdks_load refuses a missing file, a file that is not a checkpoint and a truncated
    header with TDKS_EINVAL before any CUDA call (so this runs without a GPU)."""
    import ctypes
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_07921_gb300 import _lib
    lib = _lib.load()
    out = ctypes.c_void_p()
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"NOTACKPT" + bytes(400))
    short = tmp_path / "short.ckpt"
    short.write_bytes(b"TDKSCKP1" + bytes(40))
    for path in (tmp_path / "missing.ckpt", bad, short):
        assert lib.tdks_load(str(path).encode(), None, ctypes.byref(out)) == 1
        assert out.value is None
    assert lib.tdks_load(str(bad).encode(), None, ctypes.byref(out)) == 1
    assert b"not a checkpoint" in lib.tdks_last_error()
    assert lib.tdks_save(None, str(tmp_path / "x").encode()) == 1
