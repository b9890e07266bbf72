"""The C-ABI library builds, loads and exports every entry point include/pl.h
declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "pl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pl_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_paper_entry_points():
    names = _declared()
    for n in ["pl_sample", "pl_fit_mle", "pl_ks_stat", "pl_ks_cutoffs", "pl_bootstrap_pvalue"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1305_6738_gb300 import build
    lib = ctypes.CDLL(build.build())
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_1305_6738_gb300 import build
    build.build()
    from paper_1305_6738_gb300 import pl
    assert sorted(pl.EXPORTS) == _declared()
