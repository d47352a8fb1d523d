"""The C-ABI library loads without a GPU and exports every symbol that
include/emin.h declares; the Python binding uses the same names."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(emin_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2208_02995_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for s in ("emin_create", "emin_iterate", "emin_energy", "emin_get_p", "emin_backward",
              "emin_destroy", "emin_stats", "emin_strerror"):
        assert s in names


def test_library_exports_declared_symbols(libpath):
    L = ctypes.CDLL(libpath)
    missing = [s for s in sorted(_declared()) if not hasattr(L, s)]
    assert not missing, missing


def test_binding_names_match(libpath):
    from paper_2208_02995_gb300 import emin as E
    for s in _declared():
        assert hasattr(E, s), s
    assert E.strerror(E.EMIN_ERR_BREAKDOWN).startswith("conjugate gradient breakdown")
    o = E.emin_default_opts()
    assert o.precision == E.EMIN_FP64 and o.rank_policy == E.EMIN_RANK_STRICT


def test_no_oracle_in_product_path():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2208_02995_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"(?:import|from)\s+(\w+)", txt), f


def test_create_rejects_unknown_check_mode(libpath):
    """emin_opts.checks is 0 or 1; anything else is rejected before any
    device work."""
    import numpy as np
    from paper_2208_02995_gb300 import emin as E
    o = E.emin_default_opts()
    o.checks = 2
    z = np.zeros(2, dtype=np.int32)
    with pytest.raises(E.EminError) as err:
        E.emin_create(1, 1, 1, z, z, np.zeros(1), z, z, np.zeros(1), np.ones(1), np.ones(1),
                      opts=o, inputs_on_device=False)
    assert err.value.status == E.EMIN_ERR_ARG
