"""The C-ABI library loads and exports every entry point that include/nesa.h declares
(no GPU needed: nothing is called that touches a device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(nesa_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def libnesa():
    from paper_1801_03589_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_every_declared_symbol_is_exported(libnesa):
    names = _declared()
    assert "nesa_build" in names and "nesa_matvec" in names
    missing = [n for n in names if not hasattr(libnesa, n)]
    assert not missing, missing


def test_host_only_entry_points(libnesa):
    import paper_1801_03589_gb300 as nesa
    p = nesa.default_params()
    assert p.leaf_size == 0.25 and p.q_mode == nesa.Q_AUTO and p.q_fixed == 100
    assert abs(p.rho_test - (2 - 3 ** 0.5 / 2) / (3 ** 0.5 / 2)) < 1e-15
    for s in (0, -1, -2, -3, -4, -5, -6, -7):
        assert nesa.lib().nesa_status_str(s)
    # null arguments are rejected before any device work
    assert nesa.lib().nesa_build(None, 1.0, None, None) == nesa.ERR_INVALID_ARG
    assert nesa.lib().nesa_matvec(None, None, None, 1) == nesa.ERR_INVALID_ARG
