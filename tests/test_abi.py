"""The C-ABI library loads and exports every symbol include/lbfmm.h declares,
and its host-only calls behave (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbfmm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1306_0612_gb300.build import build

    build()
    from paper_1306_0612_gb300 import lbfmm

    return lbfmm


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbf_[a-z_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    raw = C.CDLL(lib.LIB)
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(raw, n), n
    assert sorted(lib.exported_symbols()) == names


def test_default_options_follow_paper(lib):
    o = lib.lbf_default_options()
    assert o.restart == 50  # Sec. 6: GMRES restarted every 50 iterations
    assert o.tol <= 1e-11   # Sec. 6 uses 1e-11; the build's default is tighter
    assert o.matvec == lib.LBF_MATVEC_FMM and o.border == 1


def test_workspace_size_host_only(lib):
    ptr = np.array([0, 512, 1024], dtype=np.int64)
    o = lib.lbf_default_options()
    b = lib.lbf_workspace_size(ptr, o)
    assert b > 1024 * 8 * 10
    o2 = lib.lbf_default_options(restart=100)
    assert lib.lbf_workspace_size(ptr, o2) > b
    o3 = lib.lbf_default_options(border=0)
    assert lib.lbf_workspace_size(ptr, o3) < b


@pytest.mark.parametrize("field,value", [("restart", 0), ("p", 70), ("leaf_size", 0),
                                         ("max_depth", 31), ("matvec", 5), ("tol", -1.0)])
def test_invalid_options_rejected(lib, field, value):
    ptr = np.array([0, 64], dtype=np.int64)
    o = lib.lbf_default_options(**{field: value})
    with pytest.raises(lib.LbfError) as e:
        lib.lbf_workspace_size(ptr, o)
    assert e.value.status == lib.LBF_EINVAL


def test_bad_island_pointer_rejected(lib):
    o = lib.lbf_default_options()
    for ptr in ([1, 64], [0, 2], [0, 64, 60]):
        with pytest.raises(lib.LbfError):
            lib.lbf_workspace_size(np.array(ptr, dtype=np.int64), o)


def test_status_strings(lib):
    assert lib.lbf_status_string(0) == "ok"
    assert "pole" in lib.lbf_status_string(lib.LBF_EPOLE)
    assert lib.lbf_status_string(12345) == "unknown status"
