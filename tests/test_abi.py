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


def test_batch_workspace_size_host_only(lib):
    """A batch item's workspace: the plan's bytes (rounded up to 256), then the lockstep
    slabs of its right-hand sides (lbf_gmres_solve_many), which grow with their number up
    to one group of 16 and are absent where right-hand sides run one after another (a
    single one, no border, or S^-1 by LU factors)."""
    ptr = np.array([0, 300, 700, 1000], dtype=np.int64)
    o = lib.lbf_default_options()
    plan = lib.lbf_workspace_size(ptr, o)
    rnd = (plan + 255) // 256 * 256
    assert lib.lbf_batch_workspace_size(ptr, o, 0) == plan
    assert lib.lbf_batch_workspace_size(ptr, o, 1) == plan
    b2, b8, b16 = (lib.lbf_batch_workspace_size(ptr, o, r) for r in (2, 8, 16))
    # each right-hand side's slab holds at least its Krylov basis ((restart + 1) x n doubles)
    n = int(ptr[-1]) + len(ptr) - 1
    states = 3 * 128  # per right-hand side: three staged GMRES states for the host's reads
    slab = (b16 - rnd - 16 * states) // 16
    assert (b16 - rnd - 16 * states) % (16 * 256) == 0 and slab >= 8 * 51 * n
    assert b2 - rnd == 2 * (slab + states) and b8 - rnd == 8 * (slab + states)
    assert lib.lbf_batch_workspace_size(ptr, o, 40) == b16  # groups of 16 reuse one workspace
    ir = lib.lbf_default_options(precision=lib.LBF_PRECISION_FP32_REFINE)
    assert lib.lbf_batch_workspace_size(ptr, ir, 4) > (lib.lbf_workspace_size(ptr, ir) + 255) // 256 * 256
    for opt in (lib.lbf_default_options(schur=lib.LBF_SCHUR_LU), lib.lbf_default_options(border=0)):
        assert lib.lbf_batch_workspace_size(ptr, opt, 16) == lib.lbf_workspace_size(ptr, opt)
    with pytest.raises(lib.LbfError):
        lib.lbf_batch_workspace_size(ptr, o, -1)
