"""The autotuner (lbf_autotune): the options it picks for a geometry meet its accuracy
target against the oracle, and its table records the trials that justify them."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import workloads as wl  # noqa: E402
from gpu_util import dev, host, rel_l2, zeros  # noqa: E402
from paper_1306_0612_gb300 import lbfmm as L  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fmm64", [0, 1])
def test_tuned_options_meet_the_target_against_the_oracle(oracle, fmm64):
    g = wl.star_caps(3, 256, 1024)
    x, dx, d2x, c = dev(g.x), dev(g.dx), dev(g.d2x), dev(g.centres)
    target = 1e-10
    best, table = L.lbf_autotune(g.island_ptr, x, dx, d2x, c, target,
                                 opt=L.lbf_default_options(fmm64=fmm64))
    assert best.leaf_size in (32, 48, 64) and 16 <= best.p <= 38 and best.p2p_warps in (0, 2, 8)
    assert best.fmm64 == fmm64
    trials = table["trials"]
    ok = [t for t in trials if t["status"] == 0 and 0 <= t["err"] <= target / 4]
    assert ok and min(t["ms"] for t in ok) == pytest.approx(table["best"]["ms"])
    # every leaf size stopped at the first order that met the goal
    for leaf in (32, 48, 64):
        ps = [t for t in trials if t["leaf"] == leaf and t["warps"] == 4]
        assert all(t["err"] > target / 4 for t in ps[:-1])
    p = L.lbf_plan_create(g.island_ptr, x, dx, d2x, c, opt=best)
    sig = wl.random_density(g.N, 3)
    out = zeros(g.N)
    L.lbf_apply(p, L.LBF_OP_K_ONLY, dev(sig), out)
    rows = np.sort(np.random.default_rng(7).choice(g.N, 64, replace=False))
    ref = oracle.apply_rows(g, sig, rows, op=1)
    assert rel_l2(host(out)[rows], ref) < target


def test_autotune_workspace_query_and_short_workspace():
    import ctypes as C
    g = wl.config_geometry("C2", nodes=64)
    lib = L.load()
    ptr = np.ascontiguousarray(g.island_ptr, dtype=np.int64)
    need = C.c_size_t(0)
    best = L.lbf_options()
    opt = L.lbf_default_options()
    rc = lib.lbf_autotune(g.M, ptr.ctypes.data_as(C.c_void_p), None, None, None, None, None,
                          C.byref(opt), 1e-10, None, 0, C.byref(need), C.byref(best), None, 0, None)
    assert rc == L.LBF_OK and need.value > 0
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    x = dev(g.x)
    rc = lib.lbf_autotune(g.M, ptr.ctypes.data_as(C.c_void_p), C.c_void_p(x.data_ptr()),
                          C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()),
                          C.c_void_p(x.data_ptr()), None, C.byref(opt), 1e-10,
                          C.c_void_p(ws.data_ptr()), 16, C.byref(need), C.byref(best), None, 0, None)
    assert rc == L.LBF_EWORKSPACE
