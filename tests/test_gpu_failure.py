"""Failure detection on the GPU without a fault: every device wait of the library is
bounded, records LBF_ETIMEOUT in the plan's status word when it gives up, and lets its
kernel finish.  A test-only injection makes a real wait site run out (a flag or a
barrier that nothing releases, with a short poll limit); the host reads the status, and
the context stays usable afterwards."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import workloads as wl  # noqa: E402
from gpu_util import dev, host, plan_for, rel_l2, zeros  # noqa: E402
from paper_1306_0612_gb300 import lbfmm as L  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fmm64", [0, 1])
def test_chain_parent_wait_runs_out_and_the_plan_recovers(oracle, fmm64):
    g = wl.config_geometry("C2")
    p = plan_for(g, fmm64=fmm64)
    v = wl.random_density(g.N, 4)
    out = zeros(g.N)
    L.lbf_debug_inject(p, L.LBF_INJECT_CHAIN, 2000)
    L.lbf_apply(p, L.LBF_OP_K_ONLY, dev(v), out)
    assert L.lbf_sync_status(p) == L.LBF_ETIMEOUT
    # the chain finished and reset its counters: the next application is exact again
    L.lbf_debug_clear(p)
    L.lbf_apply(p, L.LBF_OP_K_ONLY, dev(v), out)
    assert L.lbf_sync_status(p) == L.LBF_OK
    assert rel_l2(host(out), oracle.apply(g, v, 1)) < 1e-10


@pytest.mark.parametrize("schur", [L.LBF_SCHUR_GJ, L.LBF_SCHUR_LU])
def test_grid_barrier_runs_out_in_plan_creation(schur):
    g = wl.config_geometry("C2", nodes=64)
    L.lbf_debug_inject(None, L.LBF_INJECT_BARRIER, 2000)
    with pytest.raises(L.LbfError) as e:
        plan_for(g, schur=schur)
    assert e.value.status == L.LBF_ETIMEOUT
    # the injection applied to that creation only: the next one builds and solves
    p = plan_for(g, schur=schur, tol=1e-12)
    src, gam, _ = wl.pair_sources(g, 0, 1)
    data = zeros(g.N)
    L.lbf_green_sum(dev(g.x), dev(src), dev(gam), data)
    sig, a = zeros(g.N), zeros(g.M)
    rc, its, rr = L.lbf_gmres_solve(p, data, sig, a)
    assert rc == L.LBF_OK and rr <= 1e-12


def test_injection_arguments_are_checked():
    with pytest.raises(L.LbfError):
        L.lbf_debug_inject(None, L.LBF_INJECT_CHAIN, 100)
    with pytest.raises(L.LbfError):
        L.lbf_debug_inject(None, L.LBF_INJECT_BARRIER, 0)
    g = wl.config_geometry("C1", nodes=64)
    p = plan_for(g, matvec=L.LBF_MATVEC_DIRECT)
    with pytest.raises(L.LbfError):
        L.lbf_debug_inject(p, L.LBF_INJECT_CHAIN, 100)
