"""Batched solves of independent uneven geometries through the native scheduler:
every instance matches its own single-plan solve (same kernels, any stream) and the
oracle's dense solve."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import workloads as wl  # noqa: E402
from gpu_util import dev, host, plan_for, rel_l2, zeros  # noqa: E402
from paper_1306_0612_gb300 import lbfmm as L  # noqa: E402

pytestmark = pytest.mark.gpu


def _instances(count=7, nrhs=3):
    inst = wl.batch_instances(seed=44, count=count, nrhs=nrhs, max_islands=6, nodes_range=(48, 160))
    out = []
    for g, pairs in inst:
        data = np.stack([oracle.green_sum(g.x, p, gam) for p, gam in pairs])
        t = wl.targets_off_islands(g, 40, seed=3)
        out.append(dict(geom=g, data=data, island_ptr=g.island_ptr, x=dev(g.x), dx=dev(g.dx),
                        d2x=dev(g.d2x), centres=dev(g.centres), g=dev(data), targets=dev(t)))
    return out


@pytest.mark.parametrize("precision", [L.LBF_PRECISION_FP64, L.LBF_PRECISION_FP32_REFINE])
def test_batch_matches_single_solves_and_oracle(precision):
    inst = _instances()
    opt = L.lbf_default_options(tol=1e-12, precision=precision)
    res = L.lbf_batch_run(inst, opt=opt, nworkers=4)
    for ins, r in zip(inst, res):
        g = ins["geom"]
        assert r["status"] == L.LBF_OK and r["max_rel_res"] <= 1e-12
        p = plan_for(g, tol=1e-12, precision=precision)
        A = oracle.matrix(g)
        for k in range(ins["data"].shape[0]):
            sig, a = zeros(g.N), zeros(g.M)
            L.lbf_gmres_solve(p, dev(ins["data"][k]), sig, a)
            assert np.array_equal(host(r["sigma"][k]), host(sig))
            assert np.array_equal(host(r["a"][k]), host(a))
            u = zeros(40)
            L.lbf_evaluate(p, sig, a, ins["targets"], u)
            assert np.array_equal(host(r["u"][k]), host(u))
            z = np.linalg.solve(A, np.concatenate([2 * ins["data"][k], np.zeros(g.M)]))
            assert rel_l2(host(sig), z[:g.N]) < 1e-9
