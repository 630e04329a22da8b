"""lbf_evaluate_noalloc, the evaluation entry point for callers that cannot
allocate device memory (its scratch is a static device array inside the
library).  Checked through the C ABI against lbf_evaluate on two calls in a
row, so that scratch left behind by the first call cannot leak into the second.
This file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import workloads as wl  # noqa: E402
from gpu_util import dev, host, plan_for, zeros  # noqa: E402
from paper_1306_0612_gb300 import lbfmm as L  # noqa: E402

pytestmark = pytest.mark.gpu


def test_noalloc_evaluate_matches_plan_evaluate_twice():
    g = wl.config_geometry("C2", nodes=128)
    p = plan_for(g)
    N, M = g.N, g.M
    xi, w = zeros(2 * N), zeros(2 * N)
    L.lbf_geometry_out(p, xi=xi, weight=w)
    tg = dev(wl.targets_off_islands(g, 96, seed=4))
    rng = np.random.default_rng(12)
    for call in range(2):
        sig = dev(rng.standard_normal(N))
        a = dev(rng.standard_normal(M))
        ref, got = zeros(96), zeros(96)
        L.lbf_evaluate(p, sig, a, tg, ref)
        L.lbf_evaluate_noalloc(xi, w, sig, a, dev(g.centres), tg, got)
        r, q = host(ref), host(got)
        assert np.max(np.abs(q - r)) < 1e-12 * np.max(np.abs(r)), call


def test_noalloc_rejects_more_nodes_than_its_scratch_holds():
    tiny = zeros(8)
    with pytest.raises(L.LbfError) as e:
        L.lbf_evaluate_noalloc(tiny, tiny, tiny, None, None, tiny[:3], tiny[:1],
                               N=L.LBF_NOALLOC_MAX_NODES + 1)
    assert e.value.status == L.LBF_EINVAL
