"""lbf_evaluate_noalloc, the evaluation entry point for callers that cannot
allocate device memory (its scratch is a static device array inside the
library).  Checked through the C ABI against lbf_evaluate on two calls in a
row, so that scratch left behind by the first call cannot leak into the second,
and against the oracle's representation formula (Eq. u_multi).
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


def _planar(p, N):
    xi, w = zeros(2 * N), zeros(2 * N)
    L.lbf_geometry_out(p, xi=xi, weight=w)
    return xi, w


def test_noalloc_evaluate_matches_plan_evaluate_twice(oracle):
    g = wl.config_geometry("C2", nodes=128)
    p = plan_for(g)
    N, M = g.N, g.M
    xi, w = _planar(p, N)
    T = 96
    tgh = wl.targets_off_islands(g, T, seed=4)
    tg = dev(tgh)
    rng = np.random.default_rng(12)
    for call in range(2):
        sh, ah = rng.standard_normal(N), rng.standard_normal(M)
        sig, a = dev(sh), dev(ah)
        ref, got = zeros(T), zeros(T)
        L.lbf_evaluate(p, sig, a, tg, ref)
        L.lbf_evaluate_noalloc(xi, w, sig, a, dev(g.centres), tg, got)
        r, q = host(ref), host(got)
        assert np.max(np.abs(q - r)) < 1e-12 * np.max(np.abs(r)), call
        orc = oracle.evaluate(g, sh, ah, tgh)
        assert np.max(np.abs(q - orc)) < 1e-11 * np.max(np.abs(orc)), call


def test_noalloc_at_its_node_limit():
    """N = LBF_NOALLOC_MAX_NODES: 1024 blocks of 256 threads fill the partials array
    and the last-block reduction (256 islands x 1024 nodes)."""
    g = wl.star_caps(3, 256, 1024)
    assert g.N == L.LBF_NOALLOC_MAX_NODES
    p = plan_for(g)
    xi, w = _planar(p, g.N)
    T = 64
    tg = dev(wl.targets_off_islands(g, T, seed=8))
    rng = np.random.default_rng(5)
    for call in range(2):
        sig, a = dev(rng.standard_normal(g.N)), dev(rng.standard_normal(g.M))
        ref, got = zeros(T), zeros(T)
        L.lbf_evaluate(p, sig, a, tg, ref)
        L.lbf_evaluate_noalloc(xi, w, sig, a, dev(g.centres), tg, got)
        r, q = host(ref), host(got)
        assert np.max(np.abs(q - r)) < 1e-11 * np.max(np.abs(r)), call


def test_noalloc_with_a_rotated_plan(oracle):
    """A plan built with a pole rotation returns the nodes in the rotated frame, so the
    caller passes targets and multiplier sites rotated the same way."""
    g = wl.star_caps(9, 4, 96, pole=None)
    R = wl.rotation_to_pole(g.centres[0])
    p = plan_for(g, rotation=R)
    xi, w = _planar(p, g.N)
    T = 40
    tgh = wl.targets_off_islands(g, T, seed=6)
    rng = np.random.default_rng(2)
    for call in range(2):
        sh, ah = rng.standard_normal(g.N), rng.standard_normal(g.M)
        ref, got = zeros(T), zeros(T)
        L.lbf_evaluate(p, dev(sh), dev(ah), dev(tgh), ref)
        L.lbf_evaluate_noalloc(xi, w, dev(sh), dev(ah), dev(wl.apply_rotation(R, g.centres)),
                               dev(wl.apply_rotation(R, tgh)), got)
        r, q = host(ref), host(got)
        assert np.max(np.abs(q - r)) < 1e-12 * np.max(np.abs(r)), call
        orc = oracle.evaluate(g, sh, ah, tgh)
        assert np.max(np.abs(q - orc)) < 1e-11 * np.max(np.abs(orc)), call


def test_noalloc_rejects_more_nodes_than_its_scratch_holds():
    tiny = zeros(8)
    with pytest.raises(L.LbfError) as e:
        L.lbf_evaluate_noalloc(tiny, tiny, tiny, None, None, tiny[:3], tiny[:1],
                               N=L.LBF_NOALLOC_MAX_NODES + 1)
    assert e.value.status == L.LBF_EINVAL


def test_noalloc_binding_checks_sizes():
    tiny = zeros(8)
    with pytest.raises(ValueError):
        L.lbf_evaluate_noalloc(tiny, tiny, tiny, None, None, tiny[:3], tiny[:1], N=5)
    with pytest.raises(ValueError):
        L.lbf_evaluate_noalloc(tiny[:4], tiny[:4], tiny, None, None, tiny[:3], tiny[:1])
