"""The paper's numerical examples (Sec. 6) through the C ABI, on synthetic stand-ins for
their geometries: point vortices in the ocean (Example 2, lbf_point_vortices) and
elliptical islands with the exact data (1/2) sum Re 1/(xi - xi_k) (Examples 1 and 3),
preconditioned and not."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import workloads as wl  # noqa: E402
from gpu_util import dev, host, plan_for, rel_l2, zeros  # noqa: E402
from paper_1306_0612_gb300 import lbfmm as L  # noqa: E402

pytestmark = pytest.mark.gpu


def test_point_vortex_in_cap_ocean_closed_form():
    """One circular island around the north pole and one vortex in the ocean: psi against
    its closed form by a planar image (the island is |xi| > R = cot(r0/2))."""
    r0, gam = 0.6, 1.7
    g = wl.star_caps(3, 1, 256, r0=[r0], amp=[0.0], kfreq=[2])
    th, ph = r0 + 0.9, 0.4
    v = np.array([[np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)]])
    t = wl.targets_off_islands(g, 64, seed=7)
    p = plan_for(g, tol=1e-13)
    u, sig, a = zeros(64), zeros(g.N), zeros(g.M)
    rc, its, rr = L.lbf_point_vortices(p, dev(v), dev([gam]), dev(t), u, sig, a)
    assert rc == L.LBF_OK
    R = 1.0 / np.tan(r0 / 2)
    xi_t = (t[:, 0] + 1j * t[:, 1]) / (1 - t[:, 2])
    nu = (v[0, 0] + 1j * v[0, 1]) / (1 - v[0, 2])
    nus = R * R / np.conj(nu)
    H = (np.log(2.0) - np.log(4.0) - np.log(np.abs(xi_t - nus) ** 2) - np.log(np.abs(nu) ** 2 / R ** 2)
         + np.log(1 + R * R) + np.log(1 + np.abs(nu) ** 2)) / (4 * np.pi)
    G = (np.log(2.0) - np.log(np.sum((t - v) ** 2, axis=1))) / (4 * np.pi)
    exact = gam * (G - H)
    assert np.max(np.abs(host(u) - exact)) < 1e-10 * np.max(np.abs(exact))


@pytest.mark.parametrize("rotate", [False, True])
def test_point_vortices_many_islands_match_oracle(oracle, rotate):
    """Sixteen star caps and 5 vortices in the ocean, psi = 0 on every curve: against the
    oracle's decomposition psi* + sum Gamma_j G(., v_j) (dense solve), with the pole on
    island 0 given as data or as the plan's rotation."""
    g = wl.config_geometry("C2", nodes=128, pole=None if rotate else "first")
    R = wl.rotation_to_pole(g.centres[0]) if rotate else None
    t = wl.targets_off_islands(g, 90, seed=5)
    v, t = t[:5], t[5:]
    gam = np.random.default_rng(3).uniform(-2 * np.pi, 2 * np.pi, 5)
    p = plan_for(g, tol=1e-13, rotation=R)
    u, sig, a = zeros(len(t)), zeros(g.N), zeros(g.M)
    rc, its, rr = L.lbf_point_vortices(p, dev(v), dev(gam), dev(t), u, sig, a)
    assert rc == L.LBF_OK
    ref = oracle.point_vortices(g, v, gam, t)
    assert np.max(np.abs(host(u) - ref)) < 1e-9 * np.max(np.abs(ref))


def _ellipse_solve(g, **opt):
    data = zeros(g.N)
    L.lbf_dipole_sum(dev(g.x), dev(g.centres[1:]), data)
    p = plan_for(g, **opt)
    sig, a = zeros(g.N), zeros(g.M)
    rc, its, rr = L.lbf_gmres_solve(p, data, sig, a)
    t = wl.targets_off_islands(g, 75, seed=2)
    u, ue = zeros(75), zeros(75)
    L.lbf_evaluate(p, sig, a, dev(t), u)
    L.lbf_dipole_sum(dev(t), dev(g.centres[1:]), ue)
    err = float((u - ue).abs().max() / ue.abs().max())
    return rc, its, err, host(sig)


def test_dipole_sum_matches_oracle(oracle):
    g = wl.ellipse_islands(4, 30, 64)
    t = wl.targets_off_islands(g, 200, seed=3)
    out = zeros(200)
    L.lbf_dipole_sum(dev(t), dev(g.centres), out)
    ref = oracle.dipole_data(t, g.centres)
    assert np.max(np.abs(host(out) - ref)) < 1e-13 * np.max(np.abs(ref))


def test_ellipse_islands_iterations_do_not_grow_with_n():
    """Fifteen elliptical islands (Example 1): preconditioned iterations do not depend on
    the nodes per island, the error falls spectrally; without the preconditioner GMRES
    needs more iterations for the same solution."""
    its, errs = [], []
    for n in (64, 128, 256):
        g = wl.ellipse_islands(1, 15, n)
        rc, it, err, sig = _ellipse_solve(g, tol=1e-11)
        assert rc == L.LBF_OK
        its.append(it)
        errs.append(err)
        if n == 128:
            rc2, it2, err2, sig2 = _ellipse_solve(g, tol=1e-11, precond=0)
            assert rc2 == L.LBF_OK and it2 > it
            assert rel_l2(sig2, sig) < 1e-9
    assert max(its) - min(its) <= 2
    assert errs[2] < errs[0] and errs[2] < 1e-8
