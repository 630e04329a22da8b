"""Pins of the oracle's dense adjoint gradient (CPU): the inverse projection against
the generator's analytic curve derivatives, the numpy 3D-form matrices against the
C oracle, and the complex-step gradient against central differences of the dense
forward map (a different computation: repeated dense solves)."""
import numpy as np
import pytest

import oracle
import workloads as wl
from helpers import planar_nodes, rel_l2
from oracle import adjoint as adj


def _case(seed=7, M=3, nodes=24, T=40):
    g = wl.star_caps(seed, M, nodes)
    xi, d1, d2 = planar_nodes(g)
    t = wl.targets_off_islands(g, T, seed=seed + 1)
    src, gam, _ = wl.pair_sources(g, 0, min(1, M - 1))
    data = oracle.green_sum(g.x, src, gam)
    return g, xi, d1, d2, t, data


def test_sphere_from_plane_inverts_the_projection():
    g, xi, d1, d2, _, _ = _case()
    x, dx, d2x = adj.sphere_from_plane(xi[:, 0], xi[:, 1], d1[:, 0], d1[:, 1], d2[:, 0], d2[:, 1])
    assert np.max(np.abs(x - g.x)) < 1e-13
    assert np.max(np.abs(dx - g.dx)) < 1e-12 * np.max(np.abs(g.dx))
    assert np.max(np.abs(d2x - g.d2x)) < 1e-11 * np.max(np.abs(g.d2x))


def test_dense_matrices_match_the_c_oracle():
    g, _, _, _, t, _ = _case()
    A = adj.dense_system(g.island_ptr, g.x, g.dx, g.d2x, g.centres)
    assert np.max(np.abs(A - oracle.matrix(g))) < 1e-13 * np.max(np.abs(A))
    rng = np.random.default_rng(1)
    s, a = rng.standard_normal(g.N), rng.standard_normal(g.M)
    C = adj.evaluation_matrix(g.island_ptr, g.x, g.dx, g.centres, t)
    u = oracle.evaluate(g, s, a, t)
    assert rel_l2(C @ np.concatenate([s, a]), u) < 1e-13


@pytest.mark.parametrize("M", [1, 3])
def test_gradient_matches_central_differences(M):
    g, xi, d1, d2, t, data = _case(M=M)
    T = len(t)

    def loss(u):
        return float(np.mean(u ** 2))

    gg, gx, u = adj.gradient(g.island_ptr, xi, d1, d2, g.centres, t, data, lambda u: 2 * u / T)
    assert np.allclose(u, adj.forward(g.island_ptr, xi, d1, d2, g.centres, t, data), rtol=1e-13)
    rng = np.random.default_rng(3)
    h = 1e-6
    for _ in range(4):
        dg = rng.standard_normal(g.N)
        dx = rng.standard_normal((g.N, 2)) * 1e-2
        fp = loss(adj.forward(g.island_ptr, xi + h * dx, d1, d2, g.centres, t, data + h * dg))
        fm = loss(adj.forward(g.island_ptr, xi - h * dx, d1, d2, g.centres, t, data - h * dg))
        fd = (fp - fm) / (2 * h)
        an = gg @ dg + np.sum(gx * dx)
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
