"""The adjoint path through the C ABI: transposed operators, the adjoint GMRES solve,
the transposed evaluation and the gradient with respect to Dirichlet data and planar
node positions (the autograd wrapper), against the oracle's dense matrices and its
complex-step adjoint gradient, and against central differences of the GPU forward map.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import workloads as wl  # noqa: E402
from gpu_util import dev, host, plan_for, rel_l2, zeros  # noqa: E402
from helpers import planar_nodes  # noqa: E402
from oracle import adjoint as adj  # noqa: E402
from paper_1306_0612_gb300 import autograd as AG  # noqa: E402
from paper_1306_0612_gb300 import lbfmm as L  # noqa: E402

pytestmark = pytest.mark.gpu

MATVEC_TOL = 1e-10


def _ragged(seed=31):
    return wl.star_caps(seed, 5, [96, 33, 250, 64, 17], r0=[0.3, 0.15, 0.35, 0.2, 0.1],
                        amp=[0.2, 0.1, 0.25, 0.0, 0.15], kfreq=[3, 2, 5, 4, 2])


@pytest.mark.parametrize("matvec", [L.LBF_MATVEC_DIRECT, L.LBF_MATVEC_FMM])
def test_transposed_ops_match_dense(matvec):
    g = _ragged()
    p = plan_for(g, matvec=matvec, leaf_size=8)
    A = oracle.matrix(g)
    N = g.N
    Pm = oracle.preconditioner_matrix(A, N)
    v = np.random.default_rng(8).standard_normal(N + g.M)
    out = zeros(N + g.M)
    L.lbf_apply(p, L.LBF_OP_FULL | L.LBF_OP_TRANSPOSE, dev(v), out)
    assert rel_l2(host(out), A.T @ v) < MATVEC_TOL
    L.lbf_apply(p, L.LBF_OP_PRECONDITIONED | L.LBF_OP_TRANSPOSE, dev(v), out)
    assert rel_l2(host(out), np.linalg.solve(Pm.T, A.T @ v)) < MATVEC_TOL
    o2 = zeros(N)
    L.lbf_apply(p, L.LBF_OP_K_ONLY | L.LBF_OP_TRANSPOSE, dev(v[:N]), o2)
    assert rel_l2(host(o2), A[:N, :N].T @ v[:N]) < MATVEC_TOL


def test_transposed_fp32_operator_is_single_precision():
    g = wl.config_geometry("C2")
    p = plan_for(g, precision=L.LBF_PRECISION_FP32_REFINE)
    v = np.random.default_rng(9).standard_normal(g.N + g.M)
    o64, o32 = zeros(g.N + g.M), zeros(g.N + g.M)
    op = L.LBF_OP_PRECONDITIONED | L.LBF_OP_TRANSPOSE
    L.lbf_apply(p, op, dev(v), o64)
    L.lbf_apply(p, op | L.LBF_OP_FP32, dev(v), o32)
    assert 1e-12 < rel_l2(host(o32), host(o64)) < 1e-5


@pytest.mark.parametrize("precision", [L.LBF_PRECISION_FP64, L.LBF_PRECISION_FP32_REFINE])
def test_adjoint_solve_matches_dense(precision):
    g = wl.config_geometry("C2", nodes=128)
    p = plan_for(g, tol=1e-12, precision=precision)
    A = oracle.matrix(g)
    r = np.random.default_rng(10).standard_normal(g.N + g.M)
    lam = zeros(g.N + g.M)
    rc, its, rr = L.lbf_gmres_solve_transpose(p, dev(r), lam)
    assert rc == L.LBF_OK and rr <= 1e-12
    assert rel_l2(host(lam), np.linalg.solve(A.T, r)) < 1e-9


def test_evaluate_transpose_matches_dense():
    g = wl.config_geometry("C2", nodes=128)
    p = plan_for(g)
    t = wl.targets_off_islands(g, 300, seed=4)
    C = adj.evaluation_matrix(g.island_ptr, g.x, g.dx, g.centres, t)
    ub = np.random.default_rng(11).standard_normal(len(t))
    sb, ab = zeros(g.N), zeros(g.M)
    L.lbf_evaluate_transpose(p, dev(t), dev(ub), sb, ab)
    ref = C.T @ ub
    assert rel_l2(host(sb), ref[:g.N]) < 1e-12
    assert rel_l2(host(ab), ref[g.N:]) < 1e-12


def _planar_case(seed, M, nodes, T):
    g = wl.star_caps(seed, M, nodes)
    xi, d1, d2 = planar_nodes(g)
    t = wl.targets_off_islands(g, T, seed=seed + 1)
    src, gam, _ = wl.pair_sources(g, 0, 1)
    data = oracle.green_sum(g.x, src, gam)
    return g, xi, d1, d2, t, data


def _gpu_loss_and_grad(g, xi, d1, d2, t, data, opt):
    gt = dev(data).requires_grad_(True)
    xt = dev(xi).reshape(g.N, 2).requires_grad_(True)
    u = AG.solve_evaluate(gt, xt, dev(d1), dev(d2), dev(g.centres), dev(t), g.island_ptr, opt)
    loss = (u ** 2).mean()
    loss.backward()
    return float(loss), host(gt.grad), host(xt.grad), host(u)


def test_gradient_matches_dense_oracle():
    """16 islands x 128 nodes (N = 2048): the autograd gradient against the oracle's
    dense complex-step adjoint gradient, loss = mean u^2 at 1024 targets."""
    g, xi, d1, d2, t, data = _planar_case(5, 16, 128, 1024)
    opt = L.lbf_default_options(tol=1e-13)
    loss, gg, gx, u = _gpu_loss_and_grad(g, xi, d1, d2, t, data, opt)
    T = len(t)
    rg, rx, ru = adj.gradient(g.island_ptr, xi, d1, d2, g.centres, t, data, lambda v: 2 * v / T)
    assert rel_l2(u, ru) < 1e-10
    assert rel_l2(gg, rg) < 1e-8
    assert rel_l2(gx, rx) < 1e-8


def test_gradient_matches_central_differences_c5():
    """256 islands x 512 nodes (N = 131072), 4096 targets, loss = mean u^2: the
    directional derivative of the autograd gradient along 32 random directions in
    (g, xi) against central differences of the GPU forward map, h = 1e-6."""
    g, xi, d1, d2, t, data = _planar_case(5, 256, 512, 4096)
    opt = L.lbf_default_options(tol=1e-13)
    loss, gg, gx, _ = _gpu_loss_and_grad(g, xi, d1, d2, t, data, opt)
    cen, tt, dd1, dd2 = dev(g.centres), dev(t), dev(d1), dev(d2)

    def fwd(dv, xv):
        with torch.no_grad():
            u = AG.solve_evaluate(dev(dv), dev(xv).reshape(g.N, 2), dd1, dd2, cen, tt,
                                  g.island_ptr, opt)
        return float((u ** 2).mean())

    rng = np.random.default_rng(12)
    h = 1e-6
    scale_x = 1e-2 * np.std(xi)
    worst = 0.0
    for _ in range(32):
        dg = rng.standard_normal(g.N) * np.std(data)
        dx = rng.standard_normal((g.N, 2)) * scale_x
        fd = (fwd(data + h * dg, xi + h * dx) - fwd(data - h * dg, xi - h * dx)) / (2 * h)
        an = gg @ dg + np.sum(gx * dx)
        worst = max(worst, abs(fd - an) / abs(an))
    assert worst < 1e-4, worst
