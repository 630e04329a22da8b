"""The Schur complement S = D - F E of the border (Sec. 5, Eq. matrix_eqns_c) applied
through its double-float LU factors (LBF_SCHUR_LU, the default above 1024 islands)
instead of the Gauss-Jordan inverse in double.

Tolerance: the LU path's S^-1 carries rounding of about cond(S) 2^-46 (double-float
factorisation, ~48-bit significands, with some growth), so the preconditioned operator
is compared with the oracle's dense P^-1 A at max(1e-10, 64 cond(S) 2^-46), cond(S)
taken from the oracle's own S.  Solves are unaffected: GMRES meets its tolerance on the
exact operator whichever S^-1 the preconditioner uses, so their results are compared
with the Gauss-Jordan path's at the solution tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import workloads as wl  # noqa: E402
from gpu_util import dev, host, plan_for, rel_l2, zeros  # noqa: E402
from paper_1306_0612_gb300 import lbfmm as L  # noqa: E402

pytestmark = pytest.mark.gpu


def _lu_tol(A, N):
    S = A[N:, N:] - A[N:, :N] @ A[:N, N:]
    return max(1e-10, 64 * np.linalg.cond(S) * 2.0 ** -46)


@pytest.mark.parametrize("M,nodes", [(200, 8), (67, 12)])
def test_lu_preconditioned_op_matches_dense(oracle, M, nodes):
    g = wl.star_caps(41, M, nodes)
    A = oracle.matrix(g)
    Pm = oracle.preconditioner_matrix(A, g.N)
    tol = _lu_tol(A, g.N)
    p = plan_for(g, leaf_size=8, schur=L.LBF_SCHUR_LU)
    v = np.random.default_rng(4).standard_normal(g.N + g.M)
    out = zeros(g.N + g.M)
    L.lbf_apply(p, L.LBF_OP_PRECONDITIONED, dev(v), out)
    assert rel_l2(host(out), np.linalg.solve(Pm, A @ v)) < tol
    L.lbf_apply(p, L.LBF_OP_PRECONDITIONED | L.LBF_OP_TRANSPOSE, dev(v), out)
    assert rel_l2(host(out), np.linalg.solve(Pm.T, A.T @ v)) < tol
    # the same operator from the Gauss-Jordan inverse
    q = plan_for(g, leaf_size=8, schur=L.LBF_SCHUR_GJ)
    o2 = zeros(g.N + g.M)
    L.lbf_apply(q, L.LBF_OP_PRECONDITIONED, dev(v), o2)
    assert rel_l2(host(o2), np.linalg.solve(Pm, A @ v)) < 1e-10


def test_lu_singular_shared_centre():
    g = wl.config_geometry("C2", nodes=64)
    c = g.centres.copy()
    c[2] = c[1]
    with pytest.raises(L.LbfError) as e:
        L.lbf_plan_create(g.island_ptr, dev(g.x), dev(g.dx), dev(g.d2x), dev(c),
                          opt=L.lbf_default_options(schur=L.LBF_SCHUR_LU))
    assert e.value.status == L.LBF_ESINGULAR


@pytest.mark.parametrize("precision,tol,agree", [(L.LBF_PRECISION_FP64, 1e-12, 1e-8),
                                                  (L.LBF_PRECISION_FP32_REFINE, 1e-10, 1e-7)])
def test_lu_solve_many_islands_matches_gauss_jordan(precision, tol, agree):
    """2048 islands (the LU path by default) against the same solve with the
    Gauss-Jordan inverse: the same bordered system, each solved to a preconditioned
    relative residual below tol.  The preconditioned operator is applied as
    x + P^-1 [2K sigma; 0], so a solve meets the system whose Schur block is the inverse
    of the S^-1 it applies: the Gauss-Jordan path's double S^-1, unrefined, carries about
    cond(S) 2^-53 (cond(S) ~ 1e8 at 2048 star caps, so ~1e-8), the LU path's refined one
    less; the two solutions agree to that, whatever tol (1e-12 and 1e-13 give the same
    difference)."""
    g = wl.star_caps(3, 2048, 64)
    src, gam, _ = wl.pair_sources(g, 0, 1)
    data = zeros(g.N)
    L.lbf_green_sum(dev(g.x), dev(src), dev(gam), data)
    res = {}
    for schur in (L.LBF_SCHUR_AUTO, L.LBF_SCHUR_GJ):
        p = plan_for(g, tol=tol, precision=precision, schur=schur)
        sig, a = zeros(g.N), zeros(g.M)
        rc, its, rr = L.lbf_gmres_solve(p, data, sig, a)
        assert rc == L.LBF_OK and rr < tol
        res[schur] = (host(sig), host(a), its)
    s_lu, a_lu, it_lu = res[L.LBF_SCHUR_AUTO]
    s_gj, a_gj, it_gj = res[L.LBF_SCHUR_GJ]
    assert rel_l2(s_lu, s_gj) < agree
    assert rel_l2(a_lu, a_gj) < agree
    if precision == L.LBF_PRECISION_FP64:  # the same Krylov iteration to rounding
        assert abs(it_lu - it_gj) <= 2


@pytest.mark.parametrize("M,nodes", [(1100, 32), (2500, 128)])
def test_preconditioner_reproduces_multiplier_only_vectors(M, nodes):
    """P = [[I, E], [F, D]] agrees with A = [[I + 2K, E], [F, D]] on vectors [0; y], so
    P^-1 A [0; y] = [0; y] whatever S = D - F E is: the factors of S (the LU's trailing
    updates on the tensor cores included) are checked through S^-1 S y = y at sizes beyond
    the dense oracle.  Any S^-1 in double carries about cond(S) eps of S y's rounding (up
    to ~1e-8 here), so the LU path (one refinement step against the double S) is held to
    ten times the Gauss-Jordan inverse's own deviation, and both to 1e-6."""
    g = wl.star_caps(7, M, nodes)
    y = np.random.default_rng(11).standard_normal(M)
    v = np.concatenate([np.zeros(g.N), y])
    err, sig = {}, {}
    for schur in (L.LBF_SCHUR_LU, L.LBF_SCHUR_GJ):
        p = plan_for(g, schur=schur)
        out = zeros(g.N + g.M)
        L.lbf_apply(p, L.LBF_OP_PRECONDITIONED, dev(v), out)
        o = host(out)
        err[schur] = np.linalg.norm(o[g.N:] - y) / np.linalg.norm(y)
        sig[schur] = np.linalg.norm(o[:g.N]) / np.sqrt(g.N) / (np.linalg.norm(y) / np.sqrt(M))
    assert err[L.LBF_SCHUR_GJ] < 1e-6 and sig[L.LBF_SCHUR_GJ] < 1e-6, (err, sig)
    assert err[L.LBF_SCHUR_LU] < max(1e-9, 10 * err[L.LBF_SCHUR_GJ]), err
    assert sig[L.LBF_SCHUR_LU] < max(1e-9, 10 * sig[L.LBF_SCHUR_GJ]), sig
