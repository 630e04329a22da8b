"""Parity at the paths and sizes the benchmark runs (through the C ABI):

* the bordered operator (Eq. matrix_eqns) with the border on, at 1024 islands x 1024
  nodes, on sampled node rows, constraint rows (Eq. disc_constr) and the row of
  Eq. (sum_ak), in both arithmetics of the accurate FMM;
* the preconditioned operator P^-1 A at 1024 islands (16 nodes each), against P^-1
  applied on the host by block elimination with the oracle's E, F and D;
* the density operator I + 2K at 16,384 islands x 1024 nodes (N = 16,777,216) on
  sampled rows, in native double, double-float and float;
* the full step of the benchmark at that size (plan with the LU of the Schur
  complement, GMRES to 1e-10, evaluation) against the exact Green's-pair solution.

Tolerances: FP64 matvec rel-l2 1e-10 (the FMM truncation is ~1e-12 at p = 26); the
preconditioned operator max(1e-10, 16 cond(S) 2^-52), since the host's own S^-1 carries
that rounding; float operator 2e-6; solutions 1e-9 against the exact data.
"""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import workloads as wl  # noqa: E402
from gpu_util import dev, host, plan_for, rel_l2, zeros  # noqa: E402
from paper_1306_0612_gb300 import lbfmm as L  # noqa: E402

pytestmark = pytest.mark.gpu

MATVEC_TOL = 1e-10
SOLVE_TOL = 1e-9


@functools.lru_cache(maxsize=2)
def _c3(M):
    return wl.star_caps(3, M, 1024)


@pytest.mark.parametrize("fmm64", [0, 1])
def test_full_bordered_operator_sampled_rows_1024_islands(oracle, fmm64):
    g = _c3(1024)
    p = plan_for(g, fmm64=fmm64)
    rng = np.random.default_rng(8)
    v = np.concatenate([rng.standard_normal(g.N), rng.standard_normal(g.M)])
    out = zeros(g.N + g.M)
    L.lbf_apply(p, L.LBF_OP_FULL, dev(v), out)
    got = host(out)
    nodes = np.sort(rng.choice(g.N, 48, replace=False))
    cons = g.N + np.sort(rng.choice(g.M - 1, 12, replace=False))
    rows = np.concatenate([nodes, cons, [g.N + g.M - 1]])
    ref = oracle.apply_rows(g, v, rows, op=0)
    assert rel_l2(got[nodes], ref[:48]) < MATVEC_TOL
    # constraint rows: island sums of sigma; the last row: sum of a (exact sums)
    assert np.max(np.abs(got[rows[48:]] - ref[48:])) < 1e-12 * np.max(np.abs(ref[48:]))


def test_preconditioned_operator_1024_islands(oracle):
    g = wl.star_caps(3, 1024, 16)
    N, M = g.N, g.M
    p = plan_for(g, leaf_size=16)
    v = np.random.default_rng(9).standard_normal(N + M)
    out = zeros(N + M)
    L.lbf_apply(p, L.LBF_OP_PRECONDITIONED, dev(v), out)
    Av = oracle.apply(g, v, 0)
    # E (N x M, the doubled multiplier columns), F (island sums of islands 2..M), D
    E = np.empty((N, M))
    for m in range(M):
        E[:, m] = 2.0 * oracle.green_sum(g.x, g.centres[m:m + 1], np.ones(1))
    isl = g.island_of_node()
    F = np.zeros((M, N))
    for k in range(1, M):
        F[k - 1, isl == k] = 1.0
    D = np.zeros((M, M))
    D[M - 1, :] = 1.0
    S = D - F @ E
    za = np.linalg.solve(S, Av[N:] - F @ Av[:N])
    ref = np.concatenate([Av[:N] - E @ za, za])
    tol = max(MATVEC_TOL, 16 * np.linalg.cond(S) * 2.0 ** -52)
    assert rel_l2(host(out), ref) < tol


@pytest.mark.parametrize("mode", ["fp64", "df64", "fp32"])
def test_density_operator_sampled_rows_16384_islands(oracle, mode):
    g = _c3(16384)
    opt = dict(border=0, fmm64=1 if mode == "df64" else 0)
    if mode == "fp32":
        opt["precision"] = L.LBF_PRECISION_FP32_REFINE
    p = plan_for(g, **opt)
    info = p.info()
    assert info["N"] == 16777216 and info["depth"] >= 22
    sig = wl.random_density(g.N, 3)
    out = zeros(g.N)
    op = L.LBF_OP_K_ONLY | (L.LBF_OP_FP32 if mode == "fp32" else 0)
    L.lbf_apply(p, op, dev(sig), out)
    rows = np.sort(np.random.default_rng(10).choice(g.N, 48, replace=False))
    ref = oracle.apply_rows(g, sig, rows, op=1)
    assert rel_l2(host(out)[rows], ref) < (2e-6 if mode == "fp32" else MATVEC_TOL)


@pytest.mark.parametrize("precision,fmm64", [(L.LBF_PRECISION_FP64, 0),
                                             (L.LBF_PRECISION_FP32_REFINE, 1)])
def test_benchmark_step_16384_islands_matches_exact_solution(oracle, precision, fmm64):
    """The benchmark's workload: 16,384 star caps x 1024 nodes, Green's-pair data with
    sources in islands 0 and 1, GMRES(50) to 1e-10, u at 256 targets."""
    g = _c3(16384)
    src, gam, _ = wl.pair_sources(g, 0, 1)
    data = zeros(g.N)
    L.lbf_green_sum(dev(g.x), dev(src), dev(gam), data)
    p = plan_for(g, tol=1e-10, precision=precision, fmm64=fmm64)
    sig, a = zeros(g.N), zeros(g.M)
    rc, its, rr = L.lbf_gmres_solve(p, data, sig, a)
    assert rc == L.LBF_OK and rr <= 1e-10
    tg = wl.targets_off_islands(g, 256, seed=17)
    u = zeros(256)
    L.lbf_evaluate(p, sig, a, dev(tg), u)
    uex = oracle.green_sum(tg, src, gam)
    assert np.max(np.abs(host(u) - uex)) / np.max(np.abs(uex)) < SOLVE_TOL
