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
    res = L.lbf_batch_run(inst, opt=opt, nworkers=4, lockstep=False)
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


# ---- right-hand sides of one geometry in lockstep (lbf_gmres_solve_many) ------------------

def _lockstep_case(M, nodes, nrhs, seed):
    """A star-cap geometry and nrhs right-hand sides of mixed difficulty: Green's-pair
    data (the paper's exact solutions), seeded noise (needs more iterations), and one zero
    right-hand side (converged at the start)."""
    g = wl.star_caps(seed, M, nodes)
    rng = np.random.default_rng(seed + 1)
    rows = []
    for k in range(nrhs):
        if k == 2:
            rows.append(np.zeros(g.N))
        elif k % 3 == 1:
            rows.append(rng.standard_normal(g.N))
        else:
            p, gam, _ = wl.random_pair_sources(g, rng)
            rows.append(oracle.green_sum(g.x, p, gam))
    return g, np.stack(rows)


def _rows(t, k, n):
    return host(t)[k * n:(k + 1) * n]


def _separate(p, g, data):
    out = []
    for k in range(data.shape[0]):
        sig, a = zeros(g.N), zeros(g.M)
        rc, its, rr = L.lbf_gmres_solve(p, dev(data[k]), sig, a)
        out.append((rc, its, rr, host(sig), host(a)))
    return out


FP64, IR = L.LBF_PRECISION_FP64, L.LBF_PRECISION_FP32_REFINE


# fmm64 0: the accurate operator in native double (its lockstep near field is k_near_multi);
# 1: in double-float (a leaf pass per right-hand side)
@pytest.mark.parametrize("M,nodes,nrhs,restart,graphs,matvec,precision,depth,fmm64", [
    (6, 96, 5, 50, 1, L.LBF_MATVEC_FMM, FP64, 30, 0),     # graph-replayed steps, one cycle
    (6, 96, 5, 50, 1, L.LBF_MATVEC_FMM, FP64, 30, 1),     # the same, double-float operator
    (5, 120, 4, 6, 1, L.LBF_MATVEC_FMM, FP64, 30, 0),     # restarts every 6 steps
    (4, 80, 18, 50, 1, L.LBF_MATVEC_FMM, FP64, 30, 0),    # two lockstep groups (16 + 2)
    (4, 80, 18, 50, 1, L.LBF_MATVEC_FMM, FP64, 30, 1),
    (3, 100, 3, 50, 0, L.LBF_MATVEC_FMM, FP64, 30, 0),    # steps launched one by one
    (4, 150, 6, 50, 1, L.LBF_MATVEC_FMM, FP64, 3, 0),     # depth cap: leaves of well over 64 nodes
    (1, 256, 3, 50, 1, L.LBF_MATVEC_DIRECT, FP64, 30, 0), # one island, direct sums
    (6, 96, 5, 50, 1, L.LBF_MATVEC_FMM, IR, 30, 0),       # refinement: FP64 residuals, float inner solves
    (6, 96, 5, 50, 1, L.LBF_MATVEC_FMM, IR, 30, 1),
    (5, 120, 7, 8, 0, L.LBF_MATVEC_FMM, IR, 30, 0),       # refinement with inner restarts, no graphs
])
def test_lockstep_equals_separate_solves(M, nodes, nrhs, restart, graphs, matvec, precision, depth,
                                         fmm64):
    """Each right-hand side of a lockstep solve runs the kernels of a solve on its own,
    except the FMM's near field, which the lockstep group sums in one pass sharing each
    pair's geometry (k_near_multi: c (w x dz) / |dz|^2 formed as c times the pair's
    factor instead of (c w) x dz, a different rounding).  So the direct-sum plans agree
    bit for bit, and the FMM plans to the solver's tolerance: iterations within 2 and
    solutions within 1e-9 (tol 1e-12 on the preconditioned residual, the refinement's
    included: its FP64 residual decides when it stops)."""
    g, data = _lockstep_case(M, nodes, nrhs, seed=70 + M)
    p = plan_for(g, tol=1e-12, restart=restart, graphs=graphs, matvec=matvec, precision=precision,
                 max_depth=depth, fmm64=fmm64)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        sig, a = zeros(nrhs * g.N), zeros(nrhs * g.M)
        rc, its, rr = L.lbf_gmres_solve_many(p, dev(data), sig, a, stream=s)
        s.synchronize()
        ref = _separate(p, g, data)
    assert rc == L.LBF_OK
    assert its[2] == 0 and rr[2] == 0.0  # the zero right-hand side
    assert len(set(its)) > 1  # the right-hand sides stopped at different steps
    exact = matvec == L.LBF_MATVEC_DIRECT
    for k, (rck, itk, rrk, sk, ak) in enumerate(ref):
        assert rck == L.LBF_OK and rr[k] <= 1e-12
        if exact:
            assert its[k] == itk and rr[k] == rrk
            assert np.array_equal(_rows(sig, k, g.N), sk)
            assert np.array_equal(_rows(a, k, g.M), ak)
        elif k != 2:
            assert abs(its[k] - itk) <= 2
            assert rel_l2(_rows(sig, k, g.N), sk) < 1e-9
            assert rel_l2(_rows(a, k, g.M), ak) < 1e-9


@pytest.mark.parametrize("precision,fmm64", [(FP64, 0), (FP64, 1), (IR, 0)])
def test_lockstep_matches_oracle_dense_solve(precision, fmm64):
    g, data = _lockstep_case(5, 88, 6, seed=91)
    p = plan_for(g, tol=1e-12, precision=precision, fmm64=fmm64)
    sig, a = zeros(6 * g.N), zeros(6 * g.M)
    rc, its, rr = L.lbf_gmres_solve_many(p, dev(data), sig, a)
    assert rc == L.LBF_OK and max(rr) <= 1e-12
    A = oracle.matrix(g)
    for k in range(6):
        z = np.linalg.solve(A, np.concatenate([2 * data[k], np.zeros(g.M)]))
        if k == 2:
            assert not np.any(host(sig)[k * g.N:(k + 1) * g.N])
            continue
        assert rel_l2(host(sig)[k * g.N:(k + 1) * g.N], z[:g.N]) < 1e-9
        assert rel_l2(host(a)[k * g.M:(k + 1) * g.M], z[g.N:]) < 1e-9


def test_lockstep_short_workspace_and_sequential_plans():
    g, data = _lockstep_case(4, 64, 3, seed=93)
    p = plan_for(g, tol=1e-12)
    need = L.lbf_gmres_workspace_many(p, 3)
    assert need > 0
    short = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(L.LbfError):
        L.lbf_gmres_solve_many(p, dev(data), zeros(3 * g.N), zeros(3 * g.M), work=short)
    # a plan that applies S^-1 by LU factors takes no lockstep workspace and solves the
    # right-hand sides one after another
    g, data = _lockstep_case(67, 12, 3, seed=95)
    q = plan_for(g, tol=1e-12, leaf_size=8, schur=L.LBF_SCHUR_LU)
    assert L.lbf_gmres_workspace_many(q, 3) == 0
    sig, a = zeros(3 * g.N), zeros(3 * g.M)
    rc, its, rr = L.lbf_gmres_solve_many(q, dev(data), sig, a)
    for k, (rck, itk, rrk, sk, ak) in enumerate(_separate(q, g, data)):
        assert its[k] == itk and np.array_equal(_rows(sig, k, g.N), sk)


@pytest.mark.parametrize("precision,fmm64", [(FP64, 0), (FP64, 1), (IR, 0)])
def test_batch_lockstep_matches_oracle(precision, fmm64):
    """The batch runner's lockstep solves (the default) against the oracle's dense solve
    and the evaluation at the targets against the one-after-another runs."""
    inst = _instances(count=6, nrhs=5)
    opt = L.lbf_default_options(tol=1e-12, precision=precision, fmm64=fmm64)
    lock = L.lbf_batch_run(inst, opt=opt, nworkers=3, lockstep=True)
    seq = L.lbf_batch_run(inst, opt=opt, nworkers=3, lockstep=False)
    for ins, a, b in zip(inst, lock, seq):
        g = ins["geom"]
        assert a["status"] == b["status"] == L.LBF_OK and a["max_rel_res"] <= 1e-12
        A = oracle.matrix(g)
        for k in range(ins["data"].shape[0]):
            z = np.linalg.solve(A, np.concatenate([2 * ins["data"][k], np.zeros(g.M)]))
            assert rel_l2(host(a["sigma"][k]), z[:g.N]) < 1e-9
            assert rel_l2(host(a["u"][k]), host(b["u"][k])) < 1e-9
