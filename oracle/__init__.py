"""Oracle: a plain, slow FP64 CPU implementation of the Nystrom system.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import this package.  It shares no code with
the CUDA library; the two meet only through the seeded inputs of `workloads`.

Everything here follows the plain definitions (Sec. 2, Sec. 5, Appendix A):
the dense bordered matrix in the 3D sphere form (lbf_oracle.c), dense LU with
partial pivoting (LAPACK getrf through scipy, a library primitive), a direct
O(N^2) matvec, the representation formula at targets, and a reference
quadtree with brute-force interaction lists.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from types import SimpleNamespace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liblbf_oracle.so")
_lib = None

# GMRES options and FMM settings are not part of the oracle: it solves exactly.


def build(force: bool = False) -> str:
    """Compile lbf_oracle.c with gcc (no contraction of a*b+c, OpenMP rows)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.c_void_p
        i64 = C.c_int64
        lib.orc_green.restype = C.c_double
        lib.orc_green.argtypes = [P, P]
        lib.orc_entry.restype = C.c_double
        lib.orc_entry.argtypes = [i64, C.c_int, P, P, P, P, P, i64, i64]
        lib.orc_matrix.argtypes = [i64, C.c_int, P, P, P, P, P, P]
        lib.orc_apply_rows.argtypes = [i64, C.c_int, P, P, P, P, P, C.c_int, P, i64, P, P]
        lib.orc_evaluate.argtypes = [i64, C.c_int, P, P, P, P, P, P, i64, P, P]
        lib.orc_green_sum.argtypes = [i64, P, i64, P, P, P]
        lib.orc_project.argtypes = [i64, P, P]
        lib.orc_tree.restype = i64
        lib.orc_tree.argtypes = [i64, P, C.c_int, C.c_int, i64] + [P] * 11
        lib.orc_lists.restype = i64
        lib.orc_lists.argtypes = [i64, P, P, P, P, P, C.c_int, i64, P, P]
        lib.orc_num_threads.restype = C.c_int
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _geo(g):
    return (int(g.island_ptr[-1]), int(g.M), np.ascontiguousarray(g.island_ptr, dtype=np.int64),
            _f64(g.x), _f64(g.dx), _f64(g.d2x), _f64(g.centres))


def num_threads() -> int:
    return int(_L().orc_num_threads())


def green(x, y) -> float:
    """G(x, y), Sec. 1.1 Eq. (greens_func)."""
    return float(_L().orc_green(_p(_f64(x)), _p(_f64(y))))


def green_sum(points, src, gamma) -> np.ndarray:
    """sum_s gamma_s G(t, p_s) at each point t (boundary data of point sources)."""
    t, p, gm = _f64(points), _f64(src), _f64(gamma)
    out = np.empty(len(t))
    _L().orc_green_sum(len(t), _p(t), len(p), _p(p), _p(gm), _p(out))
    return out


def matrix(g) -> np.ndarray:
    """Dense bordered matrix [[I + 2K, 2E], [F, D]] (Sec. 5, Eq. matrix_eqns)."""
    N, M, ptr, x, dx, d2x, c = _geo(g)
    A = np.empty((N + M, N + M))
    _L().orc_matrix(N, M, _p(ptr), _p(x), _p(dx), _p(d2x), _p(c), _p(A))
    return A


def rhs(g, data) -> np.ndarray:
    """Right-hand side [2 g; 0] of Eq. (matrix_eqns)."""
    return np.concatenate([2.0 * _f64(data), np.zeros(g.M)])


def solve(g, data, A=None):
    """Dense LU solve of the bordered system; returns (sigma, a)."""
    from scipy.linalg import lu_factor, lu_solve

    if A is None:
        A = matrix(g)
    z = lu_solve(lu_factor(A, check_finite=False), rhs(g, data), check_finite=False)
    N = int(g.island_ptr[-1])
    return z[:N], z[N:]


def apply_rows(g, v, rows, op: int = 0) -> np.ndarray:
    """Rows of the matvec computed entry by entry (op 0: bordered, op 1: I + 2K)."""
    N, M, ptr, x, dx, d2x, c = _geo(g)
    v = _f64(v)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty(len(rows))
    _L().orc_apply_rows(N, M, _p(ptr), _p(x), _p(dx), _p(d2x), _p(c), op, _p(v), len(rows),
                        _p(rows), _p(out))
    return out


def apply(g, v, op: int = 0) -> np.ndarray:
    N = int(g.island_ptr[-1])
    n = N + g.M if op == 0 else N
    return apply_rows(g, v, np.arange(n), op)


def preconditioner_matrix(A, N: int) -> np.ndarray:
    """P = [[I, 2E], [F, D]]: the bordered matrix with the K block removed (Sec. 5)."""
    P = A.copy()
    P[:N, :N] = np.eye(N)
    return P


def evaluate(g, sigma, a, targets) -> np.ndarray:
    """u at off-curve targets, Eq. (u_multi)."""
    N, M, ptr, x, dx, d2x, c = _geo(g)
    t = _f64(targets)
    u = np.empty(len(t))
    _L().orc_evaluate(N, M, _p(ptr), _p(x), _p(dx), _p(c), _p(_f64(sigma)), _p(_f64(a)), len(t),
                      _p(t), _p(u))
    return u


def point_vortices(g, vortices, gamma, targets, A=None) -> np.ndarray:
    """psi at off-curve targets for point vortices in the ocean with psi = 0 on every
    curve (Sec. 6, Example 2): psi = psi* + sum_j Gamma_j G(., v_j), where psi* solves the
    Dirichlet problem with data -sum_j Gamma_j G(x, v_j) on the curves."""
    sigma, a = solve(g, -green_sum(g.x, vortices, gamma), A)
    return evaluate(g, sigma, a, targets) + green_sum(targets, vortices, gamma)


def dipole_data(points, sources) -> np.ndarray:
    """psi = (1/2) sum_k Re 1/(xi - xi_k) at each point (Sec. 6, Eq. exact_bcs: the exact
    solution of Examples 1 and 3), xi and xi_k the stereographic images (Sec. 3) of the
    point and of each source; a source at the north pole (xi_k infinite) adds nothing."""
    xi = project(points)
    z = xi[:, 0] + 1j * xi[:, 1]
    src = _f64(sources)
    fin = src[:, 2] < 1.0
    xk = project(src[fin])
    zk = xk[:, 0] + 1j * xk[:, 1]
    return 0.5 * np.real(1.0 / (z[:, None] - zk[None, :])).sum(axis=1)


def project(x) -> np.ndarray:
    """Stereographic projection xi = (x1 + i x2)/(1 - x3) (Sec. 3), as an N x 2 array."""
    x = _f64(x)
    xi = np.empty((len(x), 2))
    _L().orc_project(len(x), _p(x), _p(xi))
    return xi


def tree(xi, leaf: int, depth: int = 30, lists: bool = False, cap: int | None = None):
    """Reference quadtree on projected nodes xi (N x 2) and, optionally, the
    brute-force U/V/W/X lists (O(B^2): small inputs only)."""
    xi = _f64(xi)
    N = len(xi)
    if cap is None:
        cap = max(16, 8 * N)
    perm = np.empty(N, dtype=np.int64)
    keys = np.empty(N, dtype=np.uint64)
    bbox = np.empty(3)
    level = np.empty(cap, dtype=np.int32)
    ix = np.empty(cap, dtype=np.int64)
    iy = np.empty(cap, dtype=np.int64)
    parent = np.empty(cap, dtype=np.int64)
    fc = np.empty(cap, dtype=np.int64)
    nch = np.empty(cap, dtype=np.int32)
    beg = np.empty(cap, dtype=np.int64)
    end = np.empty(cap, dtype=np.int64)
    nb = _L().orc_tree(N, _p(xi), leaf, depth, cap, _p(perm), _p(keys), _p(bbox), _p(level),
                       _p(ix), _p(iy), _p(parent), _p(fc), _p(nch), _p(beg), _p(end))
    if nb < 0:
        raise RuntimeError("box capacity exceeded")
    t = SimpleNamespace(nbox=int(nb), perm=perm, keys=keys, xmin=bbox[0], ymin=bbox[1], L=bbox[2],
                        level=level[:nb].copy(), ix=ix[:nb].copy(), iy=iy[:nb].copy(),
                        parent=parent[:nb].copy(), first_child=fc[:nb].copy(),
                        nchild=nch[:nb].copy(), begin=beg[:nb].copy(), end=end[:nb].copy())
    if lists:
        for kind, name in enumerate("UVWX"):
            cap_l = max(64, nb * 64)
            ptr = np.empty(nb + 1, dtype=np.int64)
            idx = np.empty(cap_l, dtype=np.int64)
            n = _L().orc_lists(nb, _p(t.level), _p(t.ix), _p(t.iy), _p(t.parent), _p(t.nchild),
                               kind, cap_l, _p(ptr), _p(idx))
            if n < 0:
                raise RuntimeError("list capacity exceeded")
            setattr(t, name + "_ptr", ptr)
            setattr(t, name + "_idx", idx[:n].copy())
    return t
